// fengine_autotune: picks the work split of a plan by measurement. The split
// -- N1 of the four-step DFT (which fixes the phase-1 tile width and the
// phase-2 FFT length) and the slab of spectra per phase-1 / phase-2 launch
// pair -- changes how the work is divided, not what is computed,
// so the fastest split can be chosen by timing each candidate on zero-filled
// input through the public entry points.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../include/fengine.h"

namespace {

bool split_ok(long long N, int N1, int precision) {
    if (precision != FENGINE_FP32) {
        // tensor-core phase 1: radix 8 R with R physical columns per output
        // column, the only split (N2 = N / N1 <= 1024)
        const long long P = N / 8;
        return N1 == 8 * (P > 1024 ? P / 1024 : 1);
    }
    if (N % N1 || N / N1 > 1024 || N / N1 < 4) return false;
    return !(N1 > 8 && N / N1 < 512 / N1);
}

}  // namespace

extern "C" fengine_status fengine_autotune(const fengine_config *cfg, void *cuda_stream, int32_t calls,
                                           fengine_config *tuned, fengine_tune_entry *entries,
                                           int32_t max_entries, int32_t *n_entries) {
    if (!cfg || !tuned || calls < 1) return FENGINE_EINVAL;
    if (n_entries) *n_entries = 0;
    const long long N = 2LL * cfg->n_channels;
    if (cfg->n_antennas < 1 || cfg->chunk_samples <= 0 || N <= 0) return FENGINE_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // input and output shared by every candidate (their sizes do not depend on the split)
    const size_t in_bytes = (size_t)cfg->n_antennas * 2 * (size_t)(cfg->chunk_samples / 4 * 5);
    const size_t out_bytes = (size_t)cfg->n_antennas * (size_t)(cfg->chunk_samples / N) * cfg->n_channels * 4;
    uint8_t *d_in = nullptr;
    int8_t *d_out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fengine_status result = FENGINE_OK;
    if (cudaMalloc((void **)&d_in, in_bytes) != cudaSuccess || cudaMalloc((void **)&d_out, out_bytes) != cudaSuccess ||
        cudaMemsetAsync(d_in, 0, in_bytes, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaFree(d_in);
        cudaFree(d_out);
        if (e0) cudaEventDestroy(e0);
        return FENGINE_ENOMEM;
    }

    const int n1s[4] = {8, 16, 32, 64};
    const int sls[8] = {0, 32, 64, 128, 256, 512, 1024, 2048};
    float best = -1.0f;
    fengine_config best_cfg = *cfg;
    std::vector<int> seen;   // (n1, resolved slab) pairs already timed
    int count = 0;
    fengine_status last = FENGINE_OK;
    for (int n1 : n1s) {
        if (!split_ok(N, n1, cfg->precision)) continue;
        for (int sl : sls) {
            fengine_config c = *cfg;
            c.fft_n1 = n1;
            c.slab_spectra = sl;
            fengine_plan_t plan = nullptr;
            fengine_status s = fengine_plan_create(&c, &plan);
            if (s != FENGINE_OK) {
                last = s;
                continue;
            }
            fengine_info info;
            fengine_get_info(plan, &info);
            const int key = n1 * 100000 + info.slab_spectra;
            bool dup = false;
            for (int k : seen) dup = dup || k == key;
            if (dup) {
                fengine_plan_destroy(plan);
                continue;
            }
            seen.push_back(key);
            long long t = 0;
            int64_t first = 0;
            for (int i = 0; i < 2 && s == FENGINE_OK; i++, t += cfg->chunk_samples)
                s = fengine_process_chunk(plan, cuda_stream, d_in, t, nullptr, d_out, nullptr, nullptr, nullptr, &first);
            float ms = 0.0f;
            if (s == FENGINE_OK && cudaEventRecord(e0, st) == cudaSuccess) {
                for (int i = 0; i < calls && s == FENGINE_OK; i++, t += cfg->chunk_samples)
                    s = fengine_process_chunk(plan, cuda_stream, d_in, t, nullptr, d_out, nullptr, nullptr, nullptr, &first);
                if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                    s = FENGINE_ECUDA;
            }
            fengine_plan_destroy(plan);
            if (s != FENGINE_OK) {
                last = s;
                continue;
            }
            ms /= (float)calls;
            if (entries && count < max_entries) entries[count] = fengine_tune_entry{n1, info.slab_spectra, ms};
            count++;
            if (best < 0.0f || ms < best) {
                best = ms;
                best_cfg = c;
                best_cfg.slab_spectra = info.slab_spectra;
            }
        }
    }
    cudaStreamSynchronize(st);
    cudaFree(d_in);
    cudaFree(d_out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_entries) *n_entries = count < max_entries || !entries ? count : max_entries;
    if (best < 0.0f) return last != FENGINE_OK ? last : FENGINE_EUNSUPPORTED;
    *tuned = best_cfg;
    return result;
}

// ---- the tuner's pick cached in a JSON Lines file --------------------------
// One JSON object per line; a line applies to a configuration when every key
// field matches (device name and SM count, the hash of the library's sources,
// ABI version, the shape fields of fengine_config and the precision). Lines this code does not recognise are
// kept as they are when the file is rewritten.
namespace {

const char *kCacheInts[] = {"sms", "abi", "n_antennas", "n_channels", "n_taps", "chunk_samples",
                            "spectra_per_heap", "max_delay_samples", "min_delay_samples", "precision"};
constexpr int kCacheNInts = 10;

#ifndef FENGINE_SRC_HASH
#define FENGINE_SRC_HASH "unknown"
#endif

struct CacheKey {
    std::string device, src;
    long long v[kCacheNInts];
};

bool json_int(const std::string &line, const char *name, long long *out) {
    const std::string pat = std::string("\"") + name + "\":";
    const size_t at = line.find(pat);
    if (at == std::string::npos) return false;
    const char *p = line.c_str() + at + pat.size();
    char *end = nullptr;
    const long long v = std::strtoll(p, &end, 10);
    if (end == p) return false;
    *out = v;
    return true;
}

bool json_str(const std::string &line, const char *name, std::string *out) {
    const std::string pat = std::string("\"") + name + "\": \"";
    const size_t at = line.find(pat);
    if (at == std::string::npos) return false;
    const size_t b = at + pat.size(), e = line.find('"', b);
    if (e == std::string::npos) return false;
    *out = line.substr(b, e - b);
    return true;
}

bool cache_key(const fengine_config *cfg, CacheKey *k) {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return false;
    k->device = prop.name;
    k->src = FENGINE_SRC_HASH;
    for (char &ch : k->device)
        if (ch == '"' || ch == '\\' || (unsigned char)ch < 0x20) ch = '_';
    const long long vals[kCacheNInts] = {prop.multiProcessorCount, fengine_abi_version(), cfg->n_antennas,
                                         cfg->n_channels, cfg->n_taps, (long long)cfg->chunk_samples,
                                         cfg->spectra_per_heap, (long long)cfg->max_delay_samples,
                                         (long long)cfg->min_delay_samples, (long long)cfg->precision};
    for (int i = 0; i < kCacheNInts; ++i) k->v[i] = vals[i];
    return true;
}

bool line_matches(const std::string &line, const CacheKey &k) {
    std::string dev, src;
    if (!json_str(line, "device", &dev) || dev != k.device) return false;
    if (!json_str(line, "src", &src) || src != k.src) return false;
    for (int i = 0; i < kCacheNInts; ++i) {
        long long v;
        if (!json_int(line, kCacheInts[i], &v) || v != k.v[i]) return false;
    }
    return true;
}

}  // namespace

extern "C" fengine_status fengine_autotune_cached(const fengine_config *cfg, void *cuda_stream, int32_t calls,
                                                  const char *cache_path, fengine_config *tuned,
                                                  int32_t *from_cache) {
    if (!cfg || !tuned || !cache_path || !*cache_path || calls < 1) return FENGINE_EINVAL;
    if (from_cache) *from_cache = 0;
    CacheKey key;
    if (!cache_key(cfg, &key)) return FENGINE_ECUDA;
    std::vector<std::string> lines;
    if (FILE *f = std::fopen(cache_path, "r")) {
        char buf[1024];
        std::string cur;
        while (std::fgets(buf, sizeof buf, f)) {
            cur += buf;
            if (!cur.empty() && cur.back() == '\n') {
                cur.pop_back();
                lines.push_back(cur);
                cur.clear();
            }
        }
        if (!cur.empty()) lines.push_back(cur);
        std::fclose(f);
    }
    for (const std::string &line : lines) {
        long long n1, sl;
        if (!line_matches(line, key) || !json_int(line, "fft_n1", &n1) || !json_int(line, "slab_spectra", &sl))
            continue;
        fengine_config c = *cfg;
        c.fft_n1 = (int32_t)n1;
        c.slab_spectra = (int32_t)sl;
        // a cached split must still make a valid plan (the library may have
        // changed the set of splits it supports)
        fengine_plan_t plan = nullptr;
        if (fengine_plan_create(&c, &plan) != FENGINE_OK) continue;
        fengine_plan_destroy(plan);
        *tuned = c;
        if (from_cache) *from_cache = 1;
        return FENGINE_OK;
    }
    fengine_tune_entry entries[64];
    int32_t n = 0;
    const fengine_status s = fengine_autotune(cfg, cuda_stream, calls, tuned, entries, 64, &n);
    if (s != FENGINE_OK) return s;
    float ms = 0.0f;
    for (int i = 0; i < n; ++i)
        if (entries[i].fft_n1 == tuned->fft_n1 && entries[i].slab_spectra == tuned->slab_spectra) ms = entries[i].ms_per_call;
    char rec[1024];
    int len = std::snprintf(rec, sizeof rec, "{\"device\": \"%s\", \"src\": \"%s\"", key.device.c_str(),
                            key.src.c_str());
    for (int i = 0; i < kCacheNInts && len > 0 && len < (int)sizeof rec; ++i)
        len += std::snprintf(rec + len, sizeof rec - len, ", \"%s\": %lld", kCacheInts[i], key.v[i]);
    if (len > 0 && len < (int)sizeof rec)
        len += std::snprintf(rec + len, sizeof rec - len, ", \"fft_n1\": %d, \"slab_spectra\": %d, \"ms_per_call\": %.4f}",
                             tuned->fft_n1, tuned->slab_spectra, (double)ms);
    if (len <= 0 || len >= (int)sizeof rec) return FENGINE_OK;   // the pick stands; nothing cached
    std::vector<std::string> keep;
    for (const std::string &line : lines)
        if (!line_matches(line, key)) keep.push_back(line);
    keep.push_back(rec);
    // write beside the file and rename over it, so a reader sees the old or
    // the new file, never a partial one
    const std::string tmp = std::string(cache_path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return FENGINE_EIO;
    bool ok = true;
    for (const std::string &line : keep) ok = ok && std::fprintf(f, "%s\n", line.c_str()) > 0;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), cache_path) != 0) {
        std::remove(tmp.c_str());
        return FENGINE_EIO;
    }
    return FENGINE_OK;
}
