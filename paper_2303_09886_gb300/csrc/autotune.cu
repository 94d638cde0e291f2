// fengine_autotune: picks the work split of a plan by measurement. The split
// -- N1 of the four-step DFT (which fixes the phase-1 tile width and the
// phase-2 FFT length) and the slab of spectra per phase-1 / phase-2 launch
// pair -- changes how the work is divided, not what is computed,
// so the fastest split can be chosen by timing each candidate on zero-filled
// input through the public entry points.
#include <cuda_runtime.h>

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
