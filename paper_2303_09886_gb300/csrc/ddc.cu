// Narrow-band front end: the down-converter that feeds a narrow-band plan.
// Sec. 6 names a narrow-band mode with a low-pass filter before the PFB; the
// definition here (mix to baseband, low-pass, move the band's lower edge to
// 0, real part, decimate by D/2, requantise to 10 bits) is the library's
// reading of it, stated in include/fengine.h.
//
// One CTA computes 2048 consecutive outputs of one stream, 16 per thread. The
// input samples its outputs need are decoded once into shared memory, stored
// as D/2 phase planes (plane p holds the samples whose offset is p mod D/2),
// so that every tap of an output reads one plane, and a thread's 8 outputs
// share a sliding window of that plane in registers. The low-pass taps carry the mixing factor,
// h[u] exp(2 pi i fc u) (complex, computed in FP64 on the host), so each
// output is a complex dot product over the taps followed by one rotation
// exp(2 pi i (j/4 - fc i0)) whose phase is reduced in FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "../../include/fengine.h"
#include "fe_internal.cuh"

namespace {

constexpr int kDdcThreads = 128;
constexpr int kDdcPer = 16;                         // consecutive outputs per thread
constexpr int kDdcOut = kDdcThreads * kDdcPer;      // outputs per CTA

struct DdcParams {
    const uint8_t *chunk, *hist;   // [stream][chunk_bytes], [stream][hist_bytes]
    long long chunk_bytes, hist_bytes;
    long long L, H;                // chunk and history samples (H a multiple of 16, >= Lh)
    long long t_in;                // first input sample of the chunk
    long long j0;                  // first output of the call (= 2 t_in / D)
    int D2, lgD2, Th2, Lout;       // D / 2, log2(D / 2), Lh / (D / 2), outputs per stream
    const float2 *taps;            // [Lh] h[u] exp(2 pi i fc u)
    double fc;
    float g2;                      // 2 g
    uint8_t *out;                  // [stream][5 Lout / 4]
    float *out_float;              // optional [stream][Lout]
};

// position of plane element k: one word of padding per 16 elements, so that
// the 32 lanes of a warp, 16 elements apart, hit 32 different banks
__device__ __forceinline__ int ppos(int k) { return k + (k >> 4); }
// words per plane: every padded position of K elements, rounded up to an
// even count so that the float2 tap table after the planes is 8-byte aligned
__host__ __device__ __forceinline__ int ddc_plane_words(int K) { return (K + (K >> 4) + 2) & ~1; }

// Outputs j = jb + 16 t + r (r < 16) of thread t. Sample offsets o = i -
// i_base (i_base = (jb - Th2) D2) sit in plane o mod D2 at element o / D2;
// output j's tap u = a D2 + b reads plane (D2 - b) mod D2, element
// 16 t + r + Th2 - a - (b > 0). A block of 8 taps a0 .. a0 + 7 of one plane
// needs the 23 elements 16 t + Th2 - (b > 0) - a0 - 7 ... + 15, loaded once
// and used by all 16 outputs (128 complex multiply-adds per 31 shared loads).
__global__ void __launch_bounds__(kDdcThreads) k_ddc(const DdcParams p) {
    extern __shared__ float sm[];
    const int D2 = p.D2, Th2 = p.Th2, K = kDdcOut + Th2, KP = ddc_plane_words(K), Lh = D2 * Th2;
    float *xp = sm;                                         // [D2][KP] phase planes
    float2 *tp = reinterpret_cast<float2 *>(sm + D2 * KP);  // [Lh] taps
    const int st = blockIdx.y;
    const long long jb = p.j0 + (long long)blockIdx.x * kDdcOut;
    const long long i_base = (jb - Th2) * D2;
    const uint8_t *chunk = p.chunk + (long long)st * p.chunk_bytes;
    const uint8_t *hist = p.hist + (long long)st * p.hist_bytes;
    const long long h0 = p.t_in - p.H;                      // first history sample
    // decode 8 consecutive samples per task from 32-bit words of the packed
    // stream (history and chunk are one bit stream: 10 H is a multiple of
    // 32), zero outside it
    {
        const uint32_t *hw = reinterpret_cast<const uint32_t *>(hist);
        const uint32_t *cw = reinterpret_cast<const uint32_t *>(chunk);
        const long long hwords = 10 * p.H / 32, cwords = p.chunk_bytes / 4, n_rel = p.H + p.L;
        for (int e = threadIdx.x; 8 * e < D2 * K; e += kDdcThreads) {
            const long long rel = i_base + 8 * e - h0;
            uint32_t fld[8];
#pragma unroll
            for (int k = 0; k < 8; k++) fld[k] = 0x200u;   // offset binary: 0x200 is zero
            if (rel + 8 > 0 && rel < n_rel) {
                const long long bit = 10 * rel;
                const long long w0 = bit >> 5;   // floor, also for negative rel
                const unsigned sh = (unsigned)(bit & 31);
                uint32_t wd[5];
#pragma unroll
                for (int i = 0; i < 5; i++) {
                    const long long w = w0 + i;
                    uint32_t x = 0u;
                    if (w >= 0 && w < hwords) x = __ldg(hw + w);
                    else if (w >= hwords && w - hwords < cwords) x = __ldg(cw + (w - hwords));
                    wd[i] = __byte_perm(x, 0u, 0x0123u);   // big-endian bits
                }
                uint32_t a[4];
#pragma unroll
                for (int i = 0; i < 4; i++) a[i] = __funnelshift_l(wd[i + 1], wd[i], sh);
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const int bb = 10 * k;
                    const uint32_t f = __funnelshift_l(a[(bb >> 5) + 1], a[bb >> 5], (unsigned)(bb & 31)) >> 22;
                    fld[k] = (rel + k < 0 || rel + k >= n_rel) ? 0x200u : (f ^ 0x200u);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 8; k++) fld[k] = 0x200u;
            }
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int o = 8 * e + k;
                if (o < D2 * K) xp[(o & (D2 - 1)) * KP + ppos(o >> p.lgD2)] = (float)((int)fld[k] - 512);
            }
        }
    }
    for (int u = threadIdx.x; u < Lh; u += kDdcThreads) tp[u] = __ldg(p.taps + u);
    __syncthreads();

    const int t = threadIdx.x;
    float re[kDdcPer], im[kDdcPer];
#pragma unroll
    for (int r = 0; r < kDdcPer; r++) re[r] = im[r] = 0.0f;
    for (int b = 0; b < D2; b++) {
        const float *plane = xp + (b == 0 ? 0 : D2 - b) * KP;
        const int base = kDdcPer * t + Th2 - (b == 0 ? 0 : 1);   // element of (r = 0, a = 0)
        int a0 = 0;
        for (; a0 + 8 <= Th2; a0 += 8) {
            float x[kDdcPer + 7];
#pragma unroll
            for (int i = 0; i < kDdcPer + 7; i++) x[i] = plane[ppos(base - a0 - 7 + i)];
#pragma unroll
            for (int aa = 0; aa < 8; aa++) {
                const float2 h = tp[(a0 + aa) * D2 + b];
#pragma unroll
                for (int r = 0; r < kDdcPer; r++) {
                    re[r] = fmaf(h.x, x[r - aa + 7], re[r]);
                    im[r] = fmaf(h.y, x[r - aa + 7], im[r]);
                }
            }
        }
        for (int a = a0; a < Th2; a++) {   // taps left over when Th2 is not a multiple of 8
            const float2 h = tp[a * D2 + b];
#pragma unroll
            for (int r = 0; r < kDdcPer; r++) {
                const float x = plane[ppos(base + r - a)];
                re[r] = fmaf(h.x, x, re[r]);
                im[r] = fmaf(h.y, x, im[r]);
            }
        }
    }
    // rotation exp(2 pi i (j / 4 - fc i0)), i0 = j D2: the first output's
    // phase and the step between consecutive outputs (1/4 - fc D2) reduced in
    // FP64, later ones by repeated multiplication (16 steps, error ~1e-6);
    // requantise; pack four outputs into five bytes, MSB first
    const long long k0 = jb - p.j0 + (long long)kDdcPer * t;   // first output within the call
    const long long j_first = jb + (long long)kDdcPer * t;
    double ph = 0.25 * (double)(j_first & 3) - p.fc * (double)(j_first * D2);
    ph -= floor(ph);
    double dph = 0.25 - p.fc * (double)D2;
    dph -= floor(dph);
    float c, s, dc, ds;
    sincospif(2.0f * (float)ph, &s, &c);
    sincospif(2.0f * (float)dph, &ds, &dc);
    unsigned q[kDdcPer];
#pragma unroll
    for (int r = 0; r < kDdcPer; r++) {
        const float y = p.g2 * (c * re[r] - s * im[r]);
        const float c2 = c * dc - s * ds;
        s = s * dc + c * ds;
        c = c2;
        float rr = roundf(y);                                 // half away from zero
        rr = fminf(fmaxf(rr, -511.0f), 511.0f);
        q[r] = (unsigned)(int)rr & 0x3FFu;
        if (p.out_float && k0 + r < p.Lout) p.out_float[(long long)st * p.Lout + k0 + r] = y;
    }
    uint8_t *o = p.out + (long long)st * (5LL * p.Lout / 4) + 5 * (k0 >> 2);
#pragma unroll
    for (int g = 0; g < kDdcPer / 4; g++) {
        if (k0 + 4 * g >= p.Lout) break;
        const unsigned q0 = q[4 * g], q1 = q[4 * g + 1], q2 = q[4 * g + 2], q3 = q[4 * g + 3];
        o[5 * g + 0] = (uint8_t)(q0 >> 2);
        o[5 * g + 1] = (uint8_t)(((q0 & 0x3u) << 6) | (q1 >> 4));
        o[5 * g + 2] = (uint8_t)(((q1 & 0xFu) << 4) | (q2 >> 6));
        o[5 * g + 3] = (uint8_t)(((q2 & 0x3Fu) << 2) | (q3 >> 8));
        o[5 * g + 4] = (uint8_t)(q3 & 0xFFu);
    }
}

bool pow2_decimation(int D) { return D == 2 || D == 4 || D == 8 || D == 16 || D == 32; }

void default_filter(int D, int Th, std::vector<double> &h) {
    const long long L = (long long)D * Th;
    h.assign((size_t)L, 0.0);
    double sum = 0.0;
    for (long long u = 0; u < L; u++) {
        const double x = ((double)u + 0.5 - (double)L / 2.0) / (double)D;
        const double sinc = x == 0.0 ? 1.0 : std::sin(M_PI * x) / (M_PI * x);
        const double w = std::sin(M_PI * ((double)u + 0.5) / (double)L);
        h[(size_t)u] = w * w * sinc;
        sum += h[(size_t)u];
    }
    for (double &v : h) v /= sum;
}

}  // namespace

struct fengine_ddc_s {
    int n_streams = 0, D = 0, Th = 0, Lh = 0;
    long long L = 0, H = 0, hist_bytes = 0, chunk_bytes = 0, next = 0;
    bool started = false;
    int cur = 0;
    double fc = 0.0;
    float g = 1.0f;
    uint8_t *d_hist[2] = {nullptr, nullptr};
    float2 *d_taps = nullptr;
};

namespace {

void ddc_release(fengine_ddc_s *d) {
    cudaFree(d->d_hist[0]);
    cudaFree(d->d_hist[1]);
    cudaFree(d->d_taps);
    delete d;
}

}  // namespace

extern "C" fengine_status fengine_ddc_default_filter(int32_t decimation, int32_t taps_per_phase, float *out) {
    if (!out || !pow2_decimation(decimation) || taps_per_phase < 1 || (long long)decimation * taps_per_phase > 2048)
        return FENGINE_EINVAL;
    std::vector<double> h;
    default_filter(decimation, taps_per_phase, h);
    for (size_t u = 0; u < h.size(); u++) out[u] = (float)h[u];
    return FENGINE_OK;
}

extern "C" fengine_status fengine_ddc_create(const fengine_ddc_config *cfg, fengine_ddc_t *out) {
    if (!cfg || !out) return FENGINE_EINVAL;
    *out = nullptr;
    const int D = cfg->decimation, Th = cfg->taps_per_phase;
    if (cfg->n_antennas < 1 || cfg->n_antennas > 1024 || !pow2_decimation(D) || Th < 1 ||
        (long long)D * Th > 2048 || cfg->reserved != 0)
        return FENGINE_EINVAL;
    const long long Lh = (long long)D * Th;
    if (cfg->chunk_samples <= 0 || cfg->chunk_samples % (2 * D) || cfg->chunk_samples % 16 || cfg->chunk_samples < Lh ||
        cfg->chunk_samples > (1LL << 34))
        return FENGINE_EINVAL;
    if (!(cfg->center_frequency >= 0.0 && cfg->center_frequency < 0.5) || !std::isfinite(cfg->gain))
        return FENGINE_EINVAL;
    std::vector<double> h;
    if (cfg->filter) {
        h.assign((size_t)Lh, 0.0);
        for (long long u = 0; u < Lh; u++) {
            if (!std::isfinite(cfg->filter[u])) return FENGINE_EINVAL;
            h[(size_t)u] = cfg->filter[u];
        }
    } else {
        default_filter(D, Th, h);
    }
    auto *d = new (std::nothrow) fengine_ddc_s;
    if (!d) return FENGINE_ENOMEM;
    d->n_streams = 2 * cfg->n_antennas;
    d->D = D;
    d->Th = Th;
    d->Lh = (int)Lh;
    d->L = cfg->chunk_samples;
    d->H = (Lh + 15) / 16 * 16;
    d->hist_bytes = d->H / 4 * 5;
    d->chunk_bytes = d->L / 4 * 5;
    d->fc = cfg->center_frequency;
    d->g = cfg->gain;
    // taps with the mixing factor, h[u] exp(2 pi i fc u), the phase reduced in FP64
    std::vector<float2> taps((size_t)Lh);
    for (long long u = 0; u < Lh; u++) {
        double ph = d->fc * (double)u;
        ph -= std::floor(ph);
        taps[(size_t)u] = make_float2((float)(h[(size_t)u] * std::cos(2.0 * M_PI * ph)),
                                      (float)(h[(size_t)u] * std::sin(2.0 * M_PI * ph)));
    }
    const size_t hb = (size_t)d->hist_bytes * d->n_streams;
    if (cudaMalloc((void **)&d->d_hist[0], hb) != cudaSuccess || cudaMalloc((void **)&d->d_hist[1], hb) != cudaSuccess ||
        cudaMalloc((void **)&d->d_taps, sizeof(float2) * (size_t)Lh) != cudaSuccess) {
        cudaGetLastError();
        ddc_release(d);
        return FENGINE_ENOMEM;
    }
    if (cudaMemset(d->d_hist[0], 0, hb) != cudaSuccess || cudaMemset(d->d_hist[1], 0, hb) != cudaSuccess ||
        cudaMemcpy(d->d_taps, taps.data(), sizeof(float2) * (size_t)Lh, cudaMemcpyHostToDevice) != cudaSuccess) {
        ddc_release(d);
        return FENGINE_ECUDA;
    }
    *out = d;
    return FENGINE_OK;
}

extern "C" fengine_status fengine_ddc_destroy(fengine_ddc_t d) {
    if (!d) return FENGINE_EINVAL;
    cudaDeviceSynchronize();
    ddc_release(d);
    return FENGINE_OK;
}

extern "C" fengine_status fengine_ddc_reset(fengine_ddc_t d) {
    if (!d) return FENGINE_EINVAL;
    const size_t hb = (size_t)d->hist_bytes * d->n_streams;
    if (cudaMemset(d->d_hist[0], 0, hb) != cudaSuccess || cudaMemset(d->d_hist[1], 0, hb) != cudaSuccess)
        return FENGINE_ECUDA;
    d->started = false;
    d->cur = 0;
    return FENGINE_OK;
}

extern "C" fengine_status fengine_ddc_process(fengine_ddc_t d, void *cuda_stream, const uint8_t *d_packed,
                                              int64_t first_sample, uint8_t *d_out, float *d_out_float) {
    if (!d || !d_packed || !d_out) return FENGINE_EINVAL;
    if (((uintptr_t)d_packed & 3) || ((uintptr_t)d_out & 3) || ((uintptr_t)d_out_float & 3)) return FENGINE_EINVAL;
    if (first_sample % (2LL * d->D)) return FENGINE_EINVAL;
    if (d->started && first_sample != d->next) return FENGINE_ESEQ;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    DdcParams p{};
    p.chunk = d_packed;
    p.hist = d->d_hist[d->cur];
    p.chunk_bytes = d->chunk_bytes;
    p.hist_bytes = d->hist_bytes;
    p.L = d->L;
    p.H = d->H;
    p.t_in = first_sample;
    p.j0 = first_sample / (d->D / 2);
    p.D2 = d->D / 2;
    p.lgD2 = 0;
    while ((1 << p.lgD2) < p.D2) p.lgD2++;
    p.Th2 = d->Lh / p.D2;
    p.Lout = (int)(d->L / p.D2);
    p.taps = d->d_taps;
    p.fc = d->fc;
    p.g2 = 2.0f * d->g;
    p.out = d_out;
    p.out_float = d_out_float;
    const int KP = ddc_plane_words(kDdcOut + p.Th2);
    const size_t smem = sizeof(float) * (size_t)p.D2 * KP + sizeof(float2) * (size_t)d->Lh;
    cudaError_t e = cudaFuncSetAttribute(k_ddc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return FENGINE_ECUDA;
    dim3 grid((unsigned)((p.Lout + kDdcOut - 1) / kDdcOut), (unsigned)d->n_streams);
    k_ddc<<<grid, kDdcThreads, smem, st>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return FENGINE_ECUDA;
    // the next call's history: the last H samples of history + chunk
    if ((e = fe::launch_tail_update(d->d_hist[d->cur], d_packed, d->d_hist[1 - d->cur], d->hist_bytes, d->chunk_bytes,
                                    d->n_streams, st)) != cudaSuccess)
        return FENGINE_ECUDA;
    d->cur = 1 - d->cur;
    d->started = true;
    d->next = first_sample + d->L;
    return FENGINE_OK;
}
