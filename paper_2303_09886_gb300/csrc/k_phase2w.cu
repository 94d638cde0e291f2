// Phase 2, FP32 form for N2 = 1024: one warp computes the whole 1024-point
// FFT of one (spectrum, pol) sequence in registers, then the fine-delay
// rotation, gain, requantisation and corner turn (Sec. 2.1 steps 4-6,
// Sec. 2.2, Sec. 3.6).
//
// With t2 = 32 a + b and k2 = c + 32 d (a, b, c, d in [0, 32)):
//   Y[c][b]     = sum_a exp(-2 pi i c a / 32) B[32 a + b]
//   Y'[c][b]    = exp(-2 pi i c b / 1024) Y[c][b]
//   F[c + 32 d] = sum_b Y'[c][b] exp(-2 pi i d b / 32).
// The sequence arrives in the warp's shared-memory buffer by cp.async; lane
// b reads B[32 a + b] for every a, does the first 32-point DFT in registers,
// applies the twiddle, and writes Y'[.][b] back into the buffer (XOR
// swizzle); after that transpose lane c holds Y'[c][.] and does the second
// 32-point DFT in registers, leaving F[c + 32 d] for every d. One
// shared-memory round trip per point instead of one per radix pass.
//
// A work item is one first-stage class k1 and 4 consecutive spectra of one
// antenna; warp w computes spectrum w / 2, polarisation w % 2. The kernel is
// persistent (a contiguous range of items per CTA) so that each warp's next
// sequence is in flight while the current one is finished. Channel mapping,
// rotation split and upper-half conjugation are those of the other second
// stages:
// slot k2 is channel k1 + N1 k2 for k2 < 512, and for k2 >= 512 (classes
// k1 = 1 .. N1/2 - 1 only) the conjugate of channel N - (k1 + N1 k2).
#include <algorithm>

#include <cuda_fp16.h>

#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kWThreads = 256;
constexpr int kWR = 4;        // spectra per work item (two warps each)
constexpr int kWN2 = 1024;
constexpr int kWPQ = 65;      // per sequence: P[32], Q[32], qu

// 32-bit word of output cell (slot k2, spectrum r) in the staging buffer: the
// 4 cells of a slot are permuted by k2's bits 3-4 so that the 32 lanes of a
// store (consecutive k2) and of a corner-turn read hit 32 banks.
__device__ __forceinline__ int stg_word(int k2, int r) { return k2 * kWR + (r ^ ((k2 >> 3) & 3)); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// A work item is (antenna, class k1, group of kWR consecutive spectra), in
// that order; item -> its fields.
struct WItem {
    int ant, k1, q0;
};
__device__ __forceinline__ WItem witem(const Phase2Params &p, int it, int H1, int G) {
    const int per_ant = (H1 + 1) * G;
    WItem w;
    w.ant = it / per_ant;
    const int rem = it - w.ant * per_ant;
    w.k1 = rem / G;
    w.q0 = p.q_begin + (rem - w.k1 * G) * kWR;
    return w;
}

}  // namespace

size_t phase2w_smem_bytes() {
    return sizeof(float2) * 8 * kWN2              // per-warp sequence buffers (also the transpose tiles)
           + sizeof(unsigned) * kWN2 * kWR        // output staging
           + sizeof(float2) * 2 * kWN2            // gains of the item's slots
           + sizeof(float2) * 2 * kWR * kWPQ      // rotation factors
           + sizeof(float2) * 32 * 32             // twiddles exp(-2 pi i c b / 1024), [c][b]
           + (sizeof(long long) + sizeof(int)) * 2 * kWR;   // row info, two items
}

// Persistent: each CTA takes a contiguous range of work items of equal work.
// Warp w owns
// sequence (spectrum w / 2, polarisation w % 2) of every item; its 8 KB
// sequence arrives in its shared-memory buffer by cp.async, and the copy of
// the next item's sequence is issued as soon as the buffer has been read
// (after the transpose), so it runs under this item's second DFT, epilogue
// and corner turn.
template <bool HALF_IN>
__global__ void __launch_bounds__(kWThreads, 2) k_phase2w(const Phase2Params p, int n_ant) {
    extern __shared__ float2 smw[];
    float2 *sbuf = smw;                                                   // [8][kWN2]
    unsigned *stg = reinterpret_cast<unsigned *>(smw + 8 * kWN2);         // [kWN2][kWR]
    float2 *gsm = reinterpret_cast<float2 *>(stg + kWN2 * kWR);           // [2][kWN2]
    float2 *pq = gsm + 2 * kWN2;                                          // [2 kWR][kWPQ]
    float2 *twm = pq + 2 * kWR * kWPQ;                                    // [32 c][32 b]
    long long *rowoff_all = reinterpret_cast<long long *>(twm + 32 * 32);   // [2][kWR]
    int *rowstride_all = reinterpret_cast<int *>(rowoff_all + 2 * kWR);       // [2][kWR]

    const int M = p.M, N1 = p.N1, H1 = N1 / 2, N = p.N, n = N / 2, S_ = p.S;
    const int G = (p.q_count + kWR - 1) / kWR;
    const int n_items = n_ant * (H1 + 1) * G;
    // Contiguous ranges of equal work: classes k1 = 0 and N1/2 keep only the
    // lower half of their slots (half the epilogue and corner turn), so their
    // items count 4 units against 5 for the others; CTA b takes the items
    // whose work starts in [b W / gridDim.x, (b + 1) W / gridDim.x).
    constexpr int wL = 4, wF = 5;
    const int Wa = G * (2 * wL + (H1 - 1) * wF);   // work of one antenna
    auto first_item = [&](long long x) {          // first item whose work starts at >= x
        const int ant = (int)(x / Wa);
        const int y = (int)(x - (long long)ant * Wa);
        int k1, g;
        if (y < wL * G) {
            k1 = 0;
            g = (y + wL - 1) / wL;
        } else if (y < (wL + (H1 - 1) * wF) * G) {
            const int y1 = y - wL * G;
            k1 = 1 + y1 / (wF * G);
            g = (y1 - (k1 - 1) * wF * G + wF - 1) / wF;
        } else {
            k1 = H1;
            g = (y - (wL + (H1 - 1) * wF) * G + wL - 1) / wL;
        }
        return min(n_items, ant * (H1 + 1) * G + k1 * G + g);
    };
    const long long Wt = (long long)n_ant * Wa;
    const int it0 = first_item(Wt * blockIdx.x / gridDim.x), it1 = first_item(Wt * (blockIdx.x + 1) / gridDim.x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = warp >> 1, pol = warp & 1;
    float2 *mybuf = sbuf + warp * kWN2;

    // this warp's sequence of item it into its buffer (lane: 16-byte chunks lane + 32 i)
    // (FP16 pairs: 4 KB in the first half of the buffer)
    auto fetch = [&](int it) {
        const WItem w = witem(p, it, H1, G);
        if (w.q0 + r < p.q_begin + p.q_count) {
            const long long e0 =
                ((long long)((w.ant * 2 + pol) * p.a_spectra + (w.q0 - p.q_begin) + r) * (H1 + 1) + w.k1) * kWN2;
            if constexpr (HALF_IN) {
                const uint32_t *src = reinterpret_cast<const uint32_t *>(p.A) + e0;
                uint32_t *dst = reinterpret_cast<uint32_t *>(mybuf);
#pragma unroll
                for (int i = 0; i < 8; i++) cp_async16(dst + 4 * (lane + 32 * i), src + 4 * (lane + 32 * i));
            } else {
                const float2 *src = p.A + e0;
#pragma unroll
                for (int i = 0; i < 16; i++) cp_async16(mybuf + 2 * (lane + 32 * i), src + 2 * (lane + 32 * i));
            }
        }
        cp_async_commit();
    };
    if (it0 < it1) fetch(it0);
    // the twiddle of (c, b) at [c][b]: a warp's 32 lanes (b) read 32 consecutive entries
    for (int e = threadIdx.x; e < 32 * 32; e += kWThreads) twm[e] = __ldg(p.tw2 + (((e >> 5) * (e & 31)) & (kWN2 - 1)));
    __syncthreads();   // the twiddles are read before the first item's barrier

    long long cur = -1;   // (ant, k1, gain set of each pol) of the gains in gsm
    for (int it = it0; it < it1; it++) {
        // row info alternates between two slots: the previous item's corner
        // turn may still read its slot while this item's is written
        long long *rowoff = rowoff_all + ((it - it0) & 1) * kWR;
        int *rowstride = rowstride_all + ((it - it0) & 1) * kWR;
        const WItem w = witem(p, it, H1, G);
        const int ant = w.ant, k1 = w.k1, q0 = w.q0;
        const int Rv = min(kWR, p.q_begin + p.q_count - q0);
        const bool upper = (k1 != 0 && k1 != H1);
        const int nslot = upper ? kWN2 : kWN2 / 2;
        const bool active = r < Rv;
        const int stream = ant * 2 + pol;

        // No barrier here: the tables (pq, gsm) were last read by the previous
        // item's epilogue, before its final barrier; stg is written only after
        // the next barrier, which every thread reaches after its corner turn.
        // rotation factors of each (pol, spectrum) sequence, angles over pi:
        //   P[c] = exp(i pi (phi/pi - 2 delta (k1 + N1 c) / N)),
        //   Q[d] = exp(-i pi 2 delta 32 N1 d / N),  qu = exp(i pi (2 phi/pi - 2 delta)),
        // so that channel k1 + N1 k2 (k2 = c + 32 d) is P[c] Q[d] F[k2] and the
        // upper-half channel N - (k1 + N1 k2) is qu conj(P[c] Q[d] F[k2]).
        const float inv = 2.0f / (float)N;
        for (int e = threadIdx.x; e < 2 * kWR * kWPQ; e += kWThreads) {
            const int sq = e / kWPQ, j = e - sq * kWPQ;
            const int ps = sq / kWR, rs = sq % kWR;
            if (rs >= Rv) continue;
            const float2 f = p.ftab[(long long)(ant * 2 + ps) * M + q0 + rs];   // (delta, phi / pi)
            const int c = j & 31;
            float ang;
            if (j < 32) ang = f.y - f.x * (float)(k1 + N1 * c) * inv;
            else if (j < 64) ang = -f.x * (float)(32 * N1 * c) * inv;
            else ang = 2.0f * f.y - 2.0f * f.x;
            float sn, cs;
            sincospif(ang, &sn, &cs);
            // P carries the inverse of the FP16 intermediate's scale (a power of two)
            const float u = (HALF_IN && j < 32) ? p.tc_unscale : 1.0f;
            pq[e] = make_float2(cs * u, sn * u);
        }
        // gains staged for the gain set of the item's first spectrum in each pol
        const int gs0 = p.gsel ? p.gsel[(long long)(ant * 2) * M + q0] : 0;
        const int gs1 = p.gsel ? p.gsel[(long long)(ant * 2 + 1) * M + q0] : 0;
        const long long key = (((long long)ant * 1024 + k1) * 256 + gs0) * 256 + gs1;
        if (key != cur) {
            cur = key;
            for (int e = threadIdx.x; e < 2 * kWN2; e += kWThreads) {
                const int ps = e / kWN2, k2 = e % kWN2;
                const int kc = k1 + N1 * k2;
                const int k = k2 >= kWN2 / 2 ? N - kc : kc;
                const float2 *g = p.gains + ((long long)(ant * 2 + ps) * p.n_gsets_max + (ps ? gs1 : gs0)) * n;
                gsm[e] = (k >= 0 && k < n) ? __ldg(g + k) : make_float2(0.f, 0.f);
            }
        }
        if ((int)threadIdx.x < Rv) {
            const int q = q0 + threadIdx.x;
            const int h = q / S_, s = q - h * S_;
            const int Sh = min(S_, M - h * S_);
            rowoff[threadIdx.x] = (long long)h * S_ * n * 4 + s * 4;
            rowstride[threadIdx.x] = Sh * 4;
        }

        // With t2 = 32 a + b and k2 = c + 32 d: lane b takes B[32 a + b] for
        // every a, does the first 32-point DFT, applies the twiddle and writes
        // Y'[c][b] back to the buffer at c * 32 + (b ^ c) (conflict-free both
        // ways); after the transpose lane c holds Y'[c][.].
        cp_async_wait_all();
        __syncwarp();
        float2 z[32];
        if (active) {
            if constexpr (HALF_IN) {
                const __half2 *hb = reinterpret_cast<const __half2 *>(mybuf);
#pragma unroll
                for (int a = 0; a < 32; a++) z[a] = __half22float2(hb[32 * a + lane]);
            } else {
#pragma unroll
                for (int a = 0; a < 32; a++) z[a] = mybuf[32 * a + lane];
            }
            __syncwarp();
            fft_regc<32>(z);                                  // z[c] = Y[c][lane]
#pragma unroll
            for (int c = 1; c < 32; c++) z[c] = cmul(z[c], twm[32 * c + lane]);
#pragma unroll
            for (int c = 0; c < 32; c++) mybuf[32 * c + (lane ^ c)] = z[c];
            __syncwarp();
#pragma unroll
            for (int b = 0; b < 32; b++) z[b] = mybuf[32 * lane + (b ^ lane)];
        }
        __syncwarp();
        if (it + 1 < it1) fetch(it + 1);                      // the buffer is free again
        __syncthreads();                                      // tables and row info ready

        if (active) {
            fft_regc<32>(z);                                  // z[d] = F[lane + 32 d]
            const float2 *pqs = pq + (pol * kWR + r) * kWPQ;
            const float2 P = pqs[lane], qu = pqs[64];
            const float2 Pu = cmul(qu, cconj(P));
            const float2 *gp = gsm + pol * kWN2;
            // a spectrum whose gain set differs from the staged one (a gain
            // update inside the item) reads its gains directly
            const int gsr = p.gsel ? p.gsel[(long long)stream * M + q0 + r] : 0;
            const bool staged = gsr == (pol ? gs1 : gs0);
            const float2 *gdir = p.gains + ((long long)stream * p.n_gsets_max + gsr) * n;
            auto gain = [&](int k2) -> float2 {
                const int kc = k1 + N1 * k2;
                return staged ? gp[k2] : __ldg(gdir + (k2 >= kWN2 / 2 ? N - kc : kc));
            };
            unsigned short *stg16 = reinterpret_cast<unsigned short *>(stg);
            float2 *pre = p.prequant ? p.prequant + ((long long)stream * M + q0 + r) * n : nullptr;
            // lower half (d < 16): channel k1 + N1 k2
#pragma unroll
            for (int d = 0; d < 16; d++) {
                const int k2 = lane + 32 * d;
                const float2 y = cmul(gain(k2), cmul(cmul(P, pqs[32 + d]), z[d]));
                if (pre) pre[k1 + N1 * k2] = y;
                stg16[2 * stg_word(k2, r) + pol] =
                    (unsigned short)__byte_perm((unsigned)quant8(y.x), (unsigned)quant8(y.y), 0x0040u);
            }
            if (upper) {
                // upper half (d >= 16): channel N - (k1 + N1 k2)
#pragma unroll
                for (int d = 16; d < 32; d++) {
                    const int k2 = lane + 32 * d;
                    const float2 y = cmul(gain(k2), cmul(cmul(Pu, cconj(pqs[32 + d])), cconj(z[d])));
                    if (pre) pre[N - (k1 + N1 * k2)] = y;
                    stg16[2 * stg_word(k2, r) + pol] =
                        (unsigned short)__byte_perm((unsigned)quant8(y.x), (unsigned)quant8(y.y), 0x0040u);
                }
            }
        }
        __syncthreads();

        // corner turn: cell (slot k2, spectrum r) -> heap row of channel k; four
        // spectra of a slot with one 16-byte store when they share a heap and the
        // row is 16-byte aligned
        int8_t *out = p.out + (long long)ant * M * n * 4;
        const bool vec = Rv == kWR && S_ % 4 == 0 && rowstride[0] % 16 == 0;
        if (vec) {
            for (int k2 = threadIdx.x; k2 < nslot; k2 += kWThreads) {
                const int kc = k1 + N1 * k2;
                const int k = k2 >= kWN2 / 2 ? N - kc : kc;
                const uint4 v = make_uint4(stg[stg_word(k2, 0)], stg[stg_word(k2, 1)], stg[stg_word(k2, 2)],
                                           stg[stg_word(k2, 3)]);
                *reinterpret_cast<uint4 *>(out + rowoff[0] + (long long)k * rowstride[0]) = v;
            }
        } else {
            for (int e = threadIdx.x; e < nslot * kWR; e += kWThreads) {
                const int k2 = e / kWR, rr = e % kWR;
                if (rr >= Rv) continue;
                const int kc = k1 + N1 * k2;
                const int k = k2 >= kWN2 / 2 ? N - kc : kc;
                *reinterpret_cast<unsigned *>(out + rowoff[rr] + (long long)k * rowstride[rr]) =
                    stg[stg_word(k2, rr)];
            }
        }
    }
    cp_async_wait_all();   // nothing is left in flight when the CTA exits
}

template <bool HALF_IN>
static cudaError_t launch_w(const Phase2Params &p, int n_ant, cudaStream_t s) {
    const size_t smem = phase2w_smem_bytes();
    cudaError_t e =
        cudaFuncSetAttribute(k_phase2w<HALF_IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phase2w<HALF_IN>, kWThreads, smem)) !=
            cudaSuccess)
        return e;
    const long long items = (long long)n_ant * (p.N1 / 2 + 1) * ((p.q_count + kWR - 1) / kWR);
    if (items <= 0) return cudaSuccess;
    const int ctas = (int)std::min<long long>(items, (long long)sms * std::max(per_sm, 1));
    k_phase2w<HALF_IN><<<ctas, kWThreads, smem, s>>>(p, n_ant);
    return cudaGetLastError();
}

cudaError_t launch_phase2w(const Phase2Params &p, int n_ant, cudaStream_t s) {
    if (p.N / p.N1 != kWN2) return cudaErrorInvalidValue;
    return p.half_in ? launch_w<true>(p, n_ant, s) : launch_w<false>(p, n_ant, s);
}

}  // namespace fe
