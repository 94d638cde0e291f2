// Phase 2, FP32 form for N2 = 1024: one warp computes the whole 1024-point
// FFT of one (spectrum, pol) sequence in registers, then the fine-delay
// rotation, gain, requantisation and corner turn (Sec. 2.1 steps 4-6,
// Sec. 2.2, Sec. 3.6).
//
// With t2 = 32 a + b and k2 = c + 32 d (a, b, c, d in [0, 32)):
//   Y[c][b]     = sum_a exp(-2 pi i c a / 32) B[32 a + b]
//   Y'[c][b]    = exp(-2 pi i c b / 1024) Y[c][b]
//   F[c + 32 d] = sum_b Y'[c][b] exp(-2 pi i d b / 32).
// Lane b loads B[32 a + b] for every a (coalesced), does the first 32-point
// DFT in registers, applies the twiddle, and writes Y'[.][b] into the warp's
// padded shared-memory tile; after one transpose lane c holds Y'[c][.] and
// does the second 32-point DFT in registers, leaving F[c + 32 d] for every d.
// One shared-memory round trip per point instead of one per radix pass.
//
// A CTA owns one first-stage class k1 and 4 consecutive spectra; warp w
// computes spectrum w / 2, polarisation w % 2. Channel mapping, rotation
// split and upper-half conjugation are those of the other second stages:
// slot k2 is channel k1 + N1 k2 for k2 < 512, and for k2 >= 512 (classes
// k1 = 1 .. N1/2 - 1 only) the conjugate of channel N - (k1 + N1 k2).
#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kWThreads = 256;
constexpr int kWR = 4;        // spectra per CTA (two warps each)
constexpr int kWN2 = 1024;
constexpr int kTLd = 33;      // transpose tile row stride in float2 (conflict-free both ways)
constexpr int kWPQ = 65;      // per sequence: P[32], Q[32], qu

// 32-bit word of output cell (slot k2, spectrum r) in the staging buffer: the
// 4 cells of a slot are permuted by k2's bits 3-4 so that the 32 lanes of a
// store (consecutive k2) and of a corner-turn read hit 32 banks.
__device__ __forceinline__ int stg_word(int k2, int r) { return k2 * kWR + (r ^ ((k2 >> 3) & 3)); }

}  // namespace

size_t phase2w_smem_bytes() {
    return sizeof(float2) * (8 * 32 * kTLd)    // transpose tiles (afterwards: the staging)
           + sizeof(float2) * 2 * kWN2         // gains of the CTA's slots
           + sizeof(float2) * 2 * kWR * kWPQ   // rotation factors
           + (sizeof(long long) + sizeof(int)) * kWR;
}

__global__ void __launch_bounds__(kWThreads, 2) k_phase2w(const Phase2Params p) {
    extern __shared__ float2 smw[];
    float2 *tbuf = smw;                                            // [8][32][kTLd]
    unsigned *stg = reinterpret_cast<unsigned *>(smw);             // [kWN2][kWR], after the FFTs
    float2 *gsm = smw + 8 * 32 * kTLd;                             // [2][kWN2]
    float2 *pq = gsm + 2 * kWN2;                                   // [2 kWR][kWPQ]
    long long *rowoff = reinterpret_cast<long long *>(pq + 2 * kWR * kWPQ);
    int *rowstride = reinterpret_cast<int *>(rowoff + kWR);

    const int k1 = blockIdx.x, ant = blockIdx.z;
    const int q0 = p.q_begin + blockIdx.y * kWR;
    const int M = p.M, Rv = min(kWR, p.q_begin + p.q_count - q0);
    const int N1 = p.N1, H1 = N1 / 2, N = p.N, n = N / 2, S_ = p.S;
    const bool upper = (k1 != 0 && k1 != H1);
    const int nslot = upper ? kWN2 : kWN2 / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = warp >> 1, pol = warp & 1, stream = ant * 2 + pol;
    const bool active = r < Rv;

    // this warp's sequence: lane b takes B[32 a + b] (loads issued before the set-up)
    float2 z[32];
    if (active) {
        const float2 *src =
            p.A + ((long long)(stream * p.a_spectra + (q0 - p.q_begin) + r) * (H1 + 1) + k1) * kWN2 + lane;
#pragma unroll
        for (int a = 0; a < 32; a++) z[a] = __ldg(src + 32 * a);
    }

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
        pq[e] = make_float2(cs, sn);
    }
    for (int e = threadIdx.x; e < 2 * kWN2; e += kWThreads) {
        const int ps = e / kWN2, k2 = e % kWN2;
        const int kc = k1 + N1 * k2;
        const int k = k2 >= kWN2 / 2 ? N - kc : kc;
        gsm[e] = (k >= 0 && k < n) ? __ldg(p.gains + (long long)(ant * 2 + ps) * n + k) : make_float2(0.f, 0.f);
    }
    if ((int)threadIdx.x < Rv) {
        const int q = q0 + threadIdx.x;
        const int h = q / S_, s = q - h * S_;
        const int Sh = min(S_, M - h * S_);
        rowoff[threadIdx.x] = (long long)h * S_ * n * 4 + s * 4;
        rowstride[threadIdx.x] = Sh * 4;
    }
    __syncthreads();

    if (active) {
        fft_regc<32>(z);                                  // z[c] = Y[c][lane]
#pragma unroll
        for (int c = 1; c < 32; c++) z[c] = cmul(z[c], __ldg(p.tw2 + ((c * lane) & (kWN2 - 1))));
        float2 *tb = tbuf + warp * 32 * kTLd;
#pragma unroll
        for (int c = 0; c < 32; c++) tb[c * kTLd + lane] = z[c];
        __syncwarp();
#pragma unroll
        for (int b = 0; b < 32; b++) z[b] = tb[lane * kTLd + b];
        fft_regc<32>(z);                                  // z[d] = F[lane + 32 d]
    }
    __syncthreads();   // every tile read: the tiles become the staging buffer

    if (active) {
        const float2 *pqs = pq + (pol * kWR + r) * kWPQ;
        const float2 P = pqs[lane], qu = pqs[64];
        const float2 Pu = cmul(qu, cconj(P));
        const float2 *gp = gsm + pol * kWN2;
        unsigned short *stg16 = reinterpret_cast<unsigned short *>(stg);
        float2 *pre = p.prequant ? p.prequant + ((long long)stream * M + q0 + r) * n : nullptr;
        // lower half (d < 16): channel k1 + N1 k2
#pragma unroll
        for (int d = 0; d < 16; d++) {
            const int k2 = lane + 32 * d;
            const float2 y = cmul(gp[k2], cmul(cmul(P, pqs[32 + d]), z[d]));
            if (pre) pre[k1 + N1 * k2] = y;
            stg16[2 * stg_word(k2, r) + pol] =
                (unsigned short)__byte_perm((unsigned)quant8(y.x), (unsigned)quant8(y.y), 0x0040u);
        }
        if (upper) {
            // upper half (d >= 16): channel N - (k1 + N1 k2)
#pragma unroll
            for (int d = 16; d < 32; d++) {
                const int k2 = lane + 32 * d;
                const float2 y = cmul(gp[k2], cmul(cmul(Pu, cconj(pqs[32 + d])), cconj(z[d])));
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
            *reinterpret_cast<unsigned *>(out + rowoff[rr] + (long long)k * rowstride[rr]) = stg[stg_word(k2, rr)];
        }
    }
}

cudaError_t launch_phase2w(const Phase2Params &p, int n_ant, cudaStream_t s) {
    if (p.N / p.N1 != kWN2) return cudaErrorInvalidValue;
    const size_t smem = phase2w_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_phase2w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(p.N1 / 2 + 1, (p.q_count + kWR - 1) / kWR, n_ant);
    k_phase2w<<<grid, kWThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace fe
