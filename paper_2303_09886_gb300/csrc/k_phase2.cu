// Phase 2 of the fused F-engine: the N2-point FFT over t2 of the four-step
// split, then fine-delay rotation and bandpass gain (Sec. 2.1 steps 4-5),
// requantisation (Sec. 2.1 step 6, Sec. 3.6) and the channel-major corner
// turn into heaps (Sec. 2.2, Sec. 3.6).
//
// One CTA owns one first-stage index k1 in [0, N1/2] for R2 consecutive
// spectra of both polarisations of one antenna. The FFT of B[k1][.] gives
// F[k2] = X[k1 + N1 k2]. For k2 < N2/2 that is channel k = k1 + N1 k2
// directly; for k2 >= N2/2 it is a channel above n, whose conjugate is
// channel N - k (the real input's Hermitian symmetry), which belongs to the
// class N1 - k1. Classes k1 = 0 and k1 = N1/2 map onto themselves, so their
// CTAs keep only the lower half. Every channel in [0, n) is written once.
//
// FFT: in-place decimation in frequency, radix 16 while possible, then one
// radix-2/4/8 stage; each thread holds 16 points in registers per stage. The
// result is left in digit-reversed order and read back through the index map
// in the epilogue. Shared memory rows are padded by one complex per 16 so
// that every stage and the epilogue are free of bank conflicts.
//
// Rotation: exp(i phi) exp(-2 pi i delta k / N) for k = k1 + N1 k2 is the
// product of a per-(spectrum, pol) table over the high bits of k2 (with the
// exp(i phi) and k1 factors folded in) and one over the low 5 bits, built
// with sincospif at the start of the CTA.
//
// The CTA writes, for each of its channels, R2 consecutive spectra x 2 pols
// x (re, im) = 4 R2 contiguous bytes of one heap row.
#include <cuda_fp16.h>

#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kP2Threads = 256;

// exp(-2 pi i q / 16), q = 0..15, as compile-time constants.
__device__ __forceinline__ float2 w16(int q) {
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
    constexpr float re[16] = {1.f, c1, h, s1, 0.f, -s1, -h, -c1, -1.f, -c1, -h, -s1, 0.f, s1, h, c1};
    constexpr float im[16] = {0.f, -s1, -h, -c1, -1.f, -c1, -h, -s1, 0.f, s1, h, c1, 1.f, c1, h, s1};
    return make_float2(re[q], im[q]);
}

// In-register R-point DFT (R = 2, 4, 8, 16), natural order in and out,
// radix-2 decimation in time with compile-time twiddles.
template <int R>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
#pragma unroll
    for (int i = 0; i < R; i++) {
        const int j = bitrev<R>(i);
        if (i < j) {
            float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
#pragma unroll
    for (int len = 2; len <= R; len <<= 1) {
#pragma unroll
        for (int i = 0; i < R; i += len) {
#pragma unroll
            for (int j = 0; j < len / 2; j++) {
                const float2 w = w16(j * (16 / len));
                float2 b = v[i + j + len / 2];
                if (j != 0) b = cmul(b, w);
                const float2 a = v[i + j];
                v[i + j] = cadd(a, b);
                v[i + j + len / 2] = csub(a, b);
            }
        }
    }
}

// padded shared-memory index of element e of a sequence
__device__ __forceinline__ int pad(int e) { return e + (e >> 4); }

template <int N2>
struct P2Shape {
    static constexpr int P = N2 < 16 ? N2 : 16;                   // points per thread per stage
    static constexpr int TPS = N2 / P;                            // threads per sequence
    static constexpr int R2 = (4096 / N2) > 32 ? 32 : (4096 / N2); // spectra per CTA (2 CTAs per SM)
    static constexpr int LD = N2 + N2 / 16 + 1;                   // padded row stride
    static constexpr int LO = N2 < 32 ? N2 : 32;                  // rotation low table size
    static constexpr int HI = N2 / LO;                            // rotation high table size
};

// One DIF stage of radix R over spans of length Lspan (R divides Lspan).
// Butterfly (block b, j): v[r] = x[b Lspan + j + r Lspan/R]; V = DFT_R(v);
// x[b Lspan + j + k Lspan/R] = V[k] exp(-2 pi i j k / Lspan).
template <int N2, int R, int Lspan>
__device__ __forceinline__ void dif_stage(float2 *buf, int nseq, const float2 *tw) {
    using S = P2Shape<N2>;
    constexpr int PER = S::P / R;                 // butterflies per thread (16 points total)
    constexpr int sub = Lspan / R;
    constexpr int seq_per_round = kP2Threads / S::TPS;
    constexpr int tws = N2 / Lspan;               // twiddle table stride
    for (int s0 = 0; s0 < nseq; s0 += seq_per_round) {
        const int sq = s0 + (int)threadIdx.x / S::TPS;
        const int tl = (int)threadIdx.x % S::TPS;
        if (sq < nseq) {
            float2 *x = buf + sq * S::LD;
#pragma unroll
            for (int u = 0; u < PER; u++) {
                const int bf = tl + u * S::TPS;   // butterfly index in [0, per_seq)
                const int blk = bf / sub, j = bf - blk * sub;
                const int base = blk * Lspan + j;
                // pad(base + r sub) = pad(base) + padc(r sub): (base & 15) + (r sub & 15)
                // never carries into bit 4 (j < sub when sub < 16; r sub & 15 = 0
                // otherwise; base & 15 <= 12 with r < 4 when Lspan < 16)
                float2 *xb = x + pad(base);
                float2 v[R];
#pragma unroll
                for (int r = 0; r < R; r++) v[r] = xb[(r * sub) + ((r * sub) >> 4)];
                dft_reg<R>(v);
                if constexpr (Lspan != R) {
                    const int js = j * tws;
#pragma unroll
                    for (int k = 1; k < R; k++) v[k] = cmul(v[k], __ldg(tw + k * js));
                }
#pragma unroll
                for (int r = 0; r < R; r++) xb[(r * sub) + ((r * sub) >> 4)] = v[r];
            }
        }
    }
    __syncthreads();
}

// All DIF stages: radix 16 while the span allows, then the remaining radix.
template <int N2, int Lspan>
__device__ __forceinline__ void dif_all(float2 *buf, int nseq, const float2 *tw) {
    if constexpr (Lspan >= 16) {
        dif_stage<N2, 16, Lspan>(buf, nseq, tw);
        dif_all<N2, Lspan / 16>(buf, nseq, tw);
    } else if constexpr (Lspan > 1) {
        dif_stage<N2, Lspan, Lspan>(buf, nseq, tw);
    }
}

// Position of F[k2] after the DIF stages (digit reversal of k2 in the radix
// sequence 16, 16, ..., R_last).
template <int N2>
__device__ __forceinline__ int dif_pos(int k2) {
    int p = 0, L = N2, k = k2;
#pragma unroll
    for (int s = 0; s < 12; s++) {
        if (L <= 1) break;
        const int R = L >= 16 ? 16 : L;
        L /= R;
        p += (k % R) * L;
        k /= R;
    }
    return p;
}

}  // namespace

template <int N2, bool HALF_IN>
__global__ void __launch_bounds__(kP2Threads, 3) k_phase2(const Phase2Params p) {
    using S = P2Shape<N2>;
    constexpr int R2 = S::R2, LD = S::LD;
    extern __shared__ float2 sm[];
    float2 *buf = sm;                                  // [2 R2][LD]
    constexpr int HP = S::HI + 1, LP = S::LO + 1;      // padded table rows (no bank conflicts)
    float2 *thi = buf + 2 * R2 * LD;                   // [2 R2][HP]
    float2 *tlo = thi + 2 * R2 * HP;                   // [2 R2][LP]
    float2 *qup = tlo + 2 * R2 * LP;                   // [2 R2] upper-class factor
    long long *rowoff = reinterpret_cast<long long *>(qup + 2 * R2);   // [R2] heap row byte offset
    int *rowstride = reinterpret_cast<int *>(rowoff + R2);             // [R2] bytes per channel row

    const int k1 = blockIdx.x, ant = blockIdx.z;
    const int q0 = p.q_begin + blockIdx.y * R2;
    const int M = p.M, Rv = min(R2, p.q_begin + p.q_count - q0);
    const int N1 = p.N1, H1 = N1 / 2, N = p.N, n = N / 2, S_ = p.S;

    // stage B[k1][.] rows in (sequence = pol * R2 + r), padded
    {
        // two complex values per 16-byte load, all of a thread's loads in
        // flight before the first store; pad() keeps even pairs adjacent
        constexpr int PER = (R2 * N2 + kP2Threads - 1) / kP2Threads;
        float4 v[PER];
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int e = u * kP2Threads + threadIdx.x;
            const int sq = e / (N2 / 2), t2 = 2 * (e % (N2 / 2));
            const int pol = sq / R2, r = sq % R2;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            const long long o =
                (((long long)(ant * 2 + pol) * p.a_spectra + (q0 - p.q_begin) + r) * (H1 + 1) + k1) * N2 + t2;
            if (e < R2 * N2 && r < Rv) {
                if constexpr (HALF_IN) {
                    const uint2 h = __ldg(reinterpret_cast<const uint2 *>(reinterpret_cast<const uint32_t *>(p.A) + o));
                    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&h.x));
                    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&h.y));
                    v[u] = make_float4(a.x, a.y, b.x, b.y);
                } else {
                    v[u] = __ldg(reinterpret_cast<const float4 *>(p.A + o));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int e = u * kP2Threads + threadIdx.x;
            const int sq = e / (N2 / 2), t2 = 2 * (e % (N2 / 2));
            if (e < R2 * N2) {
                buf[sq * LD + pad(t2)] = make_float2(v[u].x, v[u].y);
                buf[sq * LD + pad(t2 + 1)] = make_float2(v[u].z, v[u].w);
            }
        }
    }
    // rotation tables: angle/pi = phi/pi - 2 delta k / N, k = k1 + N1 (LO a + b)
    const float inv = 2.0f / (float)N;
    for (int e = threadIdx.x; e < 2 * R2 * (S::HI + S::LO + 1); e += kP2Threads) {
        const int sq = e % (2 * R2), which = e / (2 * R2);
        const int pol = sq / R2, r = sq % R2;
        if (r >= Rv) continue;
        const float2 f = p.ftab[(long long)(ant * 2 + pol) * M + q0 + r];   // (delta, phi / pi)
        float sn, cs;
        if (which < S::HI) {
            const float kk = (float)(k1 + N1 * S::LO * which);
            sincospif(f.y - f.x * kk * inv, &sn, &cs);
            // with the inverse of the FP16 intermediate's scale (a power of two)
            const float us = HALF_IN ? p.tc_unscale : 1.0f;
            thi[sq * HP + which] = make_float2(cs * us, sn * us);
        } else if (which < S::HI + S::LO) {
            const int b = which - S::HI;
            sincospif(-f.x * (float)(N1 * b) * inv, &sn, &cs);
            tlo[sq * LP + b] = make_float2(cs, sn);
        } else {
            // upper class: Y = G exp(2 i phi - 2 pi i delta) conj(Z)
            sincospif(2.0f * f.y - 2.0f * f.x, &sn, &cs);
            qup[sq] = make_float2(cs, sn);
        }
    }
    if ((int)threadIdx.x < Rv) {
        const int q = q0 + threadIdx.x;
        const int h = q / S_, s = q - h * S_;
        const int Sh = min(S_, M - h * S_);
        rowoff[threadIdx.x] = (long long)h * S_ * n * 4 + s * 4;
        rowstride[threadIdx.x] = Sh * 4;
    }
    __syncthreads();

    // in-place DIF FFT over the 2 Rv sequences
    dif_all<N2, N2>(buf, 2 * R2, p.tw2);   // twiddles read through the L1 cache

    // epilogue: rotate, gain, quantise, corner turn
    const bool upper = (k1 != 0 && k1 != H1);
    const int nslot = upper ? N2 : N2 / 2;
    // each thread keeps one spectrum r (kP2Threads is a multiple of R2) and
    // walks the slots k2; lanes with consecutive r write consecutive 4-byte
    // cells of one channel row
    const int r = threadIdx.x % R2;
    if (r >= Rv) return;
    int8_t *out_r = p.out + (long long)ant * M * n * 4 + rowoff[r];
    const int rs = rowstride[r];
    const float2 *F0 = buf + r * LD, *F1 = buf + (R2 + r) * LD;
    const float2 *th0 = thi + r * HP, *th1 = thi + (R2 + r) * HP;
    const float2 *tl0 = tlo + r * LP, *tl1 = tlo + (R2 + r) * LP;
    const float2 qu0 = qup[r], qu1 = qup[R2 + r];
    // the gain set of this spectrum in each polarisation
    const int gs0 = p.gsel ? p.gsel[(long long)(ant * 2) * M + q0 + r] : 0;
    const int gs1 = p.gsel ? p.gsel[(long long)(ant * 2 + 1) * M + q0 + r] : 0;
    const float2 *gain0 = p.gains + ((long long)(ant * 2) * p.n_gsets_max + gs0) * n;
    const float2 *gain1 = p.gains + ((long long)(ant * 2 + 1) * p.n_gsets_max + gs1) * n;
    float2 *pre0 = p.prequant ? p.prequant + ((long long)(ant * 2) * M + q0 + r) * n : nullptr;
    float2 *pre1 = p.prequant ? p.prequant + ((long long)(ant * 2 + 1) * M + q0 + r) * n : nullptr;
#pragma unroll 4
    for (int k2 = threadIdx.x / R2; k2 < nslot; k2 += kP2Threads / R2) {
        const bool up = k2 >= N2 / 2;
        const int kc = k1 + N1 * k2;                    // this slot's DFT index
        const int k = up ? N - kc : kc;                 // channel written
        const int a = k2 / S::LO, b = k2 % S::LO;
        const int pos = pad(dif_pos<N2>(k2));
        const float2 z0 = cmul(cmul(th0[a], tl0[b]), F0[pos]);
        const float2 z1 = cmul(cmul(th1[a], tl1[b]), F1[pos]);
        const float2 g0 = __ldg(gain0 + k), g1 = __ldg(gain1 + k);
        const float2 y0 = up ? cmul(cmul(g0, qu0), cconj(z0)) : cmul(g0, z0);
        const float2 y1 = up ? cmul(cmul(g1, qu1), cconj(z1)) : cmul(g1, z1);
        if (pre0) {
            pre0[k] = y0;
            pre1[k] = y1;
        }
        const unsigned packed = ((unsigned)quant8(y0.x) & 0xFFu) | (((unsigned)quant8(y0.y) & 0xFFu) << 8) |
                                (((unsigned)quant8(y1.x) & 0xFFu) << 16) | ((unsigned)quant8(y1.y) << 24);
        *reinterpret_cast<unsigned *>(out_r + (long long)k * rs) = packed;
    }
}

size_t phase2_smem_bytes(int N2, int R2) {
    const int LD = N2 + N2 / 16 + 1;
    const int LO = N2 < 32 ? N2 : 32, HI = N2 / LO;
    return sizeof(float2) * ((size_t)2 * R2 * LD + 2 * R2 * ((HI + 1) + (LO + 1) + 1)) +
           (sizeof(long long) + sizeof(int)) * R2;
}

template <int N2, bool HALF_IN>
static cudaError_t launch_p2h(const Phase2Params &p, int n_ant, cudaStream_t s) {
    const int R2 = P2Shape<N2>::R2;
    if (p.R2 != R2) return cudaErrorInvalidValue;
    const size_t smem = phase2_smem_bytes(N2, R2);
    cudaError_t e = cudaFuncSetAttribute(k_phase2<N2, HALF_IN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(p.N1 / 2 + 1, (p.q_count + R2 - 1) / R2, n_ant);
    k_phase2<N2, HALF_IN><<<grid, kP2Threads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int N2>
static cudaError_t launch_p2(const Phase2Params &p, int n_ant, cudaStream_t s) {
    return p.half_in ? launch_p2h<N2, true>(p, n_ant, s) : launch_p2h<N2, false>(p, n_ant, s);
}

cudaError_t launch_phase2(int N2, const Phase2Params &p, int n_ant, cudaStream_t s) {
    switch (N2) {
        case 2: return launch_p2<2>(p, n_ant, s);
        case 4: return launch_p2<4>(p, n_ant, s);
        case 8: return launch_p2<8>(p, n_ant, s);
        case 16: return launch_p2<16>(p, n_ant, s);
        case 32: return launch_p2<32>(p, n_ant, s);
        case 64: return launch_p2<64>(p, n_ant, s);
        case 128: return launch_p2<128>(p, n_ant, s);
        case 256: return launch_p2<256>(p, n_ant, s);
        case 512: return launch_p2<512>(p, n_ant, s);
        case 1024: return launch_phase2w(p, n_ant, s);   // one warp per 1024-point sequence
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fe
