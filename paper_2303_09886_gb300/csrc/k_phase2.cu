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
    static constexpr int R2 = phase2_R2_for(N2);                  // spectra per CTA
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
#include "k_phase2_tile.inc"
}

// The tiles of several plans' second stages (same N2) in one grid.
template <int N2, bool HALF_IN>
__global__ void __launch_bounds__(kP2Threads, 3) k_phase2_group(const Phase2Group g) {
    __shared__ Phase2Params sp;
    __shared__ int sxyz[3];
    if (threadIdx.x == 0) {
        const int m = group_member(g, (int)blockIdx.x);
        const int b = (int)blockIdx.x - g.start[m], gy = g.aux[m];
        sxyz[0] = b % g.gx;
        sxyz[1] = (b / g.gx) % gy;
        sxyz[2] = b / (g.gx * gy);
        sp = g.p[m];
    }
    __syncthreads();
    const Phase2Params &p = sp;
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

    const int k1 = sxyz[0], ant = sxyz[2];
    const int q0 = p.q_begin + sxyz[1] * R2;
#include "k_phase2_tile.inc"
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

// the grid launch_phase2 uses for N2 < 1024: (classes k1, tiles of R2 spectra, antennas)
int phase2_blocks(int N2, const Phase2Params &p, int n_ant, int *gx, int *gy) {
    (void)N2;
    *gx = p.N1 / 2 + 1;
    *gy = (p.q_count + p.R2 - 1) / p.R2;
    return *gx * *gy * n_ant;
}

template <int N2, bool HALF_IN>
static cudaError_t launch_p2h_group(const Phase2Group &g, cudaStream_t s) {
    const int R2 = P2Shape<N2>::R2;
    const size_t smem = phase2_smem_bytes(N2, R2);
    cudaError_t e = cudaFuncSetAttribute(k_phase2_group<N2, HALF_IN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    for (int m = 0; m < g.n; m++)
        if (g.p[m].R2 != R2) return cudaErrorInvalidValue;
    if (g.n < 1 || g.start[g.n] < 1) return cudaSuccess;
    k_phase2_group<N2, HALF_IN><<<g.start[g.n], kP2Threads, smem, s>>>(g);
    return cudaGetLastError();
}

template <int N2>
static cudaError_t launch_p2_group(bool half_in, const Phase2Group &g, cudaStream_t s) {
    return half_in ? launch_p2h_group<N2, true>(g, s) : launch_p2h_group<N2, false>(g, s);
}

cudaError_t launch_phase2_group(int N2, bool half_in, const Phase2Group &g, cudaStream_t s) {
    switch (N2) {
        case 2: return launch_p2_group<2>(half_in, g, s);
        case 4: return launch_p2_group<4>(half_in, g, s);
        case 8: return launch_p2_group<8>(half_in, g, s);
        case 16: return launch_p2_group<16>(half_in, g, s);
        case 32: return launch_p2_group<32>(half_in, g, s);
        case 64: return launch_p2_group<64>(half_in, g, s);
        case 128: return launch_p2_group<128>(half_in, g, s);
        case 256: return launch_p2_group<256>(half_in, g, s);
        case 512: return launch_p2_group<512>(half_in, g, s);
        case 1024: return launch_phase2w_group(half_in, g, s);
        default: return cudaErrorInvalidValue;
    }
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
