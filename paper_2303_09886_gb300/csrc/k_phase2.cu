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
// The CTA writes, for each of its channels, R2 consecutive spectra x 2 pols
// x (re, im) = 4 R2 contiguous bytes of one heap row.
#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

template <int RP>
__device__ __forceinline__ void dft_small(float2 (&v)[RP]);

template <>
__device__ __forceinline__ void dft_small<2>(float2 (&v)[2]) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void dft_small<4>(float2 (&v)[4]) {
    const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const float2 t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
    const float2 mi_t3 = make_float2(t3.y, -t3.x);   // -i * t3
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, mi_t3);
    v[3] = csub(t1, mi_t3);
}

// One radix-RP Stockham pass (self-sorting, decimation in time) over nseq
// sequences of length N2 stored at rows of stride LD. Ns is the length of
// the sub-transforms already done. Butterfly j reads x[j + r N2/RP],
// multiplies by exp(-2 pi i r (j mod Ns) / (Ns RP)), takes an RP-point DFT
// and writes y[(j / Ns) Ns RP + (j mod Ns) + r Ns]. In place: every thread
// holds its butterflies in registers across a barrier.
template <int RP, int K>
__device__ __forceinline__ void stockham_pass(float2 *buf, int LD, int N2, int Ns, int nseq,
                                              const float2 *__restrict__ tw2) {
    const int B = N2 / RP;
    const int slots = (int)blockDim.x * K;
    const int spr = slots / B > 0 ? slots / B : 1;
    const int twstride = N2 / (Ns * RP);
    for (int s0 = 0; s0 < nseq; s0 += spr) {
        float2 v[K][RP];
        int dst[K];
        bool act[K];
#pragma unroll
        for (int kk = 0; kk < K; kk++) {
            const int b = threadIdx.x + kk * blockDim.x;
            const int sq = s0 + b / B, j = b % B;
            act[kk] = (b < spr * B) && (sq < nseq);
            dst[kk] = 0;
            if (act[kk]) {
                const float2 *x = buf + sq * LD;
                const int k = j % Ns;
#pragma unroll
                for (int r = 0; r < RP; r++) {
                    float2 a = x[j + r * B];
                    if (r > 0) a = cmul(a, __ldg(tw2 + r * k * twstride));
                    v[kk][r] = a;
                }
                dft_small<RP>(v[kk]);
                dst[kk] = sq * LD + (j / Ns) * Ns * RP + k;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < K; kk++) {
            if (act[kk]) {
#pragma unroll
                for (int r = 0; r < RP; r++) buf[dst[kk] + r * Ns] = v[kk][r];
            }
        }
        __syncthreads();
    }
}

template <int N2>
__global__ void __launch_bounds__(256) k_phase2(const Phase2Params p) {
    extern __shared__ float2 buf[];            // [2 R2][N2 + 1]
    constexpr int LD = N2 + 1;
    const int k1 = blockIdx.x, ant = blockIdx.z;
    const int R2 = p.R2, q0 = blockIdx.y * R2;
    const int M = p.M, Rv = min(R2, M - q0);
    const int N1 = p.N1, H1 = N1 / 2, N = p.N, n = N / 2, S = p.S;
    const int nseq = 2 * Rv;

    for (int e = threadIdx.x; e < nseq * N2; e += blockDim.x) {
        const int sq = e / N2, t2 = e % N2;
        const int pol = sq / Rv, r = sq - pol * Rv;
        buf[sq * LD + t2] =
            p.A[(((long long)(ant * 2 + pol) * M + q0 + r) * (H1 + 1) + k1) * N2 + t2];
    }
    __syncthreads();

    int Ns = 1;
    while (Ns * 4 <= N2) {
        stockham_pass<4, 4>(buf, LD, N2, Ns, nseq, p.tw2);
        Ns *= 4;
    }
    if (Ns < N2) stockham_pass<2, 4>(buf, LD, N2, Ns, nseq, p.tw2);

    const bool upper = (k1 != 0 && k1 != H1);
    const int nslot = upper ? N2 : N2 / 2;
    const float inv_n2 = 2.0f / (float)N;        // 2 / N, exact
    for (int e = threadIdx.x; e < nslot * Rv; e += blockDim.x) {
        const int r = e % Rv, k2 = e / Rv;
        const bool up = k2 >= N2 / 2;
        const int k = up ? N - (k1 + N1 * k2) : k1 + N1 * k2;
        const int q = q0 + r;
        unsigned packed = 0;
#pragma unroll
        for (int pol = 0; pol < 2; pol++) {
            float2 F = buf[(pol * Rv + r) * LD + k2];
            if (up) F.y = -F.y;
            const int st = ant * 2 + pol;
            const float2 f = p.ftab[(long long)st * M + q];    // (delta, phi / pi)
            float sn, cs;
            sincospif(f.y - f.x * (float)k * inv_n2, &sn, &cs);
            const float2 g = __ldg(p.gains + (long long)st * n + k);
            const float2 y = cmul(cmul(g, make_float2(cs, sn)), F);
            if (p.prequant) p.prequant[((long long)st * M + q) * n + k] = y;
            const unsigned qr = (unsigned)quant8(y.x) & 0xFFu, qi = (unsigned)quant8(y.y) & 0xFFu;
            packed |= (qr | (qi << 8)) << (16 * pol);
        }
        const int h = q / S, s = q - h * S;
        const int Sh = min(S, M - h * S);
        const long long off = (long long)ant * M * n * 4 + (long long)h * S * n * 4 +
                              (long long)k * Sh * 4 + (long long)s * 4;
        *reinterpret_cast<unsigned *>(p.out + off) = packed;
    }
}

size_t phase2_smem_bytes(int N2, int R2) { return (size_t)2 * R2 * (N2 + 1) * sizeof(float2); }

template <int N2>
static cudaError_t launch_p2(const Phase2Params &p, int n_ant, cudaStream_t s) {
    const size_t smem = phase2_smem_bytes(N2, p.R2);
    cudaError_t e = cudaFuncSetAttribute(k_phase2<N2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(p.N1 / 2 + 1, (p.M + p.R2 - 1) / p.R2, n_ant);
    k_phase2<N2><<<grid, 256, smem, s>>>(p);
    return cudaGetLastError();
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
        case 1024: return launch_p2<1024>(p, n_ant, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fe
