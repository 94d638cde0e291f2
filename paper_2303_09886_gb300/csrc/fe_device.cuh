// Device helpers shared by the libfengine kernels: complex arithmetic, the
// 10-bit sample fetch, the quantiser and an in-register radix-2 FFT.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fe {

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// Sample j of a packed 10-bit stream (bits [10 j, 10 j + 10), most
// significant bit first, two's complement; Sec. 2.2 fixes 10 bits/sample).
// The field lies in bytes 5j/4 and 5j/4 + 1 at bit offset 2 (j mod 4).
__device__ __forceinline__ int fetch10(const uint8_t *__restrict__ p, long long j) {
    const long long byte = (5 * j) >> 2;
    const int r = 2 * (int)(j & 3);
    unsigned v = ((unsigned)__ldg(p + byte) << 8) | (unsigned)__ldg(p + byte + 1);
    v = (v >> (6 - r)) & 0x3FFu;
    return (int)v - (int)((v & 0x200u) << 1);
}

// Requantise to an 8-bit Gaussian-integer component (Sec. 2.1 step 6,
// Sec. 3.6): saturate to [-127, 127], round half away from zero. Adding the
// largest float below 1/2 with the sign of t and truncating rounds ties away
// from zero and everything else to nearest for |t| <= 127 (FP32 addition is
// correctly rounded, so t + 0.49999997 reaches the next integer exactly when
// frac(|t|) >= 1/2). Host and device evaluate it identically.
__host__ __device__ __forceinline__ int quant8(float x) {
    float t = fminf(fmaxf(x, -127.0f), 127.0f);
    return (int)(t + copysignf(0.49999997f, t));
}

template <int NN>
__host__ __device__ constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 1; b < NN; b <<= 1) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

// exp(-2 pi i q / 64) for q in [0, 32] as compile-time constants (cos and
// sin of multiples of pi/32, evaluated in FP64 and rounded to FP32; the
// exact values 0, +-1 are written exactly so multiplications by them fold).
__host__ __device__ __forceinline__ float2 tw64c(int q) {
    constexpr float c[33] = {
        1.0f, 9.951847196e-01f, 9.807852507e-01f, 9.569403529e-01f, 9.238795042e-01f,
        8.819212914e-01f, 8.314695954e-01f, 7.730104327e-01f, 7.071067691e-01f, 6.343932748e-01f,
        5.555702448e-01f, 4.713967443e-01f, 3.826834261e-01f, 2.902846634e-01f, 1.950903237e-01f,
        9.801714122e-02f, 0.0f, -9.801714122e-02f, -1.950903237e-01f, -2.902846634e-01f,
        -3.826834261e-01f, -4.713967443e-01f, -5.555702448e-01f, -6.343932748e-01f, -7.071067691e-01f,
        -7.730104327e-01f, -8.314695954e-01f, -8.819212914e-01f, -9.238795042e-01f, -9.569403529e-01f,
        -9.807852507e-01f, -9.951847196e-01f, -1.0f};
    // sin(-2 pi q / 64) = -cos(2 pi (16 - q) / 64) = -c[|16 - q|] for q in [0, 32]
    const int m = q <= 16 ? 16 - q : q - 16;
    return make_float2(c[q], -c[m]);
}

// Multiply by a compile-time twiddle exp(-2 pi i q / 64), folding q = 0
// (identity) and q = 16 (-i).
__device__ __forceinline__ float2 cmul_tw64c(float2 a, int q) {
    if (q == 0) return a;
    if (q == 16) return make_float2(a.y, -a.x);
    return cmul(a, tw64c(q));
}

// In-register real DFT of NN points (NN = 2, 4, ..., 64): bins 0..NN/2 of
// X[k] = sum_t x[t] exp(-2 pi i k t / NN), radix-2 decimation in time on the
// real sequence. With E and O the half-length DFTs of the even and odd
// samples (both real sequences, so E[NN/2 - k] = conj E[k]),
//   X[k] = E[k] + w^k O[k],  X[NN/2 - k] = conj(E[k] - w^k O[k]),  k <= NN/4,
// w = exp(-2 pi i / NN); w^(NN/4) = -i and the k = 0 terms are real.
template <int NN>
__device__ __forceinline__ void rdft_reg(const float (&x)[NN], float2 (&X)[NN / 2 + 1]) {
    if constexpr (NN == 2) {
        X[0] = make_float2(x[0] + x[1], 0.0f);
        X[1] = make_float2(x[0] - x[1], 0.0f);
    } else {
        constexpr int H = NN / 2, Q = NN / 4;
        float xe[H], xo[H];
#pragma unroll
        for (int t = 0; t < H; t++) {
            xe[t] = x[2 * t];
            xo[t] = x[2 * t + 1];
        }
        float2 E[Q + 1], O[Q + 1];
        rdft_reg<H>(xe, E);
        rdft_reg<H>(xo, O);
        X[0] = make_float2(E[0].x + O[0].x, 0.0f);
        X[H] = make_float2(E[0].x - O[0].x, 0.0f);
#pragma unroll
        for (int k = 1; k < Q; k++) {
            const float2 t = cmul_tw64c(O[k], k * (64 / NN));
            X[k] = cadd(E[k], t);
            X[H - k] = make_float2(E[k].x - t.x, t.y - E[k].y);
        }
        X[Q] = make_float2(E[Q].x, -O[Q].x);
    }
}

// In-register NN-point complex DFT with compile-time twiddles (NN <= 64),
// radix-2 decimation in time; natural order in and out.
template <int NN>
__device__ __forceinline__ void fft_regc(float2 (&z)[NN]) {
#pragma unroll
    for (int i = 0; i < NN; i++) {
        const int j = bitrev<NN>(i);
        if (i < j) {
            float2 t = z[i];
            z[i] = z[j];
            z[j] = t;
        }
    }
#pragma unroll
    for (int len = 2; len <= NN; len <<= 1) {
#pragma unroll
        for (int i = 0; i < NN; i += len) {
#pragma unroll
            for (int j = 0; j < len / 2; j++) {
                const float2 v = cmul_tw64c(z[i + j + len / 2], j * (64 / len));
                const float2 u = z[i + j];
                z[i + j] = cadd(u, v);
                z[i + j + len / 2] = csub(u, v);
            }
        }
    }
}

// In-register NN-point complex DFT, X[k] = sum_t z[t] exp(-2 pi i k t / NN),
// radix-2 decimation in time; natural order in and out. tw64[q] holds
// exp(-2 pi i q / 64) for q in [0, 32], so NN <= 64.
template <int NN>
__device__ __forceinline__ void fft_reg(float2 (&z)[NN], const float2 *tw64) {
#pragma unroll
    for (int i = 0; i < NN; i++) {
        const int j = bitrev<NN>(i);
        if (i < j) {
            float2 t = z[i];
            z[i] = z[j];
            z[j] = t;
        }
    }
#pragma unroll
    for (int len = 2; len <= NN; len <<= 1) {
#pragma unroll
        for (int i = 0; i < NN; i += len) {
#pragma unroll
            for (int j = 0; j < len / 2; j++) {
                const float2 w = tw64[j * (64 / len)];
                const float2 v = cmul(z[i + j + len / 2], w);
                const float2 u = z[i + j];
                z[i + j] = cadd(u, v);
                z[i + j + len / 2] = csub(u, v);
            }
        }
    }
}

}  // namespace fe
