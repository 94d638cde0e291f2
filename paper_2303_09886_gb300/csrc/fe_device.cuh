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
