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
// The same sums as packed FP32x2 instructions (two round-to-nearest adds in
// one; the results are those of cadd and csub).
__device__ __forceinline__ float2 cadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

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
#ifdef __CUDA_ARCH__
    // The truncating conversion to an 8-bit integer saturates at +127 by
    // itself (and at -128, which the lower clamp keeps out of reach); only
    // the low byte of the result is used.
    const float t = fmaxf(x, -127.0f);
    int d;
    asm("cvt.rzi.s8.f32 %0, %1;" : "=r"(d) : "f"(t + copysignf(0.49999997f, t)));
    return d;
#else
    float t = fminf(fmaxf(x, -127.0f), 127.0f);
    return (int)(t + copysignf(0.49999997f, t));
#endif
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

// cos(2 pi q / 64) for q in [0, 32] (FP64 values rounded to FP32; the exact
// values 0 and +-1 are written exactly so that multiplications by them fold).
__host__ __device__ constexpr float cos64(int q) {
    constexpr float c[33] = {
        1.0f, 9.951847196e-01f, 9.807852507e-01f, 9.569403529e-01f, 9.238795042e-01f,
        8.819212914e-01f, 8.314695954e-01f, 7.730104327e-01f, 7.071067691e-01f, 6.343932748e-01f,
        5.555702448e-01f, 4.713967443e-01f, 3.826834261e-01f, 2.902846634e-01f, 1.950903237e-01f,
        9.801714122e-02f, 0.0f, -9.801714122e-02f, -1.950903237e-01f, -2.902846634e-01f,
        -3.826834261e-01f, -4.713967443e-01f, -5.555702448e-01f, -6.343932748e-01f, -7.071067691e-01f,
        -7.730104327e-01f, -8.314695954e-01f, -8.819212914e-01f, -9.238795042e-01f, -9.569403529e-01f,
        -9.807852507e-01f, -9.951847196e-01f, -1.0f};
    return c[q];
}

// a * exp(-2 pi i Q / 64) for a compile-time Q in [0, 32]: Q = 0 and
// Q = 16 (-i) fold to moves; otherwise cos - i sin with sin(2 pi Q / 64) =
// cos(2 pi |16 - Q| / 64).
template <int Q>
__device__ __forceinline__ float2 cmul_w64(float2 a) {
    static_assert(Q >= 0 && Q <= 32, "twiddle index");
    if constexpr (Q == 0) {
        return a;
    } else if constexpr (Q == 16) {
        return make_float2(a.y, -a.x);
    } else {
        constexpr float c = cos64(Q), s = cos64(Q <= 16 ? 16 - Q : Q - 16);
        return cmul(a, make_float2(c, -s));
    }
}

namespace detail {

// X[K] = E[K] + w^K O[K], X[K + NN/2] = E[K] - w^K O[K] for K = K0 .. NN/2 - 1
template <int NN, int K>
__device__ __forceinline__ void dit_combine(float2 (&z)[NN], const float2 (&e)[NN / 2], const float2 (&o)[NN / 2]) {
    if constexpr (K < NN / 2) {
        const float2 t = cmul_w64<K * (64 / NN)>(o[K]);
        z[K] = cadd2(e[K], t);
        z[K + NN / 2] = csub2(e[K], t);
        dit_combine<NN, K + 1>(z, e, o);
    }
}

// bins 1 .. NN/4 - 1 of the real DFT from the half-length DFTs E and O
template <int NN, int K>
__device__ __forceinline__ void rdit_combine(float2 (&X)[NN / 2 + 1], const float2 (&E)[NN / 4 + 1],
                                             const float2 (&O)[NN / 4 + 1]) {
    if constexpr (K < NN / 4) {
        const float2 t = cmul_w64<K * (64 / NN)>(O[K]);
        X[K] = cadd2(E[K], t);
        const float2 d = csub2(E[K], t);
        X[NN / 2 - K] = make_float2(d.x, -d.y);
        rdit_combine<NN, K + 1>(X, E, O);
    }
}

}  // namespace detail

// In-register real DFT of NN points (NN = 2, 4, ..., 64): bins 0..NN/2 of
// X[k] = sum_t x[t] exp(-2 pi i k t / NN), radix-2 decimation in time on the
// real sequence. With E and O the half-length DFTs of the even and odd
// samples (both real sequences, so E[NN/2 - k] = conj E[k]),
//   X[k] = E[k] + w^k O[k],  X[NN/2 - k] = conj(E[k] - w^k O[k]),  k <= NN/4,
// w = exp(-2 pi i / NN); w^(NN/4) = -i and the k = 0 terms are real. Every
// index and twiddle is a compile-time constant.
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
        detail::rdit_combine<NN, 1>(X, E, O);
        X[Q] = make_float2(E[Q].x, -O[Q].x);
    }
}

// In-register NN-point complex DFT (NN = 1, 2, 4, ..., 64), natural order in
// and out: recursive radix-2 decimation in time, every index and twiddle a
// compile-time constant.
template <int NN>
__device__ __forceinline__ void fft_regc(float2 (&z)[NN]) {
    if constexpr (NN > 1) {
        float2 e[NN / 2], o[NN / 2];
#pragma unroll
        for (int t = 0; t < NN / 2; t++) {
            e[t] = z[2 * t];
            o[t] = z[2 * t + 1];
        }
        fft_regc<NN / 2>(e);
        fft_regc<NN / 2>(o);
        detail::dit_combine<NN, 0>(z, e, o);
    }
}

// The member of a grouped launch (GroupArgs) that owns block b: the last m
// with start[m] <= b (binary search over the n members' first blocks).
template <class G>
__device__ __forceinline__ int group_member(const G &g, int b) {
    int lo = 0, hi = g.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace fe
