// Phase 1 of the fused F-engine: 10-bit unpack, coarse delay, PFB FIR (Eq. 1)
// and the first stage of the four-step real DFT.
//
// Four-step split of the N-point DFT of one spectrum's filtered samples g:
//   t = N2 t1 + t2, k = k1 + N1 k2,
//   X[k1 + N1 k2] = sum_t2 exp(-2 pi i k2 t2 / N2) * B[k1][t2],
//   B[k1][t2]     = exp(-2 pi i k1 t2 / N) * sum_t1 g[N2 t1 + t2] exp(-2 pi i k1 t1 / N1).
// g is real, so only k1 in [0, N1/2] is kept (the rest is the conjugate).
//
// One CTA owns a tile of kP1Rows consecutive spectra x C = N1 * W columns
// {N2 t1 + t2 : t1 < N1, t2 in [t2_0, t2_0 + W)} of one (antenna, pol)
// stream. For each run of spectra with one coarse delay (Sec. 3.3: each PFB
// window uses one consistent delay) it
//   1. unpacks the (rows + T - 1) x N1 row segments of delayed samples into
//      shared memory as FP32 (exact for 10-bit integers): every thread decodes
//      whole 5-byte groups of 4 samples aligned to the packed stream, so each
//      segment of W samples is stored with its 0-3 sample misalignment;
//   2. runs the T-tap FIR down each column with the weights and a sliding
//      window of T samples in registers (one shared-memory load and T FMAs
//      per output), writing g in place;
// and finally, for each (spectrum, t2), does the real N1-point DFT over t1
// in registers (an N1/2-point complex FFT of even/odd pairs plus the split),
// multiplies by the twiddle and stores B to the intermediate.
#pragma once
#include "fe_device.cuh"
#include "fe_mma.cuh"
#include "fe_internal.cuh"

namespace fe {

constexpr int kP1Threads = 256;

template <int T, int N1, int W>
struct P1Shape {
    static constexpr int R = kP1Rows;
    static constexpr int NG = (W + 3) / 4 + 1;   // 4-sample groups per row segment
    static constexpr int SW = 4 * NG;            // shared-memory floats per row segment
    static constexpr int ROW = N1 * SW;          // floats per tile row
    static constexpr int C = N1 * W;             // FIR columns per tile
    static constexpr int ROWS = R + T - 1;
};

constexpr int kUB = 8;   // unpack groups per thread per batch

// A 5-byte group at packed byte b of a 4-byte aligned buffer whose length is
// a multiple of 4 is read with the two aligned 32-bit words at b & ~3: the
// group ends at b + 5 <= length, so length - (b & ~3) >= 5 and, being a
// multiple of 4, >= 8 -- both words are inside the buffer.

// Exact float of the 10-bit two's-complement field in the low bits of x:
// (field ^ 512) is the offset-binary value in [0, 1024), placed in the
// mantissa of 2^23 and the bias 2^23 + 512 subtracted (both steps exact).
__device__ __forceinline__ float field10_to_float(unsigned x) {
    return __uint_as_float(((x & 0x3FFu) ^ 0x200u) | 0x4B000000u) - 8389120.0f;
}

// 4 samples of the 5-byte group whose first byte is byte j of w0 (the group
// continues into w1): byte permutes build the group's bits 0-31 and 8-39 in
// big-endian order, and the four 10-bit fields are shifted out of them.
// All-zero words decode to four zero samples (a zero field is the value 0),
// which is what a group past the received samples must read as.
__device__ __forceinline__ float4 decode_group_perm(unsigned w0, unsigned w1, unsigned j) {
    const unsigned hi = __byte_perm(w0, w1, 0x0123u + j * 0x1111u);   // group bits 0..31
    const unsigned lo = __byte_perm(w0, w1, 0x1234u + j * 0x1111u);   // group bits 8..39
    return make_float4(field10_to_float(hi >> 22), field10_to_float(lo >> 20), field10_to_float(lo >> 10),
                       field10_to_float(lo));
}

// ---- reduced-precision form: the 16-point real DFT over t1 on tensor cores
//
// For one spectrum row r and 8 consecutive t2 columns the DFT is the real
// 16 x 16 x 8 product D x G, D[m][t] = cos(2 pi m t / 16) for m < 8,
// D[8][t] = cos(pi t), D[8 + k][t] = -sin(2 pi k t / 16) for k = 1..7, so
// that rows m and m + 8 of the result, held by the same lane of
// mma.m16n8k16, are Re and Im of A[m] (m >= 1) or A[0] and A[8] (m = 0).
// FP16: one MMA with FP16 operands and FP32 accumulation. BF16: the
// operands are split into bf16 hi + lo parts and three MMAs
// (hi.hi + hi.lo + lo.hi) keep the product near FP32 accuracy. Inputs are
// scaled by the plan's power of two p.dft_scale (from the weights' bound, so
// every D x G fits FP16) and the results by its inverse.

// D[m][t] of the 16-point real DFT in the row layout above.
// (Evaluated once per thread with sincospif on the exactly reduced phase
// (m t mod 16) / 8; the values are rounded to FP16/BF16 afterwards.)
__device__ __forceinline__ float dft16_entry(int m, int t) {
    if (m == 8) return (t & 1) ? -1.0f : 1.0f;
    const int k = m < 8 ? m : m - 8;
    float s, c;
    sincospif((float)((k * t) & 15) / 8.0f, &s, &c);
    return m < 8 ? c : -s;
}

template <int PREC, int ROW, int SW, int W>
__device__ __forceinline__ void dft16_tensor(const Phase1Params &p, const float *xs, const int *off_sm,
                                             const float2 *tw1_sm, int Rv, int stream, int q0, int t2_0) {
    constexpr int H1 = 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, c = lane & 3;
    // A fragments (rows g, g+8; columns 2c, 2c+1, 2c+8, 2c+9)
    unsigned ahi[4], alo[4];
    {
        const int rows[4] = {g, g + 8, g, g + 8}, cols[4] = {2 * c, 2 * c, 2 * c + 8, 2 * c + 8};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const float v0 = dft16_entry(rows[i], cols[i]), v1 = dft16_entry(rows[i], cols[i] + 1);
            ahi[i] = pack2<PREC>(v0, v1);
            if constexpr (PREC == 2) alo[i] = pack2<PREC>(v0 - bf16_round(v0), v1 - bf16_round(v1));
        }
    }
    const float sc = p.dft_scale, usc = 1.0f / p.dft_scale;
    const int N2 = p.N2;
    constexpr int NT = W / 8;                      // n-tiles per spectrum row
    for (int tile = warp; tile < Rv * NT; tile += kP1Threads / 32) {
        const int r = tile / NT, w0 = (tile % NT) * 8;
        const float *x = xs + r * ROW + off_sm[r] + w0 + g;   // column n = g of the tile
        const float x0 = x[(2 * c) * SW] * sc, x1 = x[(2 * c + 1) * SW] * sc;
        const float x8 = x[(2 * c + 8) * SW] * sc, x9 = x[(2 * c + 9) * SW] * sc;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        const unsigned b0 = pack2<PREC>(x0, x1), b1 = pack2<PREC>(x8, x9);
        mma16816<PREC>(d, ahi, b0, b1);
        if constexpr (PREC == 2) {
            const unsigned l0 = pack2<PREC>(x0 - bf16_round(x0), x1 - bf16_round(x1));
            const unsigned l1 = pack2<PREC>(x8 - bf16_round(x8), x9 - bf16_round(x9));
            mma16816<PREC>(d, ahi, l0, l1);
            mma16816<PREC>(d, alo, b0, b1);
        }
        // lane holds columns 2c, 2c+1 of rows g (Re A[g]) and g + 8 (Im A[g], or
        // A[8] for g = 0, whose own Im is zero); every lane stores A[g], the
        // g = 0 lanes store A[8] as well
        const int w = w0 + 2 * c, t2 = t2_0 + w;
        float2 *out = p.A + ((long long)stream * p.a_spectra + (q0 - p.q_begin) + r) * (H1 + 1) * N2 + t2;
        const float i0 = g ? d[2] : 0.f, i1 = g ? d[3] : 0.f;
        const float2 e0 = cmul(make_float2(d[0] * usc, i0 * usc), tw1_sm[g * W + w]);
        const float2 e1 = cmul(make_float2(d[1] * usc, i1 * usc), tw1_sm[g * W + w + 1]);
        *reinterpret_cast<float4 *>(out + (long long)g * N2) = make_float4(e0.x, e0.y, e1.x, e1.y);
        if (g == 0) {
            const float2 f0 = cmul(make_float2(d[2] * usc, 0.f), tw1_sm[8 * W + w]);
            const float2 f1 = cmul(make_float2(d[3] * usc, 0.f), tw1_sm[8 * W + w + 1]);
            *reinterpret_cast<float4 *>(out + (long long)8 * N2) = make_float4(f0.x, f0.y, f1.x, f1.y);
        }
    }
}

template <int T, int N1, int W, int PREC = 0>
__global__ void __launch_bounds__(kP1Threads, 2) k_phase1(const Phase1Params p) {
    using S = P1Shape<T, N1, W>;
    constexpr int R = S::R, H1 = N1 / 2;
    extern __shared__ float xs[];              // [ROWS][N1][SW]
    __shared__ int c_sm[R];
    __shared__ int off_sm[R];                  // segment misalignment of each row's run
    __shared__ float2 tw1_sm[(H1 + 1) * W];    // exp(-2 pi i k1 t2 / N) for this tile's t2

    const int N = p.N, N2 = p.N2;
    const int stream = blockIdx.z;
    const int t2_0 = blockIdx.x * W;
    const int q0 = p.q_begin + blockIdx.y * R;
    const int Rv = min(R, p.q_begin + p.q_count - q0);
    const uint8_t *chunk = p.chunk + (long long)stream * p.chunk_bytes;
    const uint8_t *hist = p.hist + (long long)stream * p.hist_bytes;
    const long long HL = p.H + p.L;
    // rel index (from the first history sample) of tile row 0, column t = 0, before the delay
    const long long rel_base = (long long)N * (p.m0 + q0) - (p.t_in - p.H) + t2_0;

    for (int i = threadIdx.x; i < Rv; i += kP1Threads) c_sm[i] = p.ctab[(long long)stream * p.M + q0 + i];
    for (int i = threadIdx.x; i < (H1 + 1) * W; i += kP1Threads) {
        const int k = i / W, w = i % W;
        tw1_sm[i] = __ldg(p.tw1 + (long long)k * N2 + t2_0 + w);
    }
    __syncthreads();

    int off = 0;   // misalignment (0..3) of every segment of the current run
    int ra = 0;
    while (ra < Rv) {
        const int cd = c_sm[ra];
        int rb = ra + 1;
        while (rb < Rv && c_sm[rb] == cd) rb++;
        const long long rel0 = rel_base - cd;  // rel of (row 0, t1 0, w 0) at this delay
        off = (int)(rel0 & 3);
        // 1. unpack rows [ra, rb + T - 1), whole aligned groups
        const int rows = rb + T - 1 - ra;
        const int ngroups = rows * N1 * S::NG;
        // batches of kUB groups per thread: all word loads of a batch are in
        // flight before the first is decoded
        // sample indices relative to the first history sample fit 32 bits (the
        // plan keeps H + L < 2^31)
        const unsigned rel0u = (unsigned)rel0, Hu = (unsigned)p.H, HLu = (unsigned)HL;
        for (int e0 = 0; e0 < ngroups; e0 += kUB * kP1Threads) {
            unsigned w0[kUB], w1[kUB], j[kUB];
            int dst[kUB];
#pragma unroll
            for (int u = 0; u < kUB; u++) {
                const int e = e0 + u * kP1Threads + threadIdx.x;
                dst[u] = -1;
                w0[u] = w1[u] = 0u;
                j[u] = 0u;
                if (e < ngroups) {
                    const int gi = e % S::NG;
                    const int seg = e / S::NG;
                    const int t1 = seg % N1, row = ra + seg / N1;
                    const unsigned g = ((rel0u + (unsigned)(N * row + N2 * t1)) & ~3u) + 4u * gi;
                    dst[u] = row * S::ROW + t1 * S::SW + 4 * gi;
                    if (g < HLu) {   // else past the received samples: zeros
                        const bool h = g < Hu;
                        const unsigned b = ((h ? g : g - Hu) >> 2) * 5u;
                        const unsigned *wp = reinterpret_cast<const unsigned *>((h ? hist : chunk) + (b & ~3u));
                        w0[u] = __ldg(wp);
                        w1[u] = __ldg(wp + 1);
                        j[u] = b & 3u;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kUB; u++) {
                if (dst[u] < 0) continue;
                *reinterpret_cast<float4 *>(xs + dst[u]) = decode_group_perm(w0[u], w1[u], j[u]);
            }
        }
        __syncthreads();
        if (p.window_tap) {
            for (int e = threadIdx.x; e < (rb - ra) * S::C; e += kP1Threads) {
                const int row = ra + e / S::C, col = e % S::C;
                const int t1 = col / W, w = col % W;
                p.window_tap[((long long)stream * p.M + q0 + row) * N + N2 * t1 + t2_0 + w] =
                    (int)xs[row * S::ROW + t1 * S::SW + off + w];
            }
            __syncthreads();   // the FIR below overwrites these slots in place
        }
        // 2. FIR down each column, g written over the row it starts at
        if (ra == 0 && rb == R) {
            // one delay for the whole tile: no predicates, two columns per
            // thread (c and c + C/2) through packed FP32x2 FMAs
            for (int pc = threadIdx.x; pc < S::C / 2; pc += kP1Threads) {
                const int ca = pc, cb = pc + S::C / 2;
                const int ta = N2 * (ca / W) + t2_0 + ca % W, tb = N2 * (cb / W) + t2_0 + cb % W;
                float *xa = xs + (ca / W) * S::SW + off + ca % W;
                float *xb = xs + (cb / W) * S::SW + off + cb % W;
                // outputs in pairs (r, r + 1), two independent FMA chains, from a
                // ring of T + 1 window rows
                float2 w2[T], win[T + 1];
#pragma unroll
                for (int j = 0; j < T; j++)
                    w2[j] = make_float2(__ldg(p.w + ta + (long long)N * j), __ldg(p.w + tb + (long long)N * j));
#pragma unroll
                for (int row = 0; row < R + T - 1; row++) {
                    win[row % (T + 1)] = make_float2(xa[row * S::ROW], xb[row * S::ROW]);
                    const int r = row - T;      // pair (r, r + 1) is complete once row r + T is in
                    if (r >= 0 && (r & 1) == 0) {
                        float2 acc0 = make_float2(0.0f, 0.0f), acc1 = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int j = 0; j < T; j++) {
                            acc0 = __ffma2_rn(w2[j], win[(r + j) % (T + 1)], acc0);
                            acc1 = __ffma2_rn(w2[j], win[(r + 1 + j) % (T + 1)], acc1);
                        }
                        xa[r * S::ROW] = acc0.x;
                        xb[r * S::ROW] = acc0.y;
                        xa[(r + 1) * S::ROW] = acc1.x;
                        xb[(r + 1) * S::ROW] = acc1.y;
                    }
                }
            }
        } else
        for (int col = threadIdx.x; col < S::C; col += kP1Threads) {
            const int t1 = col / W, w = col % W;
            const int t = N2 * t1 + t2_0 + w;
            float *x = xs + t1 * S::SW + off + w;
            float wr[T], win[T];
#pragma unroll
            for (int j = 0; j < T; j++) wr[j] = __ldg(p.w + t + (long long)N * j);
#pragma unroll
            for (int row = 0; row < R + T - 1; row++) {
                if (row >= ra && row < rb + T - 1) win[row % T] = x[row * S::ROW];
                const int r = row - (T - 1);
                if (r >= ra && r < rb) {
                    float acc = 0.0f;
#pragma unroll
                    for (int j = 0; j < T; j++) acc = fmaf(wr[j], win[(r + j) % T], acc);
                    x[r * S::ROW] = acc;
                }
            }
        }
        for (int r = ra + (int)threadIdx.x; r < rb; r += kP1Threads) off_sm[r] = off;
        __syncthreads();
        ra = rb;
    }

    // 3. real N1-point DFT over t1, twiddle, store B[k1][t2]
    if constexpr (PREC != 0) {
        dft16_tensor<PREC, S::ROW, S::SW, W>(p, xs, off_sm, tw1_sm, Rv, stream, q0, t2_0);
    } else
    for (int pi = threadIdx.x; pi < Rv * W; pi += kP1Threads) {
        const int r = pi / W, w = pi % W;
        const float *g = xs + r * S::ROW + off_sm[r] + w;
        float2 z[H1];
#pragma unroll
        for (int q = 0; q < H1; q++) z[q] = make_float2(g[(2 * q) * S::SW], g[(2 * q + 1) * S::SW]);
        fft_regc<H1>(z);
        float2 *out = p.A + ((long long)stream * p.a_spectra + (q0 - p.q_begin) + r) * (H1 + 1) * N2 + t2_0 + w;
#pragma unroll
        for (int k = 0; k <= H1; k++) {
            const float2 zk = z[k % H1], zm = z[(H1 - k) % H1];
            // even part E = (Z[k] + conj Z[H1-k]) / 2, odd part O = (Z[k] - conj Z[H1-k]) / 2i
            const float2 E = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            const float2 O = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
            const float2 a = cadd(E, k == H1 ? make_float2(-O.x, -O.y) : cmul_tw64c(O, k * (64 / N1)));
            out[(long long)k * N2] = cmul(a, tw1_sm[k * W + w]);
        }
    }
}

template <int T, int N1, int W, int PREC = 0>
cudaError_t launch_phase1_tw(const Phase1Params &p, int n_streams, cudaStream_t s) {
    using S = P1Shape<T, N1, W>;
    if (p.W != W || p.N2 % W) return cudaErrorInvalidValue;
    const size_t smem = (size_t)S::ROWS * S::ROW * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_phase1<T, N1, W, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(p.N2 / W, (p.q_count + kP1Rows - 1) / kP1Rows, n_streams);
    k_phase1<T, N1, W, PREC><<<grid, kP1Threads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int T>
cudaError_t launch_phase1_n1(int N1, const Phase1Params &p, int n_streams, cudaStream_t s) {
    if (p.precision != 0) {
        // reduced-precision form: tensor-core 16-point first stage (N1 = 16)
        if (N1 != 16 || p.W != 32) return cudaErrorInvalidValue;
        return p.precision == 1 ? launch_phase1_tw<T, 16, 32, 1>(p, n_streams, s)
                                : launch_phase1_tw<T, 16, 32, 2>(p, n_streams, s);
    }
    switch (N1 * 1000 + p.W) {
        case 8064: return launch_phase1_tw<T, 8, 64>(p, n_streams, s);
        case 16032: return launch_phase1_tw<T, 16, 32>(p, n_streams, s);
        case 32016: return launch_phase1_tw<T, 32, 16>(p, n_streams, s);
        case 64008: return launch_phase1_tw<T, 64, 8>(p, n_streams, s);
        case 8032: return launch_phase1_tw<T, 8, 32>(p, n_streams, s);
        case 8016: return launch_phase1_tw<T, 8, 16>(p, n_streams, s);
        case 8008: return launch_phase1_tw<T, 8, 8>(p, n_streams, s);
        case 8004: return launch_phase1_tw<T, 8, 4>(p, n_streams, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fe
