// Phase 1 of the fused F-engine: 10-bit unpack, coarse delay, PFB FIR (Eq. 1)
// and the first stage of the four-step real DFT.
//
// Four-step split of the N-point DFT of one spectrum's filtered samples g:
//   t = N2 t1 + t2, k = k1 + N1 k2,
//   X[k1 + N1 k2] = sum_t2 exp(-2 pi i k2 t2 / N2) * B[k1][t2],
//   B[k1][t2]     = exp(-2 pi i k1 t2 / N) * sum_t1 g[N2 t1 + t2] exp(-2 pi i k1 t1 / N1).
// g is real, so only k1 in [0, N1/2] is kept (the rest is the conjugate).
//
// One CTA owns kP1Rows consecutive output spectra x C = N1 * W columns
// {N2 t1 + t2 : t1 < N1, t2 in [t2_0, t2_0 + W)} of one (antenna, pol)
// stream. Output row r is the FIR over input rows r .. r + T - 1 (input row
// i holds the samples of spectrum q0 + i; Eq. 1's w[t + N j] weights row
// r + j). For each run of output rows with one coarse delay (Sec. 3.3: each
// PFB window uses one consistent delay) it
//   1. unpacks the run's input rows into shared memory as FP32 (exact for
//      10-bit integers): four lanes share a row segment (row, t1) of W
//      samples and decode whole 5-byte groups aligned to the packed stream,
//      so a segment is stored with its 0-3 sample misalignment;
//   2. runs the T-tap FIR down each column: each thread owns two columns
//      (packed FP32x2 FMAs) and a ring of T + 1 input rows in registers, and
//      emits output rows in pairs (two independent FMA chains), writing g in
//      place;
// and finally, for each (output row, t2), does the real N1-point DFT over
// t1 in registers, multiplies by the twiddle and stores B to the
// intermediate.
#pragma once
#include <cuda_fp16.h>

#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

constexpr int kP1Threads = 256;

template <int T, int N1, int W>
struct P1Shape {
    static constexpr int R = kP1Rows;
    static constexpr int NG = (W + 3) / 4 + 1;   // 4-sample groups per row segment
    static constexpr int SW = 4 * NG;            // shared-memory floats per row segment
    static constexpr int ROW = N1 * SW;          // floats per buffered row
    static constexpr int C = N1 * W;             // FIR columns per tile
    static constexpr int ROWS = R + T - 1;       // input rows of a full tile
    static constexpr int NI = (NG + 3) / 4;      // groups per lane per segment
    static constexpr int SPT = 2;                // segments per 4-lane group per batch
};

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

// Packed words of one chunk's row segments, loaded ahead of their decode.
template <class S>
struct P1Pending {
    unsigned w0[S::SPT][S::NI], w1[S::SPT][S::NI], j[S::SPT], ga[S::SPT];
    int mode[S::SPT];   // 0 nothing, 1 fast (words loaded), 2 slow (decoded with its own loads)
    int dst[S::SPT];    // float offset of the segment in the buffer
};

struct P1Stream {
    const uint8_t *chunk, *hist;
    unsigned rel0, H, HL;   // relative sample index of (input row 0, t1 0, w 0); history; history + chunk
};

// Issue the loads of segments seg0 + u * (kP1Threads / 4) + (this lane's
// slot), u < SPT, of input rows [i0, i_end): segment (i - i0) * N1 + t1.
// Four lanes share a segment: lane l4 takes groups l4 + 4 k, 20 k bytes
// apart, so its byte alignment and word offsets are fixed per segment. A
// warp's 8 segments are permuted so that the two sharing an 8-lane phase of
// the 16-byte stores are 4 apart in t1 (4 SW floats: no bank conflicts).
template <class S, int N1>
__device__ __forceinline__ void p1_load(P1Pending<S> &pd, const P1Stream &st, int seg0, int i0, int i_end, int N,
                                        int N2) {
    const int l4 = threadIdx.x & 3, sl = (threadIdx.x >> 2) & 7;
    const int seg_lane = (threadIdx.x >> 5) * 8 + (sl & 1) * 4 + (sl >> 1);
    const int nseg = (i_end - i0) * N1;
#pragma unroll
    for (int u = 0; u < S::SPT; u++) {
        const int seg = seg0 + u * (kP1Threads / 4) + seg_lane;
        const int t1 = seg & (N1 - 1), i = i0 + seg / N1;
        pd.mode[u] = 0;
        pd.j[u] = 0u;
        pd.ga[u] = 0u;
        pd.dst[u] = i * S::ROW + t1 * S::SW;
        if (seg < nseg) {
            // sample indices relative to the first history sample fit 32 bits
            // (the plan keeps H + L < 2^31)
            const unsigned ga = (st.rel0 + (unsigned)(N * i + N2 * t1)) & ~3u;   // first group's sample
            const unsigned ge = ga + 4u * S::NG;                                 // one past the last
            pd.ga[u] = ga;
            const bool in_hist = ge <= st.H, in_chunk = ga >= st.H && ge <= st.HL;
            pd.mode[u] = (in_hist || in_chunk) ? 1 : 2;
            if (pd.mode[u] == 1) {
                const unsigned bl = ((in_hist ? ga : ga - st.H) >> 2) * 5u + 5u * l4;
                const unsigned *wp =
                    reinterpret_cast<const unsigned *>((in_hist ? st.hist : st.chunk) + (bl & ~3u));
                pd.j[u] = bl & 3u;
#pragma unroll
                for (int k = 0; k < S::NI; k++) {
                    if (l4 + 4 * k < S::NG) {
                        pd.w0[u][k] = __ldg(wp + 5 * k);
                        pd.w1[u][k] = __ldg(wp + 5 * k + 1);
                    }
                }
            }
        }
    }
}

template <class S>
__device__ __forceinline__ void p1_decode(const P1Pending<S> &pd, const P1Stream &st, float *buf) {
    const int l4 = threadIdx.x & 3;
#pragma unroll
    for (int u = 0; u < S::SPT; u++) {
        float *dst = buf + pd.dst[u];
        if (pd.mode[u] == 1) {
#pragma unroll
            for (int k = 0; k < S::NI; k++)
                if (l4 + 4 * k < S::NG)
                    *reinterpret_cast<float4 *>(dst + 4 * l4 + 16 * k) =
                        decode_group_perm(pd.w0[u][k], pd.w1[u][k], pd.j[u]);
        } else if (pd.mode[u] == 2) {
            // straddles the history/chunk boundary or the end of the received
            // samples (zeros past it)
            for (int gi = l4; gi < S::NG; gi += 4) {
                const unsigned g = pd.ga[u] + 4u * gi;
                unsigned v0 = 0u, v1 = 0u, j = 0u;
                if (g < st.HL) {
                    const bool h = g < st.H;
                    const unsigned bb = ((h ? g : g - st.H) >> 2) * 5u;
                    const unsigned *wq = reinterpret_cast<const unsigned *>((h ? st.hist : st.chunk) + (bb & ~3u));
                    v0 = __ldg(wq);
                    v1 = __ldg(wq + 1);
                    j = bb & 3u;
                }
                *reinterpret_cast<float4 *>(dst + 4 * gi) = decode_group_perm(v0, v1, j);
            }
        }
    }
}

template <int T, int N1, int W, bool HALF>
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
    P1Stream st;
    st.chunk = p.chunk + (long long)stream * p.chunk_bytes;
    st.hist = p.hist + (long long)stream * p.hist_bytes;
    st.H = (unsigned)p.H;
    st.HL = (unsigned)(p.H + p.L);
    // rel index (from the first history sample) of input row 0, column t = 0, before the delay
    const long long rel_base = (long long)N * (p.m0 + q0) - (p.t_in - p.H) + t2_0;

    for (int i = threadIdx.x; i < Rv; i += kP1Threads) c_sm[i] = p.ctab[(long long)stream * p.M + q0 + i];
    for (int i = threadIdx.x; i < (H1 + 1) * W; i += kP1Threads) {
        const int k = i / W, w = i % W;
        tw1_sm[i] = __ldg(p.tw1 + (long long)k * N2 + t2_0 + w);
    }
    __syncthreads();

    P1Pending<S> pd;
    int ra = 0;
    while (ra < Rv) {
        const int cd = c_sm[ra];
        int rb = ra + 1;
        while (rb < Rv && c_sm[rb] == cd) rb++;
        const long long rel0 = rel_base - cd;   // rel of (input row 0, t1 0, w 0) at this delay
        st.rel0 = (unsigned)rel0;
        const int off = (int)(rel0 & 3);         // misalignment of every segment of the run
        const int i_end = rb + T - 1;            // input rows [ra, i_end)
        // 1. unpack, SPT segments per 4-lane group per batch with all their
        // loads in flight before the first decode
        for (int seg0 = 0; seg0 < (i_end - ra) * N1; seg0 += S::SPT * (kP1Threads / 4)) {
            p1_load<S, N1>(pd, st, seg0, ra, i_end, N, N2);
            p1_decode<S>(pd, st, xs);
        }
        __syncthreads();
        if (p.window_tap) {
            // the window tap of output row r is its first input row, i = r
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
                // ring of T + 1 input rows
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
                if constexpr ((R & 1) != 0) {
                    // R odd: the last output row has no partner
                    constexpr int r = R - 1;
                    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int j = 0; j < T; j++) acc = __ffma2_rn(w2[j], win[(r + j) % (T + 1)], acc);
                    xa[r * S::ROW] = acc.x;
                    xb[r * S::ROW] = acc.y;
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
    for (int e = threadIdx.x; e < Rv * W; e += kP1Threads) {
        const int r = e / W, w = e % W;
        const float *g = xs + r * S::ROW + off_sm[r] + w;
        float x[N1];
#pragma unroll
        for (int t1 = 0; t1 < N1; t1++) x[t1] = g[t1 * S::SW];
        float2 X[H1 + 1];
        rdft_reg<N1>(x, X);
        const long long o = ((long long)stream * p.a_spectra + (q0 - p.q_begin) + r) * (H1 + 1) * N2 + t2_0 + w;
        const float2 t0 = tw1_sm[w];   // exp(0), times the plan's scale
        const float2 th = tw1_sm[H1 * W + w];
        float2 b[H1 + 1];
        b[0] = make_float2(X[0].x * t0.x, X[0].x * t0.y);
#pragma unroll
        for (int k = 1; k < H1; k++) b[k] = cmul(X[k], tw1_sm[k * W + w]);
        b[H1] = make_float2(X[H1].x * th.x, X[H1].x * th.y);
        if constexpr (HALF) {
            // FP16 (re, im) pairs: the rounding the FP16 second stage applies to its operands anyway
            __half2 *out = reinterpret_cast<__half2 *>(p.A) + o;
#pragma unroll
            for (int k = 0; k <= H1; k++) out[(long long)k * N2] = __floats2half2_rn(b[k].x, b[k].y);
        } else {
            float2 *out = p.A + o;
#pragma unroll
            for (int k = 0; k <= H1; k++) out[(long long)k * N2] = b[k];
        }
    }
}

template <int T, int N1, int W, bool HALF = false>
cudaError_t launch_phase1_tw(const Phase1Params &p, int n_streams, cudaStream_t s) {
    using S = P1Shape<T, N1, W>;
    if (p.W != W || p.N2 % W) return cudaErrorInvalidValue;
    const size_t smem = (size_t)S::ROWS * S::ROW * sizeof(float);
    cudaError_t e =
        cudaFuncSetAttribute(k_phase1<T, N1, W, HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(p.N2 / W, (p.q_count + kP1Rows - 1) / kP1Rows, n_streams);
    k_phase1<T, N1, W, HALF><<<grid, kP1Threads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int T>
cudaError_t launch_phase1_n1(int N1, const Phase1Params &p, int n_streams, cudaStream_t s) {
    if (p.half_out) {
        // FP16 intermediate: the splits with a 1024-point second stage
        switch (N1 * 1000 + p.W) {
            case 8064: return launch_phase1_tw<T, 8, 64, true>(p, n_streams, s);
            case 16032: return launch_phase1_tw<T, 16, 32, true>(p, n_streams, s);
            case 32016: return launch_phase1_tw<T, 32, 16, true>(p, n_streams, s);
            case 64008: return launch_phase1_tw<T, 64, 8, true>(p, n_streams, s);
            default: return cudaErrorInvalidValue;
        }
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
