// Phase 1 of the fused F-engine: 10-bit unpack, coarse delay, PFB FIR
// (Eq. 1) and the first stage of the four-step real DFT.
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
// r + j); every PFB window uses one coarse delay (Sec. 3.3), so a tile is
// processed per run of output rows with one delay.
//
// Each thread owns two FIR columns and decodes their 10-bit samples itself:
// sample s occupies bits [10 s, 10 s + 10) (most significant bit first),
// i.e. bytes 5 s / 4 and 5 s / 4 + 1 at a bit offset 2 (s mod 4) that is the
// same for every row of a column (a row is N samples, a multiple of 4), and
// the row's bytes sit 5 N / 4 further on. A tile of one delay run inside the
// chunk first copies its rows' packed bytes into a shared-memory ring
// (cp.async, a few rows ahead of the FIR) and decodes from there; other tiles
// decode straight from global memory. The FIR keeps T + 1 input rows in a
// register ring and emits output rows in pairs (packed FP32x2 FMAs); g goes
// to shared memory, and for each (output row, t2) the real N1-point DFT over
// t1 runs in registers, is multiplied by the twiddle and stored (FP32 pairs,
// or FP16 pairs for the FP16 form).
#pragma once
#include <cuda_fp16.h>

#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

constexpr int kP1Threads = 256;

template <int T, int N1, int W>
struct P1Shape {
    static constexpr int R = kP1Rows;
    static constexpr int GW = W + 1;         // shared-memory floats per (row, t1) segment of g
    static constexpr int ROW = N1 * GW;      // floats per output row
    static constexpr int C = N1 * W;         // FIR columns per tile
    static constexpr int ROWS = R + T - 1;   // input rows of a full tile
    // Staged input (tiles of one delay run inside the chunk, every thread
    // owning a column pair): the packed bytes of each (input row, t1 segment
    // of W columns) are copied into a shared-memory ring by 16-byte cp.async
    // from the segment's first byte rounded down to 16, SEG bytes (the W
    // samples' bytes plus up to 15 in front and the second byte of the last
    // field), SG rows per commit group, NGRING groups in the ring.
    static constexpr bool STAGED = (C == 2 * kP1Threads);
    static constexpr int SEG = (15 + (5 * (W - 1) + 3) / 4 + 2 + 15) / 16 * 16;
    static constexpr int SG = 8;
    static constexpr int NGRING = (N1 * SEG <= 1024) ? 3 : 2;
    static constexpr int RING = NGRING * SG;
    static constexpr int STAGE_BYTES = STAGED ? RING * N1 * SEG : 0;
    static constexpr size_t SMEM = (size_t)R * ROW * sizeof(float) + STAGE_BYTES;
};

__device__ __forceinline__ void p1_cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void p1_cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void p1_cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void p1_cp_async8(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

// Whether a tile can take the staged form, and the chunk sample s00 of its
// (input row 0, column 0) at its delay: a full tile of one delay run (lane i
// of every warp holds the delay of output row i), no window tap, rows of a
// multiple of 16 bytes in a 16-byte aligned stream, every window inside the
// chunk, and the last 16-byte copy ending inside the stream's chunk bytes.
template <int T, int N1, int W>
__device__ __forceinline__ bool p1_stage_plan(const Phase1Params &p, const uint8_t *chunk, int cdl, int Rv,
                                              long long rel_base, unsigned long long &s00) {
    using S = P1Shape<T, N1, W>;
    const int N = p.N, N2 = p.N2;
    const unsigned RB = (unsigned)N / 4u * 5u;
    const long long H = p.H, HL = p.H + p.L;
    const int lane = threadIdx.x & 31;
    const int cd = __shfl_sync(0xffffffffu, cdl, 0);
    const bool one_run = __all_sync(0xffffffffu, lane >= Rv || cdl == cd);
    const long long rel0 = rel_base - cd;
    const long long hi = rel0 + (long long)N * (S::ROWS - 1) + (long long)N2 * (N1 - 1) + W;
    s00 = (unsigned long long)(rel0 - H);
    if (!(one_run && Rv == S::R && !p.window_tap && (RB & 15u) == 0u && ((uintptr_t)chunk & 15u) == 0u &&
          rel0 >= H && hi <= HL))
        return false;
    const long long sl = rel0 - H + (long long)N2 * (N1 - 1) + (long long)N * (S::ROWS - 1);
    const long long al = ((sl >> 2) * 5 + ((sl & 3) * 5 >> 2)) & ~15LL;
    return al + S::SEG <= p.chunk_bytes;
}

// First byte of segment j (columns N2 j + t2_0 ...) in input row 0 of a staged
// tile, rounded down to 16; row i starts RB i bytes further (RB a multiple of 16).
__device__ __forceinline__ unsigned long long p1_seg_start(unsigned long long s00, int N2, int j) {
    const unsigned long long s = s00 + (unsigned long long)N2 * j;
    return ((s >> 2) * 5ull + ((s & 3ull) * 5ull >> 2)) & ~15ull;
}

// Copy group g (input rows g SG .. g SG + SG - 1) of a staged tile into its
// ring slots and commit it (an empty group past the last row, so that the
// group after g is always the newest when g is waited for).
template <int T, int N1, int W>
__device__ __forceinline__ void p1_stage_group(uint8_t *stg, const uint8_t *chunk, unsigned long long s00, int N2,
                                               unsigned RB, int g) {
    using S = P1Shape<T, N1, W>;
    constexpr int SEG = S::SEG, SG = S::SG, RING = S::RING, NR = S::ROWS;
    constexpr int CPR = N1 * (SEG / 16);                      // 16-byte copies per input row
    constexpr int PER = (SG * CPR + kP1Threads - 1) / kP1Threads;
#pragma unroll
    for (int k = 0; k < PER; k++) {
        const int e = threadIdx.x + k * kP1Threads;
        const int row = g * SG + e / CPR, j = (e % CPR) / (SEG / 16), c16 = e % (SEG / 16);
        if (e < SG * CPR && row < NR)
            p1_cp_async16(stg + ((row % RING) * N1 + j) * SEG + 16 * c16,
                          chunk + p1_seg_start(s00, N2, j) + (unsigned long long)RB * row + 16 * c16);
    }
    p1_cp_async_commit();
}

// Output rows (r, r + 1) of a column pair from the ring win of T + 1 input
// rows (win[i % (T + 1)] holds input row i), r even, row r + T the newest in
// the ring: packed FP32x2 FMAs in four independent chains (each output row's
// taps in two halves, added at the end).
template <int T, class S>
__device__ __forceinline__ void p1_fir_pair(int r, const float2 (&win)[T + 1], const float2 (&w2)[T], float *ga,
                                            float *gb) {
    constexpr int TH = T >= 4 ? T / 2 : T;
    float2 a0 = make_float2(0.0f, 0.0f), a1 = make_float2(0.0f, 0.0f);
    float2 b0 = make_float2(0.0f, 0.0f), b1 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < TH; j++) {
        a0 = __ffma2_rn(w2[j], win[(r + j) % (T + 1)], a0);
        a1 = __ffma2_rn(w2[j], win[(r + 1 + j) % (T + 1)], a1);
    }
#pragma unroll
    for (int j = TH; j < T; j++) {
        b0 = __ffma2_rn(w2[j], win[(r + j) % (T + 1)], b0);
        b1 = __ffma2_rn(w2[j], win[(r + 1 + j) % (T + 1)], b1);
    }
    if constexpr (TH < T) {
        a0 = __fadd2_rn(a0, b0);
        a1 = __fadd2_rn(a1, b1);
    }
    ga[r * S::ROW] = a0.x;
    gb[r * S::ROW] = a0.y;
    ga[(r + 1) * S::ROW] = a1.x;
    gb[(r + 1) * S::ROW] = a1.y;
}

// Exact float of the 10-bit two's-complement field in the low bits of x:
// (field ^ 512) is the offset-binary value in [0, 1024), placed in the
// mantissa of 2^23 and the bias 2^23 + 512 subtracted (both steps exact).
__device__ __forceinline__ float field10_to_float(unsigned x) {
    return __uint_as_float(((x & 0x3FFu) ^ 0x200u) | 0x4B000000u) - 8389120.0f;
}

// The sample whose field starts in byte b[0] at bit offset sh from the top
// (sh = 2 (s mod 4)): the two bytes as a big-endian 16-bit word, shifted down
// by 6 - sh.
__device__ __forceinline__ float sample10(const uint8_t *b, unsigned sh) {
    const unsigned v = __byte_perm((unsigned)__ldg(b), (unsigned)__ldg(b + 1), 0x0004u);   // b[0] << 8 | b[1]
    return field10_to_float(v >> (6u - sh));
}

// Sample at relative index s (from the first history sample), or 0 past the
// received samples.
__device__ __forceinline__ float sample10_at(const uint8_t *hist, const uint8_t *chunk, unsigned s, unsigned H,
                                             unsigned HL) {
    if (s >= HL) return 0.0f;
    const bool h = s < H;
    const unsigned u = h ? s : s - H;
    return sample10((h ? hist : chunk) + (u >> 2) * 5u + ((u & 3u) * 5u >> 2), 2u * (s & 3u));
}

// General case of the FIR: a run of output rows [ra, rb) of a tile that
// touches the history or has several delay runs; samples checked one by one
// (history / chunk / past the received samples), one row of loads at a time.
// The window tap of output row r is its first input row, i = r. Kept out of
// line so that its registers do not weigh on the common path.
template <int T, class S>
__device__ __noinline__ void p1_fir_general(const Phase1Params &p, const uint8_t *hist, const uint8_t *chunk,
                                            unsigned H, unsigned HL, unsigned s0a, unsigned s0b, int ra, int rb,
                                            float *ga, float *gb, int stream, int q0, int t2_0, int ta, int tb) {
    const int N = p.N;
    float2 w2[T];
#pragma unroll
    for (int j = 0; j < T; j++)
        w2[j] = make_float2(__ldg(p.w + t2_0 + ta + (long long)N * j), __ldg(p.w + t2_0 + tb + (long long)N * j));
    unsigned dep = 0u;
    float2 win[T];
#pragma unroll 1
    for (int row = ra; row < rb + T - 1; row++) {
        const float xa = sample10_at(hist, chunk, s0a + (unsigned)(row * N) + dep, H, HL);
        const float xb = sample10_at(hist, chunk, s0b + (unsigned)(row * N) + dep, H, HL);
        asm volatile("" : "+r"(dep) : "f"(xa), "f"(xb));
        // shift the window: win[j] holds input row (row - T + 1 + j)
#pragma unroll
        for (int j = 0; j < T - 1; j++) win[j] = win[j + 1];
        win[T - 1] = make_float2(xa, xb);
        if (p.window_tap && row < rb) {
            int *tap = p.window_tap + ((long long)stream * p.M + q0 + row) * N + t2_0;
            tap[ta] = (int)xa;
            tap[tb] = (int)xb;
        }
        const int r = row - (T - 1);
        if (r >= ra) {
            // the taps' two halves in separate chains, added at the end: the
            // summation order of p1_fir_pair, so that a window gives the same
            // bits whichever path filters it
            constexpr int TH = T >= 4 ? T / 2 : T;
            float2 a = make_float2(0.0f, 0.0f), b = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int j = 0; j < TH; j++) a = __ffma2_rn(w2[j], win[j], a);
#pragma unroll
            for (int j = TH; j < T; j++) b = __ffma2_rn(w2[j], win[j], b);
            if constexpr (TH < T) a = __fadd2_rn(a, b);
            ga[r * S::ROW] = a.x;
            gb[r * S::ROW] = a.y;
        }
    }
}

// One tile per CTA: (t2 block, spectrum block, stream) = (blockIdx.x, .y, .z).
template <int T, int N1, int W, bool HALF>
__global__ void __launch_bounds__(kP1Threads, 2) k_phase1(const Phase1Params p) {
    using S = P1Shape<T, N1, W>;
    constexpr int R = S::R, H1 = N1 / 2;
    extern __shared__ __align__(16) float gs[];   // [R][N1][GW] FIR output g, then the staged-input ring
    __shared__ int c_sm[R];
    __shared__ __align__(16) float2 tw1_sm[(H1 + 1) * W];   // exp(-2 pi i k1 t2 / N) for this tile's t2

    const int N = p.N, N2 = p.N2;
    const int stream = blockIdx.z;
    const int t2_0 = blockIdx.x * W;
    const int q0 = p.q_begin + blockIdx.y * R;
    const int Rv = min(R, p.q_begin + p.q_count - q0);
    const int lane = threadIdx.x & 31;
    const int cdl = lane < Rv ? __ldg(p.ctab + (long long)stream * p.M + q0 + lane) : 0;
#include "k_phase1_tile.inc"
}

// The tiles of several plans' launches (same T, N1, W) in one grid: the
// member's parameters are staged in shared memory, its block decomposed into
// the (t2 block, spectrum block, stream) of its own launch.
template <int T, int N1, int W, bool HALF>
__global__ void __launch_bounds__(kP1Threads, 2) k_phase1_group(const Phase1Group g) {
    using S = P1Shape<T, N1, W>;
    constexpr int R = S::R, H1 = N1 / 2;
    extern __shared__ __align__(16) float gs[];   // [R][N1][GW] FIR output g, then the staged-input ring
    __shared__ int c_sm[R];
    __shared__ __align__(16) float2 tw1_sm[(H1 + 1) * W];   // exp(-2 pi i k1 t2 / N) for this tile's t2
    __shared__ Phase1Params sp;
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
    const Phase1Params &p = sp;
    const int N = p.N, N2 = p.N2;
    const int stream = sxyz[2];
    const int t2_0 = sxyz[0] * W;
    const int q0 = p.q_begin + sxyz[1] * R;
    const int Rv = min(R, p.q_begin + p.q_count - q0);
    const int lane = threadIdx.x & 31;
    const int cdl = lane < Rv ? p.ctab[(long long)stream * p.M + q0 + lane] : 0;
#include "k_phase1_tile.inc"
}

template <int T, int N1, int W>
cudaError_t launch_phase1_tw_group(const Phase1Group &g, cudaStream_t s) {
    using S = P1Shape<T, N1, W>;
    const size_t smem = S::SMEM;
    cudaError_t e =
        cudaFuncSetAttribute(k_phase1_group<T, N1, W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (g.n < 1 || g.start[g.n] < 1) return cudaSuccess;
    k_phase1_group<T, N1, W, false><<<g.start[g.n], kP1Threads, smem, s>>>(g);
    return cudaGetLastError();
}

template <int T, int N1, int W, bool HALF = false>
cudaError_t launch_phase1_tw(const Phase1Params &p, int n_streams, cudaStream_t s) {
    using S = P1Shape<T, N1, W>;
    if (p.W != W || p.N2 % W) return cudaErrorInvalidValue;
    const size_t smem = S::SMEM;
    cudaError_t e =
        cudaFuncSetAttribute(k_phase1<T, N1, W, HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(p.N2 / W, (p.q_count + kP1Rows - 1) / kP1Rows, n_streams);
    k_phase1<T, N1, W, HALF><<<grid, kP1Threads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int T>
cudaError_t launch_phase1_group_n1(int N1, const Phase1Group &g, cudaStream_t s) {
    switch (N1 * 1000 + g.p[0].W) {
        case 8064: return launch_phase1_tw_group<T, 8, 64>(g, s);
        case 16032: return launch_phase1_tw_group<T, 16, 32>(g, s);
        case 32016: return launch_phase1_tw_group<T, 32, 16>(g, s);
        case 64008: return launch_phase1_tw_group<T, 64, 8>(g, s);
        case 8032: return launch_phase1_tw_group<T, 8, 32>(g, s);
        case 8016: return launch_phase1_tw_group<T, 8, 16>(g, s);
        case 8008: return launch_phase1_tw_group<T, 8, 8>(g, s);
        case 8004: return launch_phase1_tw_group<T, 8, 4>(g, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int T>
cudaError_t launch_phase1_n1(int N1, const Phase1Params &p, int n_streams, cudaStream_t s) {
    if (p.half_out) return cudaErrorInvalidValue;   // FP16 output: unused by the FP32 form
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
