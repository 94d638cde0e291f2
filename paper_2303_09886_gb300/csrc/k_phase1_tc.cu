// Phase 1 of the reduced-precision forms on the 5th-generation tensor cores
// (tcgen05): 10-bit unpack, coarse delay, PFB FIR (Eq. 1) and the first
// stage of the four-step real DFT as ONE contraction per FIR column,
// accumulated in tensor memory.
//
// Split of the N-point DFT (N = 2n): physical FIR column t in [0, P), P = N/8,
// and radix-8 digit t1: the sample offset of a spectrum is t_full = P t1 + t.
// With u = 8 m + r, r = t1 + 8 jj (jj the tap), Eq. 1's samples of spectrum m
// at column t are x_t[8 m + r] where x_t[u] = s[t0(0) - c + t + P u]: for one
// column, consecutive spectra advance by 8 along one sequence (a Hankel
// matrix with rows 8 apart). The first DFT stage has radix N1 = 8 R: the R
// physical columns t = t2 + N2 j (j < R, N2 = N / N1) form output column t2,
//   Z[k1][t2] = sum_j sum_r B_t[k1][r] x_t[8 m + r],
//   B_t[k1][r] = w[t + P r] exp(-2 pi i k1 (P (r mod 8) + t) / N),
// which is the first stage of the split t = N2 t1' + t2, k = k1 + N1 k2
// (t1' = R (r mod 8) + j) with its twiddle exp(-2 pi i k1 t2 / N) folded into
// B; k1 in [0, N1/2] since g is real.
//
// On the tensor core, per pass of 128 consecutive spectra of one stream:
//  - A (M = 128 spectra, K = 8 T): the decoded sequence x_t in shared memory
//    as 16-bit values; row m starts 16 bytes after row m - 1, so one K-major
//    no-swizzle matrix descriptor with leading-byte offset 16 and stride-byte
//    offset 128 describes the Hankel matrix without copying a sample twice;
//  - B (N = NM >= 2 (N1/2 + 1) rows (Re, Im of each k1), K = 8 T): the
//    column's weight x DFT x twiddle block, resident for the CTA's columns,
//    scaled by a power of two per output column (per-block scaling);
//  - D (128 lanes x NM columns, FP32) in tensor memory; the R columns of one
//    output column accumulate into the same D.
// FP16 form: 10-bit integers are exact in FP16. BF16 form: a sample is split
// into hi + lo BF16 parts (both exact), two MMAs per K step.
//
// The packed stream is first unpacked into FP16 column sequences
// (k_unpack_cols: coalesced reads of the packed rows, one transpose through
// shared memory), so that a CTA reads each of its columns contiguously. A
// CTA owns 8 physical columns (CW = 8 / R output columns) and a range of
// (stream, 128-spectrum tile) items; each tile is one pass per run of equal
// coarse delay. Warp roles overlap the passes: fill warps copy pass p + 1's
// column sequences into shared memory while the MMA warp runs pass p on the
// tensor core and the epilogue warps drain pass p - 1 from the other half of
// tensor memory (tcgen05.ld), scale it and store the second-stage input
// [stream][spectrum][k1][t2] (FP16 pairs, or FP32 pairs in the BF16 form).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <vector>

#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kTcRows = 128;     // spectra per pass: the MMA's M

__host__ __device__ constexpr int tc_tp(int T) { return T < 2 ? 2 : T; }                 // K = 8 T' >= 16
__host__ __device__ constexpr int tc_xl(int T) { return 8 * (kTcRows - 1 + tc_tp(T)); } // samples per column
// k1 values of one of ks slices of [0, 4 R], and the operand rows (Re, Im) they take, padded to 16
__host__ __device__ constexpr int tc_kps(int R, int ks) { return (4 * R + 1 + ks - 1) / ks; }
__host__ __device__ constexpr int tc_nm(int R, int ks) { return 16 * ((2 * tc_kps(R, ks) + 15) / 16); }
constexpr long long kTcSmemMax = 227 * 1024;

// Shared-memory bytes with ph physical columns per CTA, ks k1-slices and nxb
// data buffers: the operand blocks (BF16: hi and lo planes) and the data
// (BF16: hi and lo).
__host__ __device__ constexpr long long tc_smem_ph(int ph, int R, int T, int prec, int ks, int nxb) {
    return 2LL * ((prec == 2 ? 2 : 1) * ph * (long long)tc_nm(R, ks) * 8 * tc_tp(T) +
                  (long long)nxb * (prec == 2 ? 2 : 1) * ph * tc_xl(T)) +
           4 * kTcRows + 64 + 2048 + 256;
}
// Physical FIR columns per CTA: 16 where the FP16 form's operands of R <= 2
// fit with two data buffers (the epilogue then stores 8 consecutive FP16
// pairs = one whole 32-byte sector per (spectrum, k1), whatever the other
// CTAs do), else 8 (one CTA per SM with 16, two with 8).
__host__ __device__ constexpr int tc_phys(int R, int T, int prec) {
    return (prec == 1 && R <= 2 && tc_smem_ph(16, R, T, prec, 1, 2) <= kTcSmemMax) ? 16 : 8;
}
__host__ __device__ constexpr long long tc_smem(int ph, int R, int T, int prec, int ks, int nxb) {
    return tc_smem_ph(ph, R, T, prec, ks, nxb);
}
// fewest k1-slices, then two decode buffers (the decode of the next pass
// under the current one's MMAs), that fit in shared memory; 0 if none does
__host__ __device__ constexpr int tc_ks(int ph, int R, int T, int prec) {
    return tc_smem(ph, R, T, prec, 1, 1) <= kTcSmemMax   ? 1
           : tc_smem(ph, R, T, prec, 2, 1) <= kTcSmemMax ? 2
           : tc_smem(ph, R, T, prec, 4, 1) <= kTcSmemMax ? 4
           : tc_smem(ph, R, T, prec, 8, 1) <= kTcSmemMax ? 8
                                                          : 0;
}
__host__ __device__ constexpr int tc_ks1(int ph, int R, int T, int prec) {
    return tc_ks(ph, R, T, prec) > 0 ? tc_ks(ph, R, T, prec) : 1;
}
__host__ __device__ constexpr int tc_nxb(int ph, int R, int T, int prec) {
    return tc_smem(ph, R, T, prec, tc_ks1(ph, R, T, prec), 2) <= kTcSmemMax ? 2 : 1;
}
// tensor-memory columns: two pass buffers of CW x NM, a power of two >= 32
__host__ __device__ constexpr int tc_tmem_cols(int ph, int R, int T, int prec) {
    return 2 * (ph / R) * tc_nm(R, tc_ks1(ph, R, T, prec)) <= 256 ? 256 : 512;
}

// One CTA per SM when the CTA's shared memory leaves no room for a second
// (and always at PH = 16), else two. Warps: 4 epilogue (one per 32
// tensor-memory lanes), F fill, 1 MMA; four fill warps at one CTA per SM,
// two at two CTAs per SM (which leaves each thread 128 registers).
constexpr long long kTcTwoCtaSmem = 113 * 1024;
__host__ __device__ constexpr bool tc_one_cta(int ph, int R, int T, int prec) {
    return ph == 16 || tc_smem(ph, R, T, prec, tc_ks1(ph, R, T, prec), tc_nxb(ph, R, T, prec)) > kTcTwoCtaSmem;
}
__host__ __device__ constexpr int tc_fill_warps(bool one) { return one ? 4 : 2; }
__host__ __device__ constexpr int tc_threads(bool one) { return 32 * (5 + tc_fill_warps(one)); }

// ---- tcgen05 / mbarrier primitives (PTX ISA, sm_100a family) ----

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading- and stride-byte
// offsets (16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B both FP16
// (bf16 = 0) or both BF16 (bf16 = 1), K-major, M x N.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N, int bf16) {
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16_ss(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// try_wait with a suspend-time hint: the thread sleeps (up to about 20 us)
// until the phase completes instead of spinning on issue slots
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, "
        "p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
                 : "r"(taddr));
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
    v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3);
    v[4] = __uint_as_float(r4);
    v[5] = __uint_as_float(r5);
    v[6] = __uint_as_float(r6);
    v[7] = __uint_as_float(r7);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- 10-bit samples ----

// FP16 of a 10-bit two's-complement field f: the FP16 with exponent 2^10 and
// mantissa (f ^ 512) is 1024 + (v + 512); subtracting 1536 (exact) gives v.
__device__ __forceinline__ uint16_t field_to_half(uint32_t f) {
    const __half h = __hsub(__ushort_as_half((unsigned short)(((f ^ 0x200u) | 0x6400u) & 0xFFFFu)),
                            __ushort_as_half(0x6600u));
    return __half_as_ushort(h);
}

// Two fields as an FP16 pair (f0 in the low half).
__device__ __forceinline__ uint32_t fields_to_half2(uint32_t f0, uint32_t f1) {
    const uint32_t h = (((f0 ^ 0x200u) | 0x6400u) & 0xFFFFu) | ((((f1 ^ 0x200u) | 0x6400u) & 0xFFFFu) << 16);
    const __half2 r = __hsub2(*reinterpret_cast<const __half2 *>(&h),
                              __halves2half2(__ushort_as_half(0x6600u), __ushort_as_half(0x6600u)));
    return *reinterpret_cast<const uint32_t *>(&r);
}

// BF16 hi and lo parts of two integer samples held as an FP16 pair: hi =
// RN(v), lo = v - hi, both exact (|v| <= 512).
__device__ __forceinline__ void half2_to_bf16x2(uint32_t h2, uint32_t &hi, uint32_t &lo) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&h2));
    const __nv_bfloat16 h0 = __float2bfloat16_rn(f.x), h1 = __float2bfloat16_rn(f.y);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(f.x - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(f.y - __bfloat162float(h1));
    hi = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
}

__device__ __forceinline__ long long floor_div(long long a, long long b) {
    const long long q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

// ---- pass enumeration (one warp at a time, every role the same sequence) ----
//
// A pass is a run of consecutive spectra [ra, rb) of one (stream, 128-spectrum
// tile) item with one coarse delay c (Eq. 1's window start moves with c). A
// warp keeps the delay-change flags of the current item as a 128-bit ballot
// mask and loads the next item's flags, row-0 delay and its stream's first
// delay c0 one item ahead, so that no load latency sits between passes.
struct Pass {
    int st, q0, ra, rb, c, c0;
};

struct PassIter {
    int it, it_end, ra, rows, st, q0, c_row0, c0;
    unsigned m[4];            // bit l of m[k]: the delay changes at row 32 k + l
    unsigned char f[4];       // prefetched flags of rows 32 k + lane of the next item
    int pc_row0, pc0;         // prefetched delays of the next item
};

__device__ __forceinline__ void pass_prefetch(PassIter &s, const Phase1TcParams &p, int n_tiles, int item) {
    const int lane = threadIdx.x & 31;
    if (item >= s.it_end) return;
    const int st = item / n_tiles, q0 = p.q_begin + (item % n_tiles) * kTcRows;
    const int rows = min(kTcRows, p.q_begin + p.q_count - q0);
    const unsigned char *cf = p.cchg + (long long)st * p.M + q0;
#pragma unroll
    for (int k = 0; k < 4; k++) s.f[k] = (32 * k + lane < rows) ? __ldg(cf + 32 * k + lane) : (unsigned char)0;
    s.pc_row0 = __ldg(p.ctab + (long long)st * p.M + q0);
    s.pc0 = __ldg(p.ctab + (long long)st * p.M);
}

__device__ __forceinline__ bool warp_next_pass(PassIter &s, Pass &ps, const Phase1TcParams &p, int n_tiles) {
    for (;;) {
        if (s.ra < 0) {
            if (s.it >= s.it_end) return false;
            s.st = s.it / n_tiles;
            s.q0 = p.q_begin + (s.it % n_tiles) * kTcRows;
            s.rows = min(kTcRows, p.q_begin + p.q_count - s.q0);
#pragma unroll
            for (int k = 0; k < 4; k++) s.m[k] = __ballot_sync(0xFFFFFFFFu, s.f[k] != 0);
            s.c_row0 = s.pc_row0;
            s.c0 = s.pc0;
            s.ra = 0;
            pass_prefetch(s, p, n_tiles, s.it + 1);
        }
        if (s.ra >= s.rows) {
            s.ra = -1;
            s.it++;
            continue;
        }
        // first change after ra
        int rb = s.rows;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int lo = s.ra + 1 - 32 * k;   // rows >= ra + 1 in this word
            unsigned mk = s.m[k];
            if (lo >= 32) mk = 0u;
            else if (lo > 0) mk &= ~0u << lo;
            if (mk && rb == s.rows) rb = 32 * k + __ffs(mk) - 1;
        }
        if (rb > s.rows) rb = s.rows;
        const int c = s.ra == 0 ? s.c_row0 : __ldg(p.ctab + (long long)s.st * p.M + s.q0 + s.ra);
        ps = Pass{s.st, s.q0, s.ra, rb, c, s.c0};
        s.ra = rb;
        return true;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Unpack into FP16 columns, pre-delayed by each stream's first coarse delay
// c0 = ctab[stream][0]: cols[st][col][r] holds the sample at timestamp
// (rb + r) P + col - c0 (zero before the history and past the chunk), so that
// for every pass with coarse delay c0 a FIR column's sequence x_t[u] starts
// at a row that is a multiple of 8 (16-byte aligned) and is read as one
// contiguous block. Tile: 64 rows x 64 columns per CTA: the packed rows are
// read as aligned 32-bit words straight from global memory (five per
// 8-sample run of a row; neighbouring threads share words through L1), a
// thread converts 8 samples of two rows into FP16 pairs, and the tile goes
// through shared memory once to be written out column by column.
__global__ void __launch_bounds__(256) k_unpack_cols(const UnpackColsParams p) {
    __shared__ uint32_t tile[64][33];    // [column][row pair] FP16 pairs
    const int col0 = blockIdx.x * 64, r0 = p.row_begin + blockIdx.y * 64, st = blockIdx.z;
    const int tid = threadIdx.x;
    const long long c0 = p.ctab[(long long)st * p.M];
    // relative sample (from the first history sample) of row 0, column col0;
    // history and chunk are one bit stream (10 H is a multiple of 32)
    const long long rel00 = (p.rb + r0) * (long long)p.P + col0 - c0 - (p.t_in - p.H);
    const long long bit00 = 10 * rel00;
    const int off = (int)(bit00 & 31);   // the same for every row (10 P is a multiple of 32)
    const uint32_t *hw = reinterpret_cast<const uint32_t *>(p.hist + (long long)st * p.hist_bytes);
    const uint32_t *cw = reinterpret_cast<const uint32_t *>(p.chunk + (long long)st * p.chunk_bytes);
    const long long hwords = 10 * p.H / 32, cwords = p.chunk_bytes / 4;
    {
        // thread: rows 2 rp, 2 rp + 1, samples 8 g .. 8 g + 7 (bits off + 80 g .. + 80)
        const int rp = tid >> 3, g = tid & 7;
        const int b0 = off + 80 * g, wi = b0 >> 5, sh = b0 & 31;
        uint32_t f[2][8];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int row = 2 * rp + h;
            const long long wrow = ((bit00 + (long long)row * 10 * p.P) >> 5) + wi;
            const bool live = r0 + row < p.RT;
            uint32_t raw[5];
#pragma unroll
            for (int i = 0; i < 5; i++) {
                const long long w = wrow + i;
                uint32_t v = 0u;
                if (live && w >= 0) {
                    if (w < hwords) v = __ldg(hw + w);
                    else if (w - hwords < cwords) v = __ldg(cw + (w - hwords));
                }
                raw[i] = __byte_perm(v, 0u, 0x0123u);   // big-endian bits
            }
            uint32_t a[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = __funnelshift_l(raw[i + 1], raw[i], (unsigned)sh);
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int bb = 10 * k;
                f[h][k] = __funnelshift_l(a[(bb >> 5) + 1], a[bb >> 5], (unsigned)(bb & 31)) >> 22;
            }
            // samples before the first history sample, or rows past the data, are zero
            const long long rel = rel00 + (long long)row * p.P + 8 * g;
            if (!live || rel + 7 < 0) {
#pragma unroll
                for (int k = 0; k < 8; k++) f[h][k] = 0u;
            } else if (rel < 0) {
#pragma unroll
                for (int k = 0; k < 8; k++)
                    if (rel + k < 0) f[h][k] = 0u;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; k++) tile[8 * g + k][rp] = fields_to_half2(f[0][k], f[1][k]);
    }
    __syncthreads();
    {
        // column c: row pairs 0 .. 31 (128 contiguous bytes), 4 threads of 32 bytes
        const int c = tid >> 2, part = tid & 3;
        uint4 *dst = reinterpret_cast<uint4 *>(p.cols + ((long long)st * p.P + col0 + c) * p.RTP + r0 + 16 * part);
        const uint32_t *t = &tile[c][8 * part];
        if (p.bf16) {
            // the BF16 form's data planes: x = hi + lo exactly
            uint32_t h[8], l[8];
#pragma unroll
            for (int i = 0; i < 8; i++) half2_to_bf16x2(t[i], h[i], l[i]);
            uint4 *dlo = reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(dst) + p.plane_elems);
            dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
            dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
            dlo[0] = make_uint4(l[0], l[1], l[2], l[3]);
            dlo[1] = make_uint4(l[4], l[5], l[6], l[7]);
        } else {
            dst[0] = make_uint4(t[0], t[1], t[2], t[3]);
            dst[1] = make_uint4(t[4], t[5], t[6], t[7]);
        }
    }
}

// The same for P < 64 (n_channels < 256): one thread per output sample,
// read as two bytes of the packed stream.
__global__ void k_unpack_cols_small(const UnpackColsParams p) {
    const long long total = (long long)p.n_streams * p.P * p.RTP;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % p.RTP);
        const long long sc = e / p.RTP;
        const int col = (int)(sc % p.P), st = (int)(sc / p.P);
        const long long rel = (p.rb + r) * (long long)p.P + col - p.ctab[(long long)st * p.M] - (p.t_in - p.H);
        uint16_t v = 0;
        if (r < p.RT && rel >= 0 && rel < p.H + p.L) {
            const bool h = rel < p.H;
            const long long u = h ? rel : rel - p.H;
            const uint8_t *b = (h ? p.hist + (long long)st * p.hist_bytes : p.chunk + (long long)st * p.chunk_bytes) +
                               ((5 * u) >> 2);
            const unsigned w = ((unsigned)__ldg(b) << 8) | (unsigned)__ldg(b + 1);
            v = field_to_half((w >> (6u - 2u * (unsigned)(u & 3))) & 0x3FFu);
        }
        if (p.bf16) {
            uint32_t hi, lo;
            half2_to_bf16x2((uint32_t)v, hi, lo);
            p.cols[e] = (uint16_t)(hi & 0xFFFFu);
            p.cols[e + p.plane_elems] = (uint16_t)(lo & 0xFFFFu);
        } else {
            p.cols[e] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// The tensor-core kernel, warp-specialised:
//   warps 0-3    epilogue: tensor memory -> scale -> second-stage input in HBM
//   next F warps fill: the pass's PH column sequences from cols into the ring
//                of shared-memory data buffers (BF16: hi and lo planes); F = 4
//                at one CTA per SM, 2 at two CTAs per SM
//   last warp    MMA: the tcgen05 chain of a pass into one of two tensor-memory
//                buffers, committed to the barriers that free its data buffer
//                and hand the accumulator to the epilogue
// Each role walks the same pass sequence; they synchronise only through
// mbarriers (xfull / xempty per data buffer, tfull / tempty per tensor-memory
// buffer), every wait bounded.
template <int R, int T, int PREC, int PH>   // PH: physical FIR columns of the CTA
__global__ void __launch_bounds__(tc_threads(tc_one_cta(PH, R, T, PREC)), tc_one_cta(PH, R, T, PREC) ? 1 : 2)
    k_phase1_tc(const Phase1TcParams p) {
    constexpr int KS = tc_ks(PH, R, T, PREC), KPS = tc_kps(R, KS);   // k1-slices, k1 values per slice
    constexpr int TMEMC = tc_tmem_cols(PH, R, T, PREC);               // tensor-memory columns allocated
    constexpr int NM = tc_nm(R, KS), TP = tc_tp(T), K = 8 * TP, XL = tc_xl(T), CW = PH / R;
    constexpr int NPL = PREC == 2 ? 2 : 1;    // data planes: BF16 hi + lo
    constexpr int NPB = PREC == 2 ? 2 : 1;    // operand planes: BF16 hi + lo
    constexpr int H1 = 4 * R;                 // k1 in [0, H1]
    constexpr int BBLK = NM * K;              // 16-bit elements per operand block
    constexpr int TMC = CW * NM;              // tensor-memory columns per pass buffer
    constexpr int NG = (2 * KPS + 7) / 8;     // 8-column groups holding (Re, Im) of the slice's k1
    constexpr int NXB = tc_nxb(PH, R, T, PREC);   // data buffers
    constexpr bool ONE = tc_one_cta(PH, R, T, PREC);                   // one CTA per SM
    constexpr int NTH = tc_threads(ONE), FT = 32 * tc_fill_warps(ONE);  // threads, fill threads
    constexpr int WMMA = 4 + tc_fill_warps(ONE);                        // the MMA warp
    static_assert(KS > 0, "shape does not fit in shared memory");
    static_assert(2 * TMC <= TMEMC, "tensor memory");
    extern __shared__ __align__(1024) uint8_t smem[];
    uint16_t *bsm = reinterpret_cast<uint16_t *>(smem);            // [NPB][PH][BBLK]
    uint16_t *xsm = bsm + NPB * PH * BBLK;                    // [NXB][NPL][PH][XL]
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(xsm + NXB * NPL * PH * XL);
    unsigned long long *xfull = bar, *xempty = bar + 2, *tfull = bar + 4, *tempty = bar + 6;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 8);
    volatile int *abort_sm = reinterpret_cast<volatile int *>(tmem_slot + 1);
    long long *fsrc = reinterpret_cast<long long *>(bar + 9);          // [NXB][PH] column source offsets
    int *fsh = reinterpret_cast<int *>(fsrc + 2 * PH);            // [NXB][PH] row0 mod 8

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tiles = (p.q_count + kTcRows - 1) / kTcRows;
    const int n_items = p.n_streams * n_tiles;
    const int P = p.N / 8, N2 = p.N2;
    // Work units: (column group, k1-slice, item), item fastest; CTA b takes a
    // contiguous range of equal length (persistent: one wave of CTAs), which
    // spans few (column group, slice) segments, each loading its operand blocks.
    const long long n_units = (long long)(N2 / CW) * KS * n_items;
    const long long u_begin = n_units * blockIdx.x / gridDim.x, u_end = n_units * (blockIdx.x + 1) / gridDim.x;
    if (tid == 0) {
        for (int i = 0; i < 2; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&xfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&xempty[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&tfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&tempty[i])), "r"(128));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_sm = 0;
    }
    if (warp == WMMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(TMEMC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // a bounded wait that also gives up once another role has
    auto wait_bar = [&](unsigned long long *b, uint32_t parity) -> bool {
        const uint32_t a = smem_addr(b);
        const long long t0 = clock64();
        while (!mbar_try(a, parity)) {
            if (*abort_sm) return false;
            if (clock64() - t0 > 2000000000LL) {
                *abort_sm = 1;
                atomicExch(p.err, 2);
                return false;
            }
        }
        return true;
    };
    auto arrive = [&](unsigned long long *b) {
        asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(b))
                     : "memory");
    };
    // pass counters of the roles: the barriers' phases run on across segments
    int pc_fill = 0, pc_mma = 0, pc_epi = 0;
    for (long long u = u_begin; u < u_end;) {
    const long long cgs = u / n_items;   // (column group, slice) of this segment
    const int it_begin = (int)(u - cgs * n_items);
    const int it_end = (int)(u_end - cgs * n_items < n_items ? u_end - cgs * n_items : n_items);
    u = cgs * n_items + it_end;
    const int cg = (int)(cgs / KS), slice = (int)(cgs % KS);
    const int k1_lo = slice * KPS, k1_hi = min(H1 + 1, k1_lo + KPS);
    // the segment's operand blocks (weights x DFT x twiddle); the previous
    // segment's MMAs have completed (its last accumulator was drained)
    {
        const uint4 *src =
            reinterpret_cast<const uint4 *>(p.bmat) + ((long long)cg * KS + slice) * (NPB * PH * BBLK / 8);
        uint4 *dst = reinterpret_cast<uint4 *>(bsm);
        for (int i = tid; i < NPB * PH * BBLK / 8; i += NTH) dst[i] = __ldg(src + i);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the operand blocks, for the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (*abort_sm) break;
    // index in the pre-delayed columns (timestamp + c0) of row v = 0 of physical
    // column i (run j = i / CW, column c = i % CW)
    auto col_start = [&](const Pass &ps, int i) -> long long {
        return (long long)p.N * (p.m0 + ps.q0) - ps.c + ps.c0 + (long long)cg * CW + (i % CW) + (long long)N2 * (i / CW);
    };

    PassIter iter{};
    iter.it = it_begin;
    iter.it_end = it_end;
    iter.ra = -1;
    pass_prefetch(iter, p, n_tiles, it_begin);
    Pass ps;
    if (warp >= 4 && warp < WMMA) {
        // ---------------- fill ----------------
        // A column's sequence starts at element row0 of its FP16 column;
        // it is copied in 16-byte chunks from the aligned element
        // row0 - sh (sh = row0 mod 8), each output chunk taking 16 bytes at
        // byte offset 2 sh of two consecutive source chunks.
        const int ft = tid - 128;
        constexpr int CPC = XL / 8;                 // 16-byte chunks per column sequence
        for (int &pc = pc_fill; warp_next_pass(iter, ps, p, n_tiles); pc++) {
            const int s = pc % NXB, use = pc / NXB;
            // the decision to go on is the same in every fill thread (a thread
            // must not leave while the others wait at the named barrier)
            int ok = use == 0 || ft != 0 || wait_bar(&xempty[s], (use - 1) & 1);
            asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %1, 0;\n\tbar.red.and.pred q, 1, %2, q;\n\t"
                         "selp.s32 %0, 1, 0, q;\n\t}\n"
                         : "=r"(ok)
                         : "r"(ok), "n"(FT)
                         : "memory");
            if (!ok) break;
            uint16_t *xb = xsm + (size_t)s * NPL * PH * XL;
            if (!p.window_tap && ps.c == ps.c0) {
                // the pass's delay is the columns' c0: every column sequence starts at
                // row 8 (m0 + q0) - rb, 16-byte aligned, one bulk copy each (per plane)
                if (ft == 0) {
                    constexpr uint32_t bytes = (uint32_t)(NPL * PH * XL * 2);
                    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                                 ::"r"(smem_addr(&xfull[s])), "r"(bytes) : "memory");
                    const long long row0 = 8LL * (p.m0 + ps.q0) - p.rb;
#pragma unroll 1
                    for (int i = 0; i < NPL * PH; i++) {
                        const int ic = i % PH, pl = i / PH;
                        const long long t = (long long)cg * CW + (ic % CW) + (long long)N2 * (ic / CW);
                        const uint16_t *src = p.cols + pl * p.plane_elems + ((long long)ps.st * P + t) * p.RTP + row0;
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                            ::"r"(smem_addr(xb + (size_t)i * XL)), "l"(src), "r"((uint32_t)(XL * 2)),
                            "r"(smem_addr(&xfull[s]))
                            : "memory");
                    }
                }
                continue;
            }
            if (ft < PH) {
                const long long a0 = col_start(ps, ft);
                const long long ra = floor_div(a0, P);
                const long long col = a0 - ra * P, row0 = ra - p.rb;
                fsrc[s * PH + ft] = ((long long)ps.st * P + col) * p.RTP + (row0 & ~7LL);
                fsh[s * PH + ft] = (int)(row0 & 7);
            }
            asm volatile("bar.sync 1, %0;" ::"n"(FT) : "memory");
            // (BF16: both data planes, unpacked already split into hi and lo)
            for (int e0 = ft; e0 < NPL * PH * CPC; e0 += FT * 3) {
                uint4 a[3], b[3];
#pragma unroll
                for (int u = 0; u < 3; u++) {
                    const int e = e0 + FT * u;
                    if (e < NPL * PH * CPC) {
                        const int ip = e / CPC, j = e - ip * CPC, i = ip % PH;
                        const uint4 *src =
                            reinterpret_cast<const uint4 *>(p.cols + (ip / PH) * p.plane_elems + fsrc[s * PH + i]) + j;
                        a[u] = __ldg(src);
                        b[u] = __ldg(src + 1);
                    }
                }
#pragma unroll
                for (int u = 0; u < 3; u++) {
                    const int e = e0 + FT * u;
                    if (e < NPL * PH * CPC) {
                        const int ip = e / CPC, j = e - ip * CPC, i = ip % PH;
                        const int sh = fsh[s * PH + i];
                        const uint32_t w[8] = {a[u].x, a[u].y, a[u].z, a[u].w, b[u].x, b[u].y, b[u].z, b[u].w};
                        uint32_t o[4];
                        const uint32_t sel = (sh & 1) ? 0x5432u : 0x3210u;   // 2-byte shift for odd sh
                        switch (sh >> 1) {
                            case 0:
#pragma unroll
                                for (int m = 0; m < 4; m++) o[m] = __byte_perm(w[m], w[m + 1], sel);
                                break;
                            case 1:
#pragma unroll
                                for (int m = 0; m < 4; m++) o[m] = __byte_perm(w[m + 1], w[m + 2], sel);
                                break;
                            case 2:
#pragma unroll
                                for (int m = 0; m < 4; m++) o[m] = __byte_perm(w[m + 2], w[m + 3], sel);
                                break;
                            default:
#pragma unroll
                                for (int m = 0; m < 4; m++) o[m] = __byte_perm(w[m + 3], w[m + 4], sel);
                                break;
                        }
                        reinterpret_cast<uint4 *>(xb + (size_t)ip * XL)[j] = make_uint4(o[0], o[1], o[2], o[3]);
                    }
                }
            }
            if (p.window_tap) {
                // debug tap: the first FIR tap of spectrum q0 + v / 8 at offset P (v % 8) + t
                asm volatile("bar.sync 1, %0;" ::"n"(FT) : "memory");
                const uint16_t *xv = xsm + (size_t)s * NPL * PH * XL;
                for (int e = ft; e < PH * 8 * kTcRows; e += FT) {
                    const int i = e / (8 * kTcRows), vv = e - i * (8 * kTcRows), mrow = vv >> 3;
                    if (mrow < ps.ra || mrow >= ps.rb) continue;
                    float x;
                    if constexpr (PREC == 2) {
                        x = __bfloat162float(__ushort_as_bfloat16(xv[(size_t)i * XL + vv])) +
                            __bfloat162float(__ushort_as_bfloat16(xv[(size_t)(PH + i) * XL + vv]));
                    } else {
                        x = __half2float(__ushort_as_half(xv[(size_t)i * XL + vv]));
                    }
                    const long long t = (long long)cg * CW + (i % CW) + (long long)N2 * (i / CW);
                    p.window_tap[((long long)ps.st * p.M + ps.q0 + mrow) * p.N + (long long)P * (vv & 7) + t] = (int)x;
                }
            }
            // every fill thread's writes, then one arrival
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.sync 1, %0;" ::"n"(FT) : "memory");
            if (ft == 0) arrive(&xfull[s]);
        }
    } else if (warp == WMMA) {
        // ---------------- MMA ----------------
        constexpr uint32_t idesc = mma_idesc(kTcRows, NM, PREC == 2 ? 1 : 0);
        for (int &pc = pc_mma; warp_next_pass(iter, ps, p, n_tiles); pc++) {
            const int s = pc % NXB, b = pc & 1;
            bool ok = true;
            if (lane == 0) {
                ok = wait_bar(&xfull[s], (pc / NXB) & 1);
                ok = ok && (pc < 2 || wait_bar(&tempty[b], ((pc >> 1) - 1) & 1));
            }
            if (!__shfl_sync(0xFFFFFFFFu, (int)ok, 0)) break;   // the same decision in every lane
            tc_fence_after();
            if (lane == 0) {
                const uint32_t d0 = tmem + (uint32_t)(b * TMC);
                const uint32_t xa0 = smem_addr(xsm + (size_t)s * NPL * PH * XL), ba0 = smem_addr(bsm);
#pragma unroll 1
                for (int c = 0; c < CW; c++) {
#pragma unroll 1
                    for (int j = 0; j < R; j++) {
                        const int i = j * CW + c;
                        // FP16: x B. BF16: x_hi B_hi + x_lo B_hi + x_hi B_lo (x_lo B_lo
                        // is below 2^-9 / 512 of the result and left out)
#pragma unroll
                        for (int pp = 0; pp < (PREC == 2 ? 3 : 1); pp++) {
                            const int pl = pp == 1 ? 1 : 0, pb = pp == 2 ? 1 : 0;
                            const uint32_t xa = xa0 + (uint32_t)((pl * PH + i) * XL * 2);
                            const uint32_t ba = ba0 + (uint32_t)((pb * PH + i) * BBLK * 2);
#pragma unroll
                            for (int kk = 0; kk < K / 16; kk++) {
                                const uint64_t ad = mat_desc(xa + 32u * kk, 16u, 128u);
                                const uint64_t bd =
                                    mat_desc(ba + (uint32_t)kk * 2u * (NM / 8) * 128u, (NM / 8) * 128u, 128u);
                                mma_f16_ss(d0 + (uint32_t)(c * NM), ad, bd, idesc, (j | pp | kk) ? 1u : 0u);
                            }
                        }
                    }
                }
                mma_commit(smem_addr(&xempty[s]));   // the data buffer is read
                mma_commit(smem_addr(&tfull[b]));    // the accumulator is complete
            }
            __syncwarp();
        }
    } else {
        // ---------------- epilogue ----------------
        const int row = 32 * warp + lane;   // this thread's tensor-memory lane = spectrum row
        float osc[CW];
#pragma unroll
        for (int c = 0; c < CW; c++) osc[c] = __ldg(p.oscale + cg * CW + c);
        for (int &pc = pc_epi; warp_next_pass(iter, ps, p, n_tiles); pc++) {
            const int b = pc & 1;
            const bool got = lane == 0 ? wait_bar(&tfull[b], (pc >> 1) & 1) : true;
            if (!__shfl_sync(0xFFFFFFFFu, (int)got, 0)) break;
            tc_fence_after();
            const bool valid = row >= ps.ra && row < ps.rb;
            const uint32_t trow = tmem + (uint32_t)(b * TMC) + ((uint32_t)(32 * warp) << 16);
            const long long q_rel = ps.q0 + row - p.q_begin;
            // store the (Re, Im) pairs of k1 = k1_lo + 4 g + kq of this row and the CW columns
            // store the (Re, Im) pairs of k1 = k1_lo + 4 g + kq of this row for
            // the NC columns c0 .. c0 + NC - 1 of the group
            auto store_cols = [&](int g, int c0, const auto &v) {
                constexpr int NC = sizeof(v) / sizeof(v[0]);
                if (!valid) return;
#pragma unroll
                for (int kq = 0; kq < 4; kq++) {
                    const int k1 = k1_lo + 4 * g + kq;
                    if (k1 >= k1_hi) break;
                    const long long o =
                        (((long long)ps.st * p.a_spectra + q_rel) * (H1 + 1) + k1) * N2 + cg * CW + c0;
                    if constexpr (PREC == 2) {
                        float2 *out = reinterpret_cast<float2 *>(p.A) + o;
#pragma unroll
                        for (int c = 0; c < NC; c++)
                            out[c] = make_float2(v[c][2 * kq] * osc[c0 + c], v[c][2 * kq + 1] * osc[c0 + c]);
                    } else {
                        uint32_t hv[NC];
#pragma unroll
                        for (int c = 0; c < NC; c++) {
                            const __half2 h =
                                __floats2half2_rn(v[c][2 * kq] * osc[c0 + c], v[c][2 * kq + 1] * osc[c0 + c]);
                            hv[c] = *reinterpret_cast<const uint32_t *>(&h);
                        }
                        uint32_t *out = reinterpret_cast<uint32_t *>(p.A) + o;
                        static_assert(NC == 1 || NC == 2 || NC % 4 == 0, "column group width");
                        if constexpr (NC % 4 == 0) {
#pragma unroll
                            for (int c = 0; c < NC; c += 4)
                                reinterpret_cast<uint4 *>(out)[c / 4] = make_uint4(hv[c], hv[c + 1], hv[c + 2], hv[c + 3]);
                        } else if constexpr (NC == 2) {
                            reinterpret_cast<uint2 *>(out)[0] = make_uint2(hv[0], hv[1]);
                        } else {
                            out[0] = hv[0];
                        }
                    }
                }
            };
            if constexpr (NG * CW <= (PH == 16 ? 16 : ONE ? 8 : 4)) {
                // all of the pass's accumulator columns in registers, one wait,
                // tensor memory released before the stores (within the register
                // budget of two CTAs per SM when PH = 8)
                float vall[NG][CW][8];
#pragma unroll
                for (int g = 0; g < NG; g++)
#pragma unroll
                    for (int c = 0; c < CW; c++) tmem_ld8(trow + (uint32_t)(c * NM + 8 * g), vall[g][c]);
                tmem_ld_wait();
                tc_fence_before();
                arrive(&tempty[b]);   // tensor memory free for the pass after next
#pragma unroll
                for (int g = 0; g < NG; g++) store_cols(g, 0, vall[g]);
            } else {
                // at most 8 columns at a time (64 registers of accumulator)
                constexpr int CH = CW < 8 ? CW : 8;
#pragma unroll 1
                for (int g = 0; g < NG; g++) {
#pragma unroll 1
                    for (int c0 = 0; c0 < CW; c0 += CH) {
                        float v[CH][8];
#pragma unroll
                        for (int c = 0; c < CH; c++) tmem_ld8(trow + (uint32_t)((c0 + c) * NM + 8 * g), v[c]);
                        tmem_ld_wait();
                        if (g == NG - 1 && c0 + CH == CW) {
                            tc_fence_before();
                            arrive(&tempty[b]);
                        }
                        store_cols(g, c0, v);
                    }
                }
            }
        }
    }
    // end of segment: every role is through its passes (the epilogue drained
    // the last accumulator, so every MMA of the segment has completed)
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    }
    // teardown: every role has left its loop; the last accumulator was read
    // (or a wait gave up: give the tensor core a bounded moment to finish)
    if (*abort_sm && warp == WMMA) {
        const long long t0 = clock64();
        while (clock64() - t0 < 20000000LL) {
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == WMMA) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEMC));
}

// ---------------------------------------------------------------- host side

// Physical FIR columns per CTA for an N-point transform: 16 where tc_phys
// allows it and the N2 output columns hold a group of 16 / R (all but N = 64)
int phase1_tc_phys(int N, int T, int precision) {
    const int R = phase1_tc_R(N);
    return tc_phys(R, T, precision) == 16 && N / 8 / R >= 16 / R ? 16 : 8;
}

static size_t tc_smem_bytes(int ph, int R, int T, int precision) {
    const size_t b = (size_t)tc_smem(ph, R, T, precision, tc_ks1(ph, R, T, precision), tc_nxb(ph, R, T, precision));
    // at most two CTAs per SM (the tensor memory of two fills the 512 columns)
    const size_t floor = 80 * 1024;
    return b < floor ? floor : b;
}

int phase1_tc_R(int N) {
    const int P = N / 8;
    return P > 1024 ? P / 1024 : 1;
}

bool phase1_tc_supported(int N, int T, int precision) {
    const int R = phase1_tc_R(N);
    return N >= 64 && N <= 65536 && (R == 1 || R == 2 || R == 4 || R == 8) && T >= 1 && T <= 32 &&
           tc_ks(phase1_tc_phys(N, T, precision), R, T, precision) > 0;
}

void build_phase1_tc_tables(int N, int T, int precision, const float *w, std::vector<uint16_t> &bmat,
                            std::vector<float> &oscale, float &s_int) {
    const int R = phase1_tc_R(N), P = N / 8, N2 = P / R, PH = phase1_tc_phys(N, T, precision), CW = PH / R;
    const int KS = tc_ks(PH, R, T, precision), KPS = tc_kps(R, KS), NM = tc_nm(R, KS), TP = tc_tp(T), K = 8 * TP;
    const int H1 = 4 * R, NPB = precision == 2 ? 2 : 1;
    const int n_cg = N2 / CW;
    // [column group][k1-slice][plane][physical column][NM x K]
    bmat.assign((size_t)n_cg * KS * NPB * PH * NM * K, 0);
    oscale.assign(N2, 1.0f);
    // global scale of the FP16 intermediate: |Z| <= 512 sum_j sum_r |w[t + P r]|
    double zmax = 0.0;
    for (int t2 = 0; t2 < N2; t2++) {
        double s = 0.0;
        for (int j = 0; j < R; j++)
            for (int r = 0; r < 8 * T; r++) s += std::fabs((double)w[t2 + (long long)N2 * j + (long long)P * r]);
        zmax = s > zmax ? s : zmax;
    }
    s_int = 1.0f;
    if (precision == 1) {
        const double bound = 512.0 * (zmax > 0.0 ? zmax : 1.0);
        s_int = (float)std::ldexp(1.0, (int)std::floor(std::log2(32768.0 / bound)));
    }
    for (int cgi = 0; cgi < n_cg; cgi++) {
        for (int c = 0; c < CW; c++) {
            const int t2 = cgi * CW + c;
            // per-block (output column) power-of-two scale of the weights operand
            double bmax = 0.0;
            for (int j = 0; j < R; j++)
                for (int r = 0; r < 8 * T; r++) {
                    const double a = std::fabs((double)w[t2 + (long long)N2 * j + (long long)P * r]);
                    bmax = a > bmax ? a : bmax;
                }
            const double sB = bmax > 0.0 ? std::ldexp(1.0, (int)std::floor(std::log2(32768.0 / bmax))) : 1.0;
            oscale[t2] = (float)((double)s_int / sB);
            for (int sl = 0; sl < KS; sl++)
                for (int j = 0; j < R; j++) {
                    const long long t = t2 + (long long)N2 * j;
                    const size_t blk0 = (((size_t)cgi * KS + sl) * NPB * PH + j * CW + c) * NM * K;
                    for (int nrow = 0; nrow < NM; nrow++) {
                        const int k1 = sl * KPS + nrow / 2, im = nrow % 2;
                        for (int k = 0; k < K; k++) {
                            const int t1 = k % 8, jj = k / 8;
                            double val = 0.0;
                            if (nrow / 2 < KPS && k1 <= H1 && jj < T) {
                                const long long tf = (long long)P * t1 + t;
                                const long long ph = ((long long)k1 * tf) % N;
                                const double ang = -2.0 * M_PI * (double)ph / (double)N;
                                val = (double)w[t + (long long)P * k] * (im ? std::sin(ang) : std::cos(ang)) * sB;
                            }
                            const size_t off =
                                (size_t)(k / 8) * (NM / 8) * 64 + (nrow / 8) * 64 + (nrow % 8) * 8 + (k % 8);
                            if (precision == 2) {
                                // hi + lo planes: val = hi + lo to 2^-16 of hi
                                const __nv_bfloat16 hi = __float2bfloat16_rn((float)val);
                                const __nv_bfloat16 lo = __float2bfloat16_rn((float)(val - (double)__bfloat162float(hi)));
                                bmat[blk0 + off] = __bfloat16_as_ushort(hi);
                                bmat[blk0 + (size_t)PH * NM * K + off] = __bfloat16_as_ushort(lo);
                            } else {
                                bmat[blk0 + off] = __half_as_ushort(__float2half_rn((float)val));
                            }
                        }
                    }
                }
        }
    }
}

template <int R, int T, int PREC, int PH>
static cudaError_t launch_tc_ph(const Phase1TcParams &p, cudaStream_t s) {
    const size_t smem = tc_smem_bytes(PH, R, T, PREC);
    cudaError_t e = cudaFuncSetAttribute(k_phase1_tc<R, T, PREC, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int n_cg = p.N2 / (PH / R);
    constexpr int KS = tc_ks1(PH, R, T, PREC);
    const long long n_units = (long long)n_cg * KS * p.n_streams * ((p.q_count + kTcRows - 1) / kTcRows);
    // one wave: two CTAs per SM when two fit in shared memory, else one
    const long long ctas = (long long)p.splits * (tc_one_cta(PH, R, T, PREC) ? 1 : 2);
    const int grid = (int)(n_units < ctas ? n_units : ctas);
    if (grid < 1) return cudaErrorInvalidValue;
    k_phase1_tc<R, T, PREC, PH><<<grid, tc_threads(tc_one_cta(PH, R, T, PREC)), smem, s>>>(p);
    return cudaGetLastError();
}

// the kernel with the column count phase1_tc_phys gives for this N
template <int R, int T, int PREC>
static cudaError_t launch_tc(const Phase1TcParams &p, cudaStream_t s) {
    if constexpr (tc_phys(R, T, PREC) == 16) {
        if constexpr (R == 1) {
            if (p.N2 < 16) return launch_tc_ph<R, T, PREC, 8>(p, s);
        }
        return launch_tc_ph<R, T, PREC, 16>(p, s);
    } else {
        return launch_tc_ph<R, T, PREC, 8>(p, s);
    }
}

template <int R, int PREC>
static cudaError_t launch_tc_t(int T, const Phase1TcParams &p, cudaStream_t s) {
    switch (T) {
        case 1: return launch_tc<R, 1, PREC>(p, s);
        case 2: return launch_tc<R, 2, PREC>(p, s);
        case 4: return launch_tc<R, 4, PREC>(p, s);
        case 8: return launch_tc<R, 8, PREC>(p, s);
        case 16: return launch_tc<R, 16, PREC>(p, s);
        case 32: return launch_tc<R, 32, PREC>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int PREC>
static cudaError_t launch_tc_r(int R, int T, const Phase1TcParams &p, cudaStream_t s) {
    switch (R) {
        case 1: return launch_tc_t<1, PREC>(T, p, s);
        case 2: return launch_tc_t<2, PREC>(T, p, s);
        case 4: return launch_tc_t<4, PREC>(T, p, s);
        case 8: return launch_tc_t<8, PREC>(T, p, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_unpack_cols(const UnpackColsParams &p, cudaStream_t s) {
    if (p.RTP % 64) return cudaErrorInvalidValue;
    if (p.row_begin % 64 || p.row_end % 64 || p.row_begin < 0 || p.row_end > p.RTP || p.row_end < p.row_begin)
        return cudaErrorInvalidValue;
    if (p.row_end == p.row_begin) return cudaSuccess;
    if (p.P % 64) {
        if (p.row_begin != 0 || p.row_end != p.RTP) return cudaErrorInvalidValue;   // whole buffer only
        const long long total = (long long)p.n_streams * p.P * p.RTP;
        const long long blocks = (total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192;
        k_unpack_cols_small<<<(unsigned)blocks, 256, 0, s>>>(p);
    } else {
        dim3 grid(p.P / 64, (p.row_end - p.row_begin) / 64, p.n_streams);
        k_unpack_cols<<<grid, 256, 0, s>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_phase1_tc(int T, int precision, const Phase1TcParams &p, cudaStream_t s) {
    if (p.q_count <= 0) return cudaSuccess;
    const int R = phase1_tc_R(p.N);
    return precision == 2 ? launch_tc_r<2>(R, T, p, s) : launch_tc_r<1>(R, T, p, s);
}

}  // namespace fe
