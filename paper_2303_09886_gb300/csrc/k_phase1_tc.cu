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
// A CTA owns 8 physical columns (CW = 8 / R output columns) and a range of
// (stream, 128-spectrum tile) items; each tile is one pass per run of equal
// coarse delay. Passes are double-buffered: the CTA decodes pass p + 1 while
// the tensor core runs pass p and the epilogue drains pass p - 1 from the
// other half of tensor memory (tcgen05.ld), scales it and stores the
// second-stage input [stream][spectrum][k1][t2] (FP16 pairs, or FP32 pairs in
// the BF16 form).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <vector>

#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcRows = 128;     // spectra per pass: the MMA's M
constexpr int kTcPhys = 8;       // physical FIR columns per CTA
constexpr int kTcTmemCols = 256; // tensor-memory columns per CTA (two pass buffers)

__host__ __device__ constexpr int tc_tp(int T) { return T < 2 ? 2 : T; }                 // K = 8 T' >= 16
__host__ __device__ constexpr int tc_xl(int T) { return 8 * (kTcRows - 1 + tc_tp(T)); } // samples per column
// k1 values of one of ks slices of [0, 4 R], and the operand rows (Re, Im) they take, padded to 16
__host__ __device__ constexpr int tc_kps(int R, int ks) { return (4 * R + 1 + ks - 1) / ks; }
__host__ __device__ constexpr int tc_nm(int R, int ks) { return 16 * ((2 * tc_kps(R, ks) + 15) / 16); }
constexpr long long kTcSmemMax = 227 * 1024;

// Shared-memory bytes with ks k1-slices and nxb decode buffers: the operand
// blocks (BF16: hi and lo planes) and the decoded data (BF16: hi and lo).
__host__ __device__ constexpr long long tc_smem(int R, int T, int prec, int ks, int nxb) {
    return 2LL * ((prec == 2 ? 2 : 1) * kTcPhys * (long long)tc_nm(R, ks) * 8 * tc_tp(T) +
                  (long long)nxb * (prec == 2 ? 2 : 1) * kTcPhys * tc_xl(T)) +
           4 * kTcRows + 64 + 2048;
}
// fewest k1-slices, then two decode buffers (the decode of the next pass
// under the current one's MMAs), that fit in shared memory; 0 if none does
__host__ __device__ constexpr int tc_ks(int R, int T, int prec) {
    return tc_smem(R, T, prec, 1, 1) <= kTcSmemMax   ? 1
           : tc_smem(R, T, prec, 2, 1) <= kTcSmemMax ? 2
           : tc_smem(R, T, prec, 4, 1) <= kTcSmemMax ? 4
           : tc_smem(R, T, prec, 8, 1) <= kTcSmemMax ? 8
                                                      : 0;
}
__host__ __device__ constexpr int tc_nxb(int R, int T, int prec) {
    return tc_smem(R, T, prec, tc_ks(R, T, prec) > 0 ? tc_ks(R, T, prec) : 1, 2) <= kTcSmemMax ? 2 : 1;
}

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

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the given phase of an mbarrier, giving up after about a second.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try(mbar, parity))
        if (clock64() - t0 > 2000000000LL) return false;
    return true;
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

// Offset-binary FP16 of a 10-bit two's-complement field f: the FP16 with
// exponent 2^10 and mantissa (f ^ 512) is 1024 + (v + 512); subtracting 1536
// (exact) gives v. Two fields at once as a half2.
__device__ __forceinline__ uint32_t fields_to_half2(uint32_t f0, uint32_t f1) {
    const uint32_t h = (((f0 ^ 0x200u) | 0x6400u) & 0xFFFFu) | ((((f1 ^ 0x200u) | 0x6400u) & 0xFFFFu) << 16);
    const __half2 r = __hsub2(*reinterpret_cast<const __half2 *>(&h), __halves2half2(__ushort_as_half(0x6600u),
                                                                                     __ushort_as_half(0x6600u)));
    return *reinterpret_cast<const uint32_t *>(&r);
}

__device__ __forceinline__ int field_value(uint32_t f) { return (int)f - (int)((f & 0x200u) << 1); }

// BF16 hi and lo parts of two integer samples (|v| <= 512): hi = RN(v), lo = v - hi, both exact.
__device__ __forceinline__ void ints_to_bf16x2(int v0, int v1, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn((float)v0), h1 = __float2bfloat16_rn((float)v1);
    const __nv_bfloat16 l0 = __float2bfloat16_rn((float)v0 - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn((float)v1 - __bfloat162float(h1));
    hi = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
}

// Sample at position s from the first history sample (history, then chunk;
// zero outside [0, HL)); fields are read as two big-endian bytes.
__device__ __forceinline__ uint32_t field_at(const uint8_t *hist, const uint8_t *chunk, long long s, long long H,
                                             long long HL) {
    if (s < 0 || s >= HL) return 0u;   // the field of value 0
    const bool h = s < H;
    const long long u = h ? s : s - H;
    const uint8_t *b = (h ? hist : chunk) + ((5 * u) >> 2);
    const unsigned v = ((unsigned)__ldg(b) << 8) | (unsigned)__ldg(b + 1);
    return (v >> (6u - 2u * (unsigned)(u & 3))) & 0x3FFu;
}

struct Pass {
    int st, q0, ra, rb, c;
};

}  // namespace

template <int R, int T, int PREC>
__global__ void __launch_bounds__(kTcThreads, 2) k_phase1_tc(const Phase1TcParams p) {
    constexpr int KS = tc_ks(R, T, PREC), KPS = tc_kps(R, KS);   // k1-slices, k1 values per slice
    constexpr int NM = tc_nm(R, KS), TP = tc_tp(T), K = 8 * TP, XL = tc_xl(T), CW = kTcPhys / R;
    constexpr int NPL = PREC == 2 ? 2 : 1;    // data planes: BF16 hi + lo
    constexpr int NPB = PREC == 2 ? 2 : 1;    // operand planes: BF16 hi + lo
    constexpr int H1 = 4 * R;                 // k1 in [0, H1]
    constexpr int BBLK = NM * K;              // 16-bit elements per operand block
    constexpr int TMC = CW * NM;              // tensor-memory columns per pass buffer
    constexpr int NG = (2 * KPS + 7) / 8;     // 8-column groups holding (Re, Im) of the slice's k1
    constexpr int NXB = tc_nxb(R, T, PREC);   // decode buffers
    static_assert(KS > 0, "shape does not fit in shared memory");
    static_assert(2 * TMC <= kTcTmemCols, "tensor memory");
    extern __shared__ __align__(1024) uint8_t smem[];
    uint16_t *bsm = reinterpret_cast<uint16_t *>(smem);            // [NPB][kTcPhys][BBLK]
    uint16_t *xsm = bsm + NPB * kTcPhys * BBLK;                    // [NXB][NPL][kTcPhys][XL]
    int *c_sm = reinterpret_cast<int *>(xsm + NXB * NPL * kTcPhys * XL);
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(c_sm + kTcRows);   // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 2);
    int *flag_sm = reinterpret_cast<int *>(tmem_slot + 1);         // [0] abort

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_cg = p.N2 / CW;
    // block = (column group, k1-slice, item range)
    const int cg = blockIdx.x / (p.splits * KS), slice = (blockIdx.x / p.splits) % KS, split = blockIdx.x % p.splits;
    const int k1_lo = slice * KPS, k1_hi = min(H1 + 1, k1_lo + KPS);
    const int n_tiles = (p.q_count + kTcRows - 1) / kTcRows;
    const int n_items = p.n_streams * n_tiles;
    const int it_begin = (int)((long long)n_items * split / p.splits);
    const int it_end = (int)((long long)n_items * (split + 1) / p.splits);
    if (cg >= n_cg) return;

    // the CTA's operand blocks (weights x DFT x twiddle), resident for all its items
    {
        const uint4 *src =
            reinterpret_cast<const uint4 *>(p.bmat) + ((long long)cg * KS + slice) * (NPB * kTcPhys * BBLK / 8);
        uint4 *dst = reinterpret_cast<uint4 *>(bsm);
        for (int i = tid; i < NPB * kTcPhys * BBLK / 8; i += kTcThreads) dst[i] = __ldg(src + i);
    }
    float osc[CW];
#pragma unroll
    for (int c = 0; c < CW; c++) osc[c] = __ldg(p.oscale + cg * CW + c);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        flag_sm[0] = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(kTcTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const long long H = p.H, HL = p.H + p.L;
    const int P = p.N / 8, N2 = p.N2;
    constexpr uint32_t idesc = mma_idesc(kTcRows, NM, PREC == 2 ? 1 : 0);

    // ---- pass generation (every thread computes the same sequence) ----
    int it = it_begin, ra = -1, rows = 0, st = 0, q0 = 0, uniform = 0;
    // coarse delay of row tid of an item, loaded one item ahead
    auto item_delay = [&](int item) -> int {
        const int s2 = item / n_tiles, qq = p.q_begin + (item % n_tiles) * kTcRows;
        return (item < it_end && qq + tid < p.q_begin + p.q_count && tid < kTcRows)
                   ? __ldg(p.ctab + (long long)s2 * p.M + qq + tid)
                   : 0;
    };
    int c_pref = item_delay(it);
    auto next_pass = [&](Pass &ps) -> bool {
        for (;;) {
            if (ra < 0) {
                if (it >= it_end) return false;
                st = it / n_tiles;
                q0 = p.q_begin + (it % n_tiles) * kTcRows;
                rows = min(kTcRows, p.q_begin + p.q_count - q0);
                const int c_this = c_pref;
                c_pref = item_delay(it + 1);
                __syncthreads();   // the previous item's delays are no longer read
                if (tid < rows) c_sm[tid] = c_this;
                __syncthreads();
                uniform = __syncthreads_and(tid >= rows || c_sm[tid] == c_sm[0]);
                ra = 0;
            }
            if (ra >= rows) {
                ra = -1;
                it++;
                continue;
            }
            const int c = c_sm[ra];
            int rb = ra + 1;
            if (ra == 0 && uniform) {
                rb = rows;
            } else {
                while (rb < rows && c_sm[rb] == c) rb++;
            }
            ps = Pass{st, q0, ra, rb, c};
            ra = rb;
            return true;
        }
    };

    // ---- decode of one pass into data buffer b ----
    // Fast path (the pass's samples all inside the chunk): a thread takes
    // (run j, rows v and v + 1) items, a run being CW consecutive columns of
    // one row; its packed words are loaded into registers by fetch() one
    // step ahead (under the previous pass's epilogue), and decode() converts
    // them into 16-bit samples in shared memory.
    constexpr int NIT = R * (XL / 2);                              // items per pass
    constexpr int MAXI = (NIT + kTcThreads - 1) / kTcThreads;      // items per thread
    constexpr int NW = (30 + 10 * CW) / 32 + 1;                    // words covering a run at any bit offset
    constexpr int PFI = MAXI * 2 * NW <= 40 ? MAXI : 40 / (2 * NW);   // items prefetched into registers
    uint32_t rw[PFI][2][NW];
    // position (from the first history sample) of row v = 0 at column t = 0
    auto pass_base = [&](const Pass &ps) -> long long {
        return (long long)p.N * (p.m0 + ps.q0) - (p.t_in - H) - ps.c;
    };
    auto is_fast = [&](const Pass &ps) -> bool {
        const long long base = pass_base(ps);
        const long long lo = base + cg * CW, hi = base + cg * CW + (long long)N2 * (R - 1) + CW +
                                                  (long long)P * (XL - 1);
        return lo >= H && hi < HL - 16 && !p.window_tap;
    };
    // bit position (from the chunk start) of the first bit of item e's row rr
    auto item_bit = [&](long long base, int e, int rr) -> long long {
        const int j = e / (XL / 2), v = 2 * (e - j * (XL / 2));
        return 10 * (base - H + cg * CW + (long long)N2 * j + (long long)P * (v + rr));
    };
    auto fetch = [&](const Pass &ps, bool fast) {
        if (!fast) return;
        const uint32_t *w32 = reinterpret_cast<const uint32_t *>(p.chunk + (long long)ps.st * p.chunk_bytes);
        const long long base = pass_base(ps);
#pragma unroll
        for (int i = 0; i < PFI; i++) {
            const int e = tid + i * kTcThreads;
            if (e < NIT) {
#pragma unroll
                for (int rr = 0; rr < 2; rr++) {
                    const uint32_t *wp = w32 + (item_bit(base, e, rr) >> 5);
#pragma unroll
                    for (int k = 0; k < NW; k++) rw[i][rr][k] = __ldg(wp + k);
                }
            }
        }
    };
    auto decode = [&](const Pass &ps, int b, bool fast) {
        uint16_t *xb = xsm + (size_t)(b % NXB) * NPL * kTcPhys * XL;
        const long long base = pass_base(ps);
        if (fast) {
            const uint32_t *w32 = reinterpret_cast<const uint32_t *>(p.chunk + (long long)ps.st * p.chunk_bytes);
#pragma unroll
            for (int i = 0; i < MAXI; i++) {
                const int e = tid + i * kTcThreads;
                if (e >= NIT) break;
                const int j = e / (XL / 2), v = 2 * (e - j * (XL / 2));
                uint32_t f[2][CW];
#pragma unroll
                for (int rr = 0; rr < 2; rr++) {
                    const long long bit = item_bit(base, e, rr);
                    const int off = (int)(bit & 31);
                    // big-endian words, then shifted so that bit 0 is the run's first bit:
                    // field c sits at the compile-time bit 10 c
                    uint32_t w[NW + 1], a[NW];
#pragma unroll
                    for (int k = 0; k < NW; k++) {
                        const uint32_t raw = i < PFI ? rw[i < PFI ? i : 0][rr][k] : __ldg(w32 + (bit >> 5) + k);
                        w[k] = __byte_perm(raw, 0u, 0x0123u);
                    }
                    w[NW] = 0u;
#pragma unroll
                    for (int k = 0; k < NW; k++) a[k] = __funnelshift_l(w[k + 1], w[k], (unsigned)off);
#pragma unroll
                    for (int c = 0; c < CW; c++) {
                        const int bb = 10 * c;
                        const uint32_t hi = a[bb >> 5], lo = (bb >> 5) + 1 < NW ? a[(bb >> 5) + 1] : 0u;
                        f[rr][c] = __funnelshift_l(lo, hi, (unsigned)(bb & 31)) >> 22;
                    }
                }
#pragma unroll
                for (int c = 0; c < CW; c++) {
                    const int i2 = j * CW + c;
                    if constexpr (PREC == 2) {
                        uint32_t h, l;
                        ints_to_bf16x2(field_value(f[0][c]), field_value(f[1][c]), h, l);
                        *reinterpret_cast<uint32_t *>(xb + (size_t)i2 * XL + v) = h;
                        *reinterpret_cast<uint32_t *>(xb + (size_t)(kTcPhys + i2) * XL + v) = l;
                    } else {
                        *reinterpret_cast<uint32_t *>(xb + (size_t)i2 * XL + v) = fields_to_half2(f[0][c], f[1][c]);
                    }
                }
            }
        } else {
            // general: every sample checked against history / chunk / range;
            // the debug window tap (first FIR tap of each spectrum) is written here
            const uint8_t *hist = p.hist + (long long)ps.st * p.hist_bytes;
            const uint8_t *chunk = p.chunk + (long long)ps.st * p.chunk_bytes;
            for (int e = tid; e < kTcPhys * (XL / 2); e += kTcThreads) {
                const int i = e / (XL / 2), v = 2 * (e - i * (XL / 2));
                const int j = i / CW, c = i - j * CW;
                const long long t = (long long)cg * CW + c + (long long)N2 * j;
                uint32_t f[2];
#pragma unroll
                for (int rr = 0; rr < 2; rr++) {
                    f[rr] = field_at(hist, chunk, base + t + (long long)P * (v + rr), H, HL);
                    const int vv = v + rr;
                    if (p.window_tap && vv < 8 * kTcRows) {
                        const int mrow = vv >> 3, t1 = vv & 7;
                        if (mrow >= ps.ra && mrow < ps.rb)
                            p.window_tap[((long long)ps.st * p.M + ps.q0 + mrow) * p.N + (long long)P * t1 + t] =
                                field_value(f[rr]);
                    }
                }
                if constexpr (PREC == 2) {
                    uint32_t h, l;
                    ints_to_bf16x2(field_value(f[0]), field_value(f[1]), h, l);
                    *reinterpret_cast<uint32_t *>(xb + (size_t)i * XL + v) = h;
                    *reinterpret_cast<uint32_t *>(xb + (size_t)(kTcPhys + i) * XL + v) = l;
                } else {
                    *reinterpret_cast<uint32_t *>(xb + (size_t)i * XL + v) = fields_to_half2(f[0], f[1]);
                }
            }
        }
    };

    // ---- MMAs of one pass (one thread) ----
    auto issue = [&](int b) {
        const uint32_t d0 = tmem + (uint32_t)(b * TMC);
        const uint32_t xa0 = smem_addr(xsm + (size_t)(b % NXB) * NPL * kTcPhys * XL), ba0 = smem_addr(bsm);
#pragma unroll 1
        for (int c = 0; c < CW; c++) {
#pragma unroll 1
            for (int j = 0; j < R; j++) {
                const int i = j * CW + c;
                // FP16: x B. BF16: x_hi B_hi + x_lo B_hi + x_hi B_lo (x_lo B_lo is
                // below 2^-9 / 512 of the result and left out)
#pragma unroll
                for (int pp = 0; pp < (PREC == 2 ? 3 : 1); pp++) {
                    const int pl = pp == 1 ? 1 : 0, pb = pp == 2 ? 1 : 0;
                    const uint32_t xa = xa0 + (uint32_t)((pl * kTcPhys + i) * XL * 2);
                    const uint32_t ba = ba0 + (uint32_t)((pb * kTcPhys + i) * BBLK * 2);
#pragma unroll
                    for (int kk = 0; kk < K / 16; kk++) {
                        const uint64_t ad = mat_desc(xa + 32u * kk, 16u, 128u);
                        const uint64_t bd = mat_desc(ba + (uint32_t)kk * 2u * (NM / 8) * 128u, (NM / 8) * 128u, 128u);
                        mma_f16_ss(d0 + (uint32_t)(c * NM), ad, bd, idesc, (j | pp | kk) ? 1u : 0u);
                    }
                }
            }
        }
        mma_commit(smem_addr(&mbar[b]));
    };

    // ---- epilogue of one pass from tensor-memory buffer b ----
    auto epilogue = [&](const Pass &ps, int b) {
        const int wg = warp >> 2, row = 32 * (warp & 3) + lane;
        const bool valid = row >= ps.ra && row < ps.rb;
        const uint32_t trow = tmem + (uint32_t)(b * TMC) + ((uint32_t)(32 * (warp & 3)) << 16);
        const long long q_rel = ps.q0 + row - p.q_begin;
        for (int g = wg; g < NG; g += 2) {
            float v[CW][8];
#pragma unroll
            for (int c = 0; c < CW; c++) tmem_ld8(trow + (uint32_t)(c * NM + 8 * g), v[c]);
            tmem_ld_wait();
            if (valid) {
#pragma unroll
                for (int kq = 0; kq < 4; kq++) {
                    const int k1 = k1_lo + 4 * g + kq;
                    if (k1 >= k1_hi) break;
                    const long long o = (((long long)ps.st * p.a_spectra + q_rel) * (H1 + 1) + k1) * N2 + cg * CW;
                    if constexpr (PREC == 2) {
                        float2 *out = reinterpret_cast<float2 *>(p.A) + o;
#pragma unroll
                        for (int c = 0; c < CW; c++)
                            out[c] = make_float2(v[c][2 * kq] * osc[c], v[c][2 * kq + 1] * osc[c]);
                    } else {
                        uint32_t hv[CW];
#pragma unroll
                        for (int c = 0; c < CW; c++) {
                            const __half2 h = __floats2half2_rn(v[c][2 * kq] * osc[c], v[c][2 * kq + 1] * osc[c]);
                            hv[c] = *reinterpret_cast<const uint32_t *>(&h);
                        }
                        uint32_t *out = reinterpret_cast<uint32_t *>(p.A) + o;
                        if constexpr (CW == 8) {
                            reinterpret_cast<uint4 *>(out)[0] = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                            reinterpret_cast<uint4 *>(out)[1] = make_uint4(hv[4], hv[5], hv[6], hv[7]);
                        } else if constexpr (CW == 4) {
                            reinterpret_cast<uint4 *>(out)[0] = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                        } else if constexpr (CW == 2) {
                            reinterpret_cast<uint2 *>(out)[0] = make_uint2(hv[0], hv[1]);
                        } else {
                            out[0] = hv[0];
                        }
                    }
                }
            }
        }
        tc_fence_before();
    };

    // ---- the pipeline ----
    Pass cur{}, prev{}, nxt{};
    bool have_prev = false;
    int b = 0;
    uint32_t parity = 0u;   // bit k: next phase parity of mbar[k]
    bool aborted = false;
    bool have_cur = next_pass(cur);
    bool fast_cur = have_cur && is_fast(cur);
    if (have_cur) fetch(cur, fast_cur);
    while (have_cur) {
        if (NXB == 1 && have_prev) {
            // one decode buffer: the previous pass's MMAs must have read it
            // (the epilogue's wait below returns at once for this phase)
            if (!mbar_wait(smem_addr(&mbar[b ^ 1]), (parity >> (b ^ 1)) & 1u)) {
                flag_sm[0] = 1;
                atomicExch(p.err, 2);
            }
        }
        decode(cur, b, fast_cur);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (flag_sm[0]) {
            aborted = true;
            break;
        }
        if (tid == 0) issue(b);
        __syncwarp();
        // the next pass's packed words are in flight during this epilogue
        const bool have_nxt = next_pass(nxt);
        const bool fast_nxt = have_nxt && is_fast(nxt);
        if (have_nxt) fetch(nxt, fast_nxt);
        if (have_prev) {
            const int pb = b ^ 1;
            const bool ok = mbar_wait(smem_addr(&mbar[pb]), (parity >> pb) & 1u);
            parity ^= 1u << pb;
            if (!ok) {
                flag_sm[0] = 1;
                atomicExch(p.err, 2);
            } else {
                tc_fence_after();
                epilogue(prev, pb);
            }
        }
        prev = cur;
        have_prev = true;
        b ^= 1;
        cur = nxt;
        have_cur = have_nxt;
        fast_cur = fast_nxt;
    }
    if (have_prev && !aborted) {
        const int pb = b ^ 1;
        const bool ok = mbar_wait(smem_addr(&mbar[pb]), (parity >> pb) & 1u);
        if (!ok) {
            atomicExch(p.err, 2);
        } else {
            tc_fence_after();
            epilogue(prev, pb);
        }
    } else if (have_prev && aborted) {
        // a wait gave up: wait (bounded) for the last committed pass before
        // releasing tensor memory
        mbar_wait(smem_addr(&mbar[b ^ 1]), (parity >> (b ^ 1)) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols));
}

// ---------------------------------------------------------------- host side

int phase1_tc_slices(int R, int T, int precision) { return tc_ks(R, T, precision); }

size_t phase1_tc_smem_bytes(int R, int T, int precision) {
    const int ks = tc_ks(R, T, precision);
    const size_t b = (size_t)tc_smem(R, T, precision, ks > 0 ? ks : 1, tc_nxb(R, T, precision));
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
           tc_ks(R, T, precision) > 0;
}

void build_phase1_tc_tables(int N, int T, int precision, const float *w, std::vector<uint16_t> &bmat,
                            std::vector<float> &oscale, float &s_int) {
    const int R = phase1_tc_R(N), P = N / 8, N2 = P / R, CW = kTcPhys / R;
    const int KS = tc_ks(R, T, precision), KPS = tc_kps(R, KS), NM = tc_nm(R, KS), TP = tc_tp(T), K = 8 * TP;
    const int H1 = 4 * R, NPB = precision == 2 ? 2 : 1;
    const int n_cg = N2 / CW;
    // [column group][k1-slice][plane][physical column][NM x K]
    bmat.assign((size_t)n_cg * KS * NPB * kTcPhys * NM * K, 0);
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
                    const size_t blk0 = (((size_t)cgi * KS + sl) * NPB * kTcPhys + j * CW + c) * NM * K;
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
                                bmat[blk0 + (size_t)kTcPhys * NM * K + off] = __bfloat16_as_ushort(lo);
                            } else {
                                bmat[blk0 + off] = __half_as_ushort(__float2half_rn((float)val));
                            }
                        }
                    }
                }
        }
    }
}

template <int R, int T, int PREC>
static cudaError_t launch_tc(const Phase1TcParams &p, cudaStream_t s) {
    const size_t smem = phase1_tc_smem_bytes(R, T, PREC);
    cudaError_t e = cudaFuncSetAttribute(k_phase1_tc<R, T, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int n_cg = p.N2 / (kTcPhys / R);
    constexpr int KS = tc_ks(R, T, PREC) > 0 ? tc_ks(R, T, PREC) : 1;
    k_phase1_tc<R, T, PREC><<<n_cg * KS * p.splits, kTcThreads, smem, s>>>(p);
    return cudaGetLastError();
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

cudaError_t launch_phase1_tc(int T, int precision, const Phase1TcParams &p, cudaStream_t s) {
    if (p.q_count <= 0) return cudaSuccess;
    const int R = phase1_tc_R(p.N);
    return precision == 2 ? launch_tc_r<2>(R, T, p, s) : launch_tc_r<1>(R, T, p, s);
}

}  // namespace fe
