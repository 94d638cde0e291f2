// Phase 2, FP32 form for N2 = 1024: one warp computes the whole 1024-point
// FFT of one (spectrum, pol) sequence in registers, then the fine-delay
// rotation, gain, requantisation and corner turn (Sec. 2.1 steps 4-6,
// Sec. 2.2, Sec. 3.6).
//
// With t2 = 32 a + b and k2 = c + 32 d (a, b, c, d in [0, 32)):
//   Y[c][b]     = sum_a exp(-2 pi i c a / 32) B[32 a + b]
//   Y'[c][b]    = exp(-2 pi i c b / 1024) Y[c][b]
//   F[c + 32 d] = sum_b Y'[c][b] exp(-2 pi i d b / 32).
// The sequence arrives in the warp's shared-memory buffer by cp.async; lane
// b reads B[32 a + b] for every a, does the first 32-point DFT in registers,
// applies the twiddle, and writes Y'[.][b] back into the buffer (XOR
// swizzle); after that transpose lane c holds Y'[c][.] and does the second
// 32-point DFT in registers, leaving F[c + 32 d] for every d. One
// shared-memory round trip per point instead of one per radix pass.
//
// A work item is one first-stage class k1 and 4 consecutive spectra of one
// antenna; warp w computes spectrum w / 2, polarisation w % 2. The kernel is
// persistent (a contiguous range of items per CTA) so that each warp's next
// sequence is in flight while the current one is finished. Channel mapping,
// rotation split and upper-half conjugation are those of the other second
// stages:
// slot k2 is channel k1 + N1 k2 for k2 < 512, and for k2 >= 512 (classes
// k1 = 1 .. N1/2 - 1 only) the conjugate of channel N - (k1 + N1 k2).
#include <algorithm>

#include <cuda_fp16.h>

#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kWThreads = 256;
constexpr int kWR = 4;        // spectra per work item (two warps each)
constexpr int kWN2 = 1024;
constexpr int kWPQ = 65;      // per sequence: P[32], Q[32], qu

// 32-bit word of output cell (slot k2, spectrum r) in the staging buffer: the
// 4 cells of a slot are permuted by k2's bits 3-4 so that the 32 lanes of a
// store (consecutive k2) and of a corner-turn read hit 32 banks.
__device__ __forceinline__ int stg_word(int k2, int r) { return k2 * kWR + (r ^ ((k2 >> 3) & 3)); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// A work item is (antenna, class k1, group of kWR consecutive spectra), in
// that order; item -> its fields.
struct WItem {
    int ant, k1, q0;
};
__device__ __forceinline__ WItem witem(const Phase2Params &p, int it, int H1, int G) {
    const int per_ant = (H1 + 1) * G;
    WItem w;
    w.ant = it / per_ant;
    const int rem = it - w.ant * per_ant;
    w.k1 = rem / G;
    w.q0 = p.q_begin + (rem - w.k1 * G) * kWR;
    return w;
}

}  // namespace

size_t phase2w_smem_bytes() {
    return sizeof(float2) * 8 * kWN2              // per-warp sequence buffers (also the transpose tiles)
           + sizeof(unsigned) * kWN2 * kWR        // output staging
           + sizeof(float2) * 2 * kWN2            // gains of the item's slots
           + sizeof(float2) * 2 * kWR * kWPQ      // rotation factors
           + sizeof(float2) * 32 * 32             // twiddles exp(-2 pi i c b / 1024), [c][b]
           + (sizeof(long long) + sizeof(int)) * 2 * kWR;   // row info, two items
}

// Persistent: each CTA takes a contiguous range of work items of equal work.
// Warp w owns sequence (spectrum w / 2, polarisation w % 2) of every item;
// its 8 KB sequence arrives in its shared-memory buffer by cp.async, and the
// copy of the next item's sequence is issued as soon as the buffer has been
// read (after the transpose), so it runs under this item's second DFT,
// epilogue and corner turn.
// The CTAs of one or several plans' second stages in one grid: member m owns
// CTAs [start[m], start[m + 1]) and aux[m] antennas.
template <bool HALF_IN>
__global__ void __launch_bounds__(kWThreads, 2) k_phase2w_group(const Phase2Group g) {
    __shared__ Phase2Params sp;
    __shared__ int sm_b[3];
    if (threadIdx.x == 0) {
        const int m = group_member(g, (int)blockIdx.x);
        sm_b[0] = (int)blockIdx.x - g.start[m];
        sm_b[1] = g.start[m + 1] - g.start[m];
        sm_b[2] = g.aux[m];
        sp = g.p[m];
    }
    __syncthreads();
    const Phase2Params &p = sp;
    const int n_ant = sm_b[2];
    const long long cta_b = sm_b[0], cta_nb = sm_b[1];
#include "k_phase2w_cta.inc"
}

// A single plan's second stage runs as a group of one member (the grouped
// kernel reads the parameters from shared memory, which leaves it without the
// register spills of a variant that reads them from the parameter bank).
template <bool HALF_IN>
static cudaError_t launch_w_group(const Phase2Group &g, cudaStream_t s);

template <bool HALF_IN>
static cudaError_t launch_w(const Phase2Params &p, int n_ant, cudaStream_t s) {
    const long long items = (long long)n_ant * (p.N1 / 2 + 1) * ((p.q_count + kWR - 1) / kWR);
    if (items <= 0) return cudaSuccess;
    const int wave = phase2w_wave();
    if (wave < 1) return cudaErrorUnknown;
    Phase2Group g{};
    g.p[0] = p;
    g.start[0] = 0;
    g.start[1] = (int)std::min<long long>(items, wave);
    g.aux[0] = n_ant;
    g.gx = 1;
    g.n = 1;
    return launch_w_group<HALF_IN>(g, s);
}

long long phase2w_items(const Phase2Params &p, int n_ant) {
    return (long long)n_ant * (p.N1 / 2 + 1) * ((p.q_count + kWR - 1) / kWR);
}

int phase2w_wave() {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(k_phase2w_group<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)phase2w_smem_bytes()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phase2w_group<false>, kWThreads,
                                                      phase2w_smem_bytes()) != cudaSuccess)
        return 0;
    return sms * std::max(per_sm, 1);
}

template <bool HALF_IN>
static cudaError_t launch_w_group(const Phase2Group &g, cudaStream_t s) {
    const size_t smem = phase2w_smem_bytes();
    cudaError_t e =
        cudaFuncSetAttribute(k_phase2w_group<HALF_IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int m = 0; m < g.n; m++)
        if (g.p[m].N / g.p[m].N1 != kWN2) return cudaErrorInvalidValue;
    if (g.n < 1 || g.start[g.n] < 1) return cudaSuccess;
    k_phase2w_group<HALF_IN><<<g.start[g.n], kWThreads, smem, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_phase2w_group(bool half_in, const Phase2Group &g, cudaStream_t s) {
    return half_in ? launch_w_group<true>(g, s) : launch_w_group<false>(g, s);
}

cudaError_t launch_phase2w(const Phase2Params &p, int n_ant, cudaStream_t s) {
    if (p.N / p.N1 != kWN2) return cudaErrorInvalidValue;
    return p.half_in ? launch_w<true>(p, n_ant, s) : launch_w<false>(p, n_ant, s);
}

}  // namespace fe
