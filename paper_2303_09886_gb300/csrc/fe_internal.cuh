// Internal declarations shared by the libfengine translation units.
//
// Device data path of one fengine_process_chunk call (Sec. 2.1 steps 1-6):
//   k_delay_table   FP64 delay/phase model per spectrum -> coarse c, fine delta, phase
//   k_phase1<T,N1>  unpack + coarse delay + PFB FIR (Eq. 1) + first FFT stage
//                   (real N1-point DFT over t1, twiddle by exp(-2 pi i k1 t2 / N))
//   k_phase2w       1024-point FFT over t2 + fine-delay rotation + gain +
//                   requantise + channel-major corner turn (FP32 form,
//                   persistent, one warp per sequence), or
//   k_phase2<N2>    the same for N2 < 1024
// In the reduced-precision forms phase 1 is k_phase1_tc (tcgen05 tensor
// cores: unpack + coarse delay + FIR + first DFT stage with its twiddle in one
// contraction); the second stage reads its FP16 (FP16 form) or FP32 (BF16
// form) output.
//   k_tail_update   keep the last H packed samples of every stream
// with the four-step split t = N2 t1 + t2, k = k1 + N1 k2 of the 2n-point
// real DFT (the exp(-2 pi i k1 t2 / N) cross term is the twiddle).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/fengine.h"

namespace fe {

constexpr int kMaxSeg = 16;   // FENGINE_MAX_DELAY_SEGMENTS
constexpr int kMaxGainSeg = 4;  // FENGINE_MAX_GAIN_SETS
constexpr int kHeapSamples = 4096;   // samples per digitiser heap (Sec. 2.2)

// One linear delay/phase segment of a stream, applied from t_apply on.
struct DelaySeg {
    long long t_apply, t_ref;
    double d0, rate, phi0, phi_rate;
};

// Per-stream delay models, device resident: seg[stream * kMaxSeg + i].
struct DelayTableParams {
    const DelaySeg *seg;
    const int *nseg;          // [stream]
    int n_streams;
    int N;                    // FFT length 2n
    long long m0;             // first spectrum of the call
    int M;                    // spectra per call
    int min_delay, max_delay; // coarse delays clamp into [min_delay, max_delay]
    int *ctab;                // out [stream][M] coarse delay
    float2 *ftab;             // out [stream][M] (fine delay delta, phase reduced to [-pi, pi))
    int *err;                 // set to 1 if a coarse delay had to be clamped
    // gain sets: the set of spectrum t0 is the last one with t_apply <= t0 (set 0 before all)
    const long long *g_tapply; // [stream][kMaxGainSeg], nullptr: one set
    const int *n_gsets;        // [stream]
    unsigned char *gsel;       // out [stream][M] gain-set index (when g_tapply is given)
    unsigned char *cchg;       // out [stream][M] 1 where the coarse delay differs from the previous spectrum's (optional)
};

// Lost data (Sec. 3.7): per-spectrum usability from the received-heap flags,
// per-output-heap flags, and the received flags of the history heaps kept for
// the next call. Heaps are kHeapSamples long and start at multiples of it.
struct LostDataParams {
    const unsigned char *valid;      // [stream][L / kHeapSamples] of this chunk, nullptr = all received
    const unsigned char *hv_in;      // [stream][HV] history heaps t_in/4096 - HV + i
    unsigned char *hv_out;           // [stream][HV] for the next call
    int HV;                          // history heaps kept
    long long heap0;                 // t_in / kHeapSamples
    int chunk_heaps;                 // L / kHeapSamples
    const int *ctab;                 // [stream][M]
    int n_ant, N, T, M, S;
    long long m0;
    unsigned char *heap_flags;       // out [ant][ceil(M / S)], nullptr = not wanted
};
cudaError_t launch_lost_data(const LostDataParams &p, cudaStream_t s);

struct Phase1Params {
    const uint8_t *chunk;     // [stream][chunk_bytes]
    const uint8_t *hist;      // [stream][hist_bytes], samples [t_in - H, t_in)
    long long chunk_bytes, hist_bytes;
    long long H;              // history samples (multiple of 4)
    long long L;              // chunk samples
    int N, N2, W, C;          // FFT length, second-stage size, t2 per CTA, columns per CTA
    int M;                    // spectra per call
    long long m0;             // first spectrum of the call
    long long t_in;           // first sample of the chunk
    const float *w;           // [N*T] prototype, w[t + N j]
    const float2 *tw1;        // [(N1/2+1)][N2] exp(-2 pi i k1 t2 / N)
    const int *ctab;          // [stream][M]
    float2 *A;                // out [stream][a_spectra][N1/2+1][N2], spectrum q at row q - q_begin
                              // (FP16 pairs in 4-byte elements when half_out)
    int half_out;             // 1: store B as FP16 (re, im) pairs (FP16 tensor-core form)
    int *window_tap;          // optional out [stream][M][N]
    int q_begin, q_count;     // the slab of spectra this launch covers
    int a_spectra;            // spectra per stream in the intermediate buffer
};

struct Phase2Params {
    const float2 *A;          // [stream][a_spectra][N1/2+1][N2], spectrum q at row q - q_begin
                              // (FP16 pairs in 4-byte elements for the FP16 tensor-core form)
    int q_begin, q_count;     // the slab of spectra this launch covers
    int a_spectra;            // spectra per stream in the intermediate buffer
    const float2 *tw2;        // [N2] exp(-2 pi i q / N2)
    const float2 *gains;      // [stream][n_gsets_max][n] gain sets
    const unsigned char *gsel;   // [stream][M] gain-set index per spectrum, nullptr = set 0
    int n_gsets_max;          // sets per stream in `gains`
    const float2 *ftab;       // [stream][M]
    int N, N1, M, S, R2;      // FFT length, first-stage size, spectra/call, spectra/heap, spectra/CTA
    int8_t *out;              // [ant][heap][n][S_h][pol][2]
    float2 *prequant;         // optional [stream][M][n]
    int half_in;              // 1: A holds FP16 (re, im) pairs (tensor-core phase 1, FP16 form)
    float tc_unscale;         // inverse of the power-of-two scale of an FP16 A (1 otherwise)
};

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_delay_table(const DelayTableParams &p, cudaStream_t s);
cudaError_t launch_tail_update(const uint8_t *hist_in, const uint8_t *chunk, uint8_t *hist_out,
                               long long hist_bytes, long long chunk_bytes, int n_streams,
                               cudaStream_t s);
cudaError_t launch_phase1(int T, int N1, const Phase1Params &p, int n_streams, cudaStream_t s);
cudaError_t launch_phase2(int N2, const Phase2Params &p, int n_ant, cudaStream_t s);
// FP32 second stage for N2 = 1024 (launch_phase2 routes it there): one warp
// per sequence, two in-register 32-point DFTs around one shared-memory transpose
cudaError_t launch_phase2w(const Phase2Params &p, int n_ant, cudaStream_t s);
size_t phase2w_smem_bytes();

// ---- grouped launches (batching): the launches of several plans that use
// one kernel instantiation, as one grid. Member m owns the blocks
// [start[m], start[m + 1]) and runs with parameters p[m]. The whole group is
// passed by value as the kernel's parameter (at most kMaxGroup members, a
// few KB), so a grouped launch is captured into a CUDA graph like any other.
constexpr int kMaxGroup = 64;
template <class P>
struct GroupArgs {
    P p[kMaxGroup];
    int start[kMaxGroup + 1];   // start[n] = blocks of the launch
    int aux[kMaxGroup];         // the member's blocks along y (grid kernels) or antennas (k_phase2w)
    int gx;                     // blocks along x, the same for every member (grid kernels)
    int n;
};
using Phase1Group = GroupArgs<Phase1Params>;
using Phase2Group = GroupArgs<Phase2Params>;
// one member's blocks and their (gx, gy) in its own launch
int phase1_blocks(int N1, const Phase1Params &p, int n_streams, int *gx, int *gy);
int phase2_blocks(int N2, const Phase2Params &p, int n_ant, int *gx, int *gy);   // N2 < 1024
long long phase2w_items(const Phase2Params &p, int n_ant);                        // work items of k_phase2w
int phase2w_wave();                                                                 // CTAs of one k_phase2w wave
cudaError_t launch_phase1_group(int T, int N1, const Phase1Group &g, cudaStream_t s);
cudaError_t launch_phase2_group(int N2, bool half_in, const Phase2Group &g, cudaStream_t s);
cudaError_t launch_phase2w_group(bool half_in, const Phase2Group &g, cudaStream_t s);

// A call of a plan with its phase launches handed back instead of enqueued
// (batching): the per-slab parameters fengine_process_chunk would launch.
// The FP32 form only; its other kernels (delay table, lost data, history
// tail) are enqueued on the call's stream as usual.
struct DeferredCall {
    int T = 0, N1 = 0, N2 = 0, n_streams = 0, n_ant = 0;
    std::vector<Phase1Params> p1;   // per slab, in order
    std::vector<Phase2Params> p2;
};
// whether process_chunk_deferred hands back this plan's phase launches
bool plan_defers(fengine_plan_t pl);
// fengine_process_chunk with the FP32 form's phase launches returned in def
// (*deferred = true); other forms run as fengine_process_chunk (*deferred =
// false). No debug outputs.
fengine_status process_chunk_deferred(fengine_plan_t pl, cudaStream_t st, const uint8_t *d_packed,
                                      int64_t first_sample, const uint8_t *d_valid, int8_t *d_out,
                                      uint8_t *d_heap_flags, int64_t *first_spectrum, DeferredCall *def,
                                      bool *deferred);

// Tile shapes (host and device agree through these).
constexpr int kP1Rows = 32;   // spectra per phase-1 CTA
inline int phase1_W(int N1, int N2) {
    int w = 512 / N1;           // 512 FIR columns per tile
    return w < N2 ? w : N2;
}
// shared memory of a k_phase2<N2> CTA of R2 spectra (the sequences of both
// pols, padded rows, the rotation tables and the heap row info)
constexpr long long phase2_smem_c(int N2, int R2) {
    const int LD = N2 + N2 / 16 + 1, LO = N2 < 32 ? N2 : 32, HI = N2 / LO;
    return 8LL * (2LL * R2 * LD + 2LL * R2 * ((HI + 1) + (LO + 1) + 1)) + 12LL * R2;
}
// spectra per k_phase2 CTA: up to 4096 / N2 (at most 32), halved while the
// CTA's shared memory would keep three CTAs (the register limit) off an SM,
// down to 8 (the corner turn writes 4 R2-byte rows: 32 bytes at R2 = 8)
constexpr int phase2_R2_for(int N2) {
    int r = 4096 / N2;
    if (r > 32) r = 32;
    if (r < 1) r = 1;
    while (r > 8 && phase2_smem_c(N2, r) > 74 * 1024) r /= 2;
    return r;
}
inline int phase2_R2(int N2) { return phase2_R2_for(N2); }
size_t phase2_smem_bytes(int N2, int R2);

// Phase 1 of the reduced-precision forms on tcgen05 tensor cores
// (k_phase1_tc.cu): first-stage radix N1 = 8 R with R = phase1_tc_R(N), so
// N2 = N / N1 <= 1024; the output is the second-stage input
// [stream][a_spectra][N1/2 + 1][N2] as FP16 pairs (FP16 form, scaled by
// s_int) or FP32 pairs (BF16 form). It reads the samples as FP16 column
// sequences: cols[stream][col][r] holds the sample at timestamp
// (rb + r) P + col - c0, P = N / 8, c0 = the stream's first coarse delay of
// the call (k_unpack_cols writes them each call).
struct UnpackColsParams {
    const uint8_t *chunk;     // [stream][chunk_bytes]
    const uint8_t *hist;      // [stream][hist_bytes], samples [t_in - H, t_in)
    long long chunk_bytes, hist_bytes;
    long long H, L, t_in;
    int P;                    // N / 8
    long long rb;             // absolute row of column row 0 (a multiple of 8)
    int RT, RTP;              // rows holding samples; rows per column (padded, a multiple of 64)
    int row_begin, row_end;   // the launch writes rows [row_begin, row_end) (multiples of 64;
                              // [0, RTP) for the whole buffer)
    int bf16;                 // 1: write BF16 hi and lo planes (the lo plane plane_elems after the hi)
    long long plane_elems;    // n_streams P RTP
    uint16_t *cols;           // out [stream][P][RTP] FP16, pre-delayed by ctab[stream][0]
    const int *ctab;          // [stream][M] coarse delays
    int M;
    int n_streams;
};

struct Phase1TcParams {
    const uint16_t *cols;     // [plane][stream][P][RTP] samples (UnpackColsParams): FP16, or BF16 hi
                              // and lo planes in the BF16 form
    long long plane_elems;    // elements per plane
    long long rb;
    int RTP;
    int N, N2;                // FFT length, second-stage size
    int M;                    // spectra per call
    long long m0;             // first spectrum of the call
    int q_begin, q_count;     // the slab of spectra this launch covers
    int a_spectra;            // spectra per stream in the intermediate buffer
    int n_streams;
    int splits;               // SMs of the device: the grid is one wave (1 or 2 CTAs per SM), each CTA a
                              // contiguous share of the passes
    const uint16_t *bmat;     // operand blocks, build_phase1_tc_tables
    const float *oscale;      // [N2] epilogue scale per output column
    const int *ctab;          // [stream][M] coarse delays
    const unsigned char *cchg;   // [stream][M] 1 where the coarse delay changes (DelayTableParams::cchg)
    void *A;                  // out: second-stage input
    int *window_tap;          // optional out [stream][M][N]
    int *err;                 // set to 2 if a bounded wait gave up
};
int phase1_tc_R(int N);
bool phase1_tc_supported(int N, int T, int precision);
int phase1_tc_phys(int N, int T, int precision);
void build_phase1_tc_tables(int N, int T, int precision, const float *w, std::vector<uint16_t> &bmat,
                            std::vector<float> &oscale, float &s_int);
cudaError_t launch_phase1_tc(int T, int precision, const Phase1TcParams &p, cudaStream_t s);
cudaError_t launch_unpack_cols(const UnpackColsParams &p, cudaStream_t s);
// rows of the FP16 column buffer: a call's history + chunk plus the reach of
// a 128-spectrum pass past the chunk end, padded to a multiple of 64
inline int unpack_cols_rows(long long H, long long L, long long D, long long Dmin, int N, int T) {
    const long long P = N / 8;
    const long long rt = (H + L + D - Dmin) / P + 3 + 8;
    const long long reach = 8LL * (127 + (T < 2 ? 2 : T)) + 64;
    return (int)((rt + reach + 63) / 64 * 64);
}

}  // namespace fe
