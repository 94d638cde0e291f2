// Internal declarations shared by the libfengine translation units.
//
// Device data path of one fengine_process_chunk call (Sec. 2.1 steps 1-6):
//   k_delay_table   FP64 delay/phase model per spectrum -> coarse c, fine delta, phase
//   k_phase1<T,N1>  unpack + coarse delay + PFB FIR (Eq. 1) + first FFT stage
//                   (real N1-point DFT over t1, twiddle by exp(-2 pi i k1 t2 / N))
//   k_phase2w       1024-point FFT over t2 + fine-delay rotation + gain +
//                   requantise + channel-major corner turn (FP32 form,
//                   persistent, one warp per sequence), or
//   k_phase2<N2>    the same for N2 < 1024 (FP32 form), or
//   k_phase2_tc     the same with the 1024-point FFT as two 32-point DFT
//                   contractions on tensor cores (FP16 / BF16 forms)
//   k_tail_update   keep the last H packed samples of every stream
// with the four-step split t = N2 t1 + t2, k = k1 + N1 k2 of the 2n-point
// real DFT (the exp(-2 pi i k1 t2 / N) cross term is the twiddle).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace fe {

constexpr int kMaxSeg = 16;   // FENGINE_MAX_DELAY_SEGMENTS

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
    int max_delay;            // coarse delays clamp into [0, max_delay]
    int *ctab;                // out [stream][M] coarse delay
    float2 *ftab;             // out [stream][M] (fine delay delta, phase reduced to [-pi, pi))
    int *err;                 // set to 1 if a coarse delay had to be clamped
};

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
    const float2 *gains;      // [stream][n]
    const float2 *ftab;       // [stream][M]
    int N, N1, M, S, R2;      // FFT length, first-stage size, spectra/call, spectra/heap, spectra/CTA
    int8_t *out;              // [ant][heap][n][S_h][pol][2]
    float2 *prequant;         // optional [stream][M][n]
    int precision;            // 0 FP32 CUDA cores, 1 FP16 / 2 BF16 tensor-core second stage
    const uint4 *tc;          // tensor-core tables (build_phase2_tc_tables), precision != 0
    float tc_unscale;         // inverse of the scale the reduced-precision path carries
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

// Tile shapes (host and device agree through these).
constexpr int kP1Rows = 32;   // spectra per phase-1 CTA
inline int phase1_W(int N1, int N2) {
    int w = 512 / N1;           // 512 FIR columns per tile
    return w < N2 ? w : N2;
}
inline int phase2_R2(int N2) {
    int r = 4096 / N2;          // 2 pols * R2 * N2 * 8 B <= 64 KiB: two CTAs per SM
    if (r > 32) r = 32;
    if (r < 1) r = 1;
    return r;
}
size_t phase2_smem_bytes(int N2, int R2);

// Reduced-precision second stage (N2 = 1024 only): two 32-point DFT
// contractions on tensor cores. The tables hold the DFT matrices as per-lane
// mma fragments (hi and lo parts) and the 32 x 32 twiddle (times 2^-5);
// kPhase2TcTableLen uint4 entries, built on the host for precision 1 (FP16)
// or 2 (BF16).
constexpr int kPhase2TcTableLen = 2560;
void build_phase2_tc_tables(int precision, uint4 *out);
size_t phase2_tc_smem_bytes(int precision);
cudaError_t launch_phase2_tc(const Phase2Params &p, int n_ant, cudaStream_t s);

}  // namespace fe
