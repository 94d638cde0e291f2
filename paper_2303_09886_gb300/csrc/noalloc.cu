// fengine_process_chunk_noalloc: the same channelizer kernels as
// fengine_process_chunk, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: their device memory is handed out in
// full by another allocator (a framework's caching allocator or a fixed
// per-process budget), or they run in a latency-critical loop where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.
// This entry point takes every input and output from the caller and keeps
// its working storage (delay table, twiddle tables, delay models and the
// inter-phase intermediate) in one file-scope device array of fixed size,
// which every GPU that loads the library holds until the process exits.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/fengine.h"
#include "fe_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)FENGINE_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The working storage. In host code this name is only a host-side handle of
// the symbol, never a device address: the kernels get the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_scratch_dev[kMaxDevices] = {nullptr};

// Set-up once per device, with that device current. The lookup is not
// attempted while `st` is being captured into a graph (the first call on a
// device must come before any capture): that call is refused instead.
cudaError_t scratch_address(unsigned char **out, cudaStream_t st, bool *capturing) {
    *capturing = false;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if ((e = cudaStreamIsCapturing(st, &cs)) != cudaSuccess) return e;
        if (cs != cudaStreamCaptureStatusNone) {
            *capturing = true;
            return cudaErrorStreamCaptureUnsupported;
        }
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Models {
    double d[FENGINE_NOALLOC_MAX_STREAMS][4];   // delay, rate, phase, phase_rate
    long long t_ref[FENGINE_NOALLOC_MAX_STREAMS];
};

// Writes one delay segment per stream into the scratch (so the shared delay
// table kernel can read it), zeroes the clamp flag, and fills the twiddle
// tables exp(-2 pi i k1 t2 / N) and exp(-2 pi i q / N2) from exactly reduced
// integer phases in FP64.
__global__ void k_noalloc_setup(Models m, int n_streams, fe::DelaySeg *seg, int *nseg, int *err,
                                float2 *tw1, float2 *tw2, int N, int N1, int N2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_streams) {
        fe::DelaySeg s;
        s.t_apply = -(1LL << 62);
        s.t_ref = m.t_ref[i];
        s.d0 = m.d[i][0];
        s.rate = m.d[i][1];
        s.phi0 = m.d[i][2];
        s.phi_rate = m.d[i][3];
        seg[(long long)i * fe::kMaxSeg] = s;
        nseg[i] = 1;
    }
    if (i == 0) *err = 0;
    const int n1 = (N1 / 2 + 1) * N2;
    if (i < n1) {
        const long long k1 = i / N2, t2 = i % N2;
        const long long r = (k1 * t2) % N;
        double sn, cs;
        sincospi(-2.0 * (double)r / (double)N, &sn, &cs);
        tw1[i] = make_float2((float)cs, (float)sn);
    }
    if (i < N2) {
        double sn, cs;
        sincospi(-2.0 * (double)i / (double)N2, &sn, &cs);
        tw2[i] = make_float2((float)cs, (float)sn);
    }
}

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" {

fengine_status fengine_process_chunk_noalloc(const fengine_noalloc_args *a, const uint8_t *d_history,
                                             const uint8_t *d_packed, const float *d_weights,
                                             const float *d_gains, const double *delay_models,
                                             int8_t *d_out, void *cuda_stream) {
    if (!a || !d_history || !d_packed || !d_weights || !d_gains || !delay_models || !d_out) return FENGINE_EINVAL;
    if (a->n_antennas < 1 || a->n_antennas > FENGINE_NOALLOC_MAX_STREAMS / 2) return FENGINE_EINVAL;
    const int n = a->n_channels, T = a->n_taps, nant = a->n_antennas, ns = 2 * nant;
    if (!is_pow2(n) || n < 16 || n > 32768) return FENGINE_EINVAL;
    if (!(T == 1 || T == 2 || T == 4 || T == 8 || T == 16 || T == 32)) return FENGINE_EINVAL;
    const long long N = 2LL * n;
    if (a->chunk_samples <= 0 || a->chunk_samples % N || a->first_sample % N) return FENGINE_EINVAL;
    if (a->max_delay_samples < 0 || a->max_delay_samples > (1LL << 30)) return FENGINE_EINVAL;
    const long long M = a->chunk_samples / N;
    const int S = a->spectra_per_heap == 0 ? (int)(M < 256 ? M : 256) : a->spectra_per_heap;
    if (S < 1 || S > M || M > (1LL << 30)) return FENGINE_EINVAL;
    if (a->chunk_samples + N * T + a->max_delay_samples + 16 >= (1LL << 31)) return FENGINE_EINVAL;
    if (((uintptr_t)d_history & 3) || ((uintptr_t)d_packed & 3) || ((uintptr_t)d_out & 3)) return FENGINE_EINVAL;
    // every model finite, t_ref an integer timestamp (converted once, used
    // by both the range check below and the device's delay table)
    Models m;
    for (int s = 0; s < ns; s++) {
        for (int j = 0; j < 5; j++)
            if (!std::isfinite(delay_models[5 * s + j])) return FENGINE_EINVAL;
        const double tr = delay_models[5 * s + 4];
        if (tr != std::floor(tr) || std::fabs(tr) > 9.0e18) return FENGINE_EINVAL;
        m.t_ref[s] = (long long)tr;
        for (int j = 0; j < 4; j++) m.d[s][j] = delay_models[5 * s + j];
    }
    for (int s = 0; s < ns; s++) {
        // the one delay model of each stream must keep c in [0, D] over the call
        const double dt0 = (double)(N * (a->first_sample / N - (T - 1)) - m.t_ref[s]);
        const double dt1 = dt0 + (double)(N * (M - 1));
        for (double dt : {dt0, dt1}) {
            volatile double prod = delay_models[5 * s + 1] * dt;
            const double d = delay_models[5 * s + 0] + prod;
            const double c = __builtin_floor(d + 0.5);
            if (!(c >= 0.0 && c <= (double)a->max_delay_samples)) return FENGINE_EDELAY;
        }
    }

    const int N1 = (int)(N / 1024 > 8 ? N / 1024 : 8), N2 = (int)(N / N1);
    long long H = N * (T - 1) + a->max_delay_samples;
    H = (H + 15) / 16 * 16;

    // scratch layout; the slab of the intermediate takes what is left
    size_t off = 0;
    const size_t o_ctab = off;   off = align256(off + sizeof(int) * ns * M);
    const size_t o_ftab = off;   off = align256(off + sizeof(float2) * ns * M);
    const size_t o_tw1 = off;    off = align256(off + sizeof(float2) * (N1 / 2 + 1) * N2);
    const size_t o_tw2 = off;    off = align256(off + sizeof(float2) * N2);
    const size_t o_seg = off;    off = align256(off + sizeof(fe::DelaySeg) * fe::kMaxSeg * ns);
    const size_t o_nseg = off;   off = align256(off + sizeof(int) * ns);
    const size_t o_err = off;    off = align256(off + sizeof(int));
    const size_t o_A = off;
    if (off >= kScratchBytes) return FENGINE_EINVAL;
    const size_t per_spec = (size_t)ns * (N1 / 2 + 1) * N2 * sizeof(float2);
    long long SL = (long long)((kScratchBytes - o_A) / per_spec) / 32 * 32;
    if (SL > (M + 31) / 32 * 32) SL = (M + 31) / 32 * 32;
    if (SL < 32) return FENGINE_EINVAL;   // this shape needs more than the fixed scratch

    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char *base = nullptr;
    bool capturing = false;
    if (scratch_address(&base, st, &capturing) != cudaSuccess) return capturing ? FENGINE_EINVAL : FENGINE_ECUDA;
    const int setup_n = (N1 / 2 + 1) * N2 > ns ? (N1 / 2 + 1) * N2 : ns;
    k_noalloc_setup<<<(setup_n + 255) / 256, 256, 0, st>>>(
        m, ns, reinterpret_cast<fe::DelaySeg *>(base + o_seg), reinterpret_cast<int *>(base + o_nseg),
        reinterpret_cast<int *>(base + o_err), reinterpret_cast<float2 *>(base + o_tw1),
        reinterpret_cast<float2 *>(base + o_tw2), (int)N, N1, N2);
    if (cudaGetLastError() != cudaSuccess) return FENGINE_ECUDA;

    const long long m0 = a->first_sample / N - (T - 1);
    fe::DelayTableParams dp{};
    dp.seg = reinterpret_cast<const fe::DelaySeg *>(base + o_seg);
    dp.nseg = reinterpret_cast<const int *>(base + o_nseg);
    dp.n_streams = ns;
    dp.N = (int)N;
    dp.m0 = m0;
    dp.M = (int)M;
    dp.min_delay = 0;
    dp.max_delay = (int)a->max_delay_samples;
    dp.ctab = reinterpret_cast<int *>(base + o_ctab);
    dp.ftab = reinterpret_cast<float2 *>(base + o_ftab);
    dp.err = reinterpret_cast<int *>(base + o_err);
    if (fe::launch_delay_table(dp, st) != cudaSuccess) return FENGINE_ECUDA;

    fe::Phase1Params p1{};
    p1.chunk = d_packed;
    p1.hist = d_history;
    p1.chunk_bytes = a->chunk_samples / 4 * 5;
    p1.hist_bytes = H / 4 * 5;
    p1.H = H;
    p1.L = a->chunk_samples;
    p1.N = (int)N;
    p1.N2 = N2;
    p1.W = fe::phase1_W(N1, N2);
    p1.C = N1 * p1.W;
    p1.M = (int)M;
    p1.m0 = m0;
    p1.t_in = a->first_sample;
    p1.w = d_weights;
    p1.tw1 = reinterpret_cast<const float2 *>(base + o_tw1);
    p1.ctab = dp.ctab;
    p1.window_tap = nullptr;
    p1.a_spectra = (int)SL;
    p1.A = reinterpret_cast<float2 *>(base + o_A);

    fe::Phase2Params p2{};
    p2.A = p1.A;
    p2.tw2 = reinterpret_cast<const float2 *>(base + o_tw2);
    p2.gains = reinterpret_cast<const float2 *>(d_gains);   // one gain set per stream
    p2.gsel = nullptr;
    p2.n_gsets_max = 1;
    p2.tc_unscale = 1.0f;
    p2.ftab = dp.ftab;
    p2.N = (int)N;
    p2.N1 = N1;
    p2.M = (int)M;
    p2.S = S;
    p2.R2 = fe::phase2_R2(N2);
    p2.out = d_out;
    p2.prequant = nullptr;
    p2.a_spectra = (int)SL;

    // one intermediate buffer: slabs run back to back on the caller's stream
    for (long long qb = 0; qb < M; qb += SL) {
        const int qc = (int)((M - qb) < SL ? (M - qb) : SL);
        p1.q_begin = p2.q_begin = (int)qb;
        p1.q_count = p2.q_count = qc;
        if (fe::launch_phase1(T, N1, p1, ns, st) != cudaSuccess) return FENGINE_ECUDA;
        if (fe::launch_phase2(N2, p2, nant, st) != cudaSuccess) return FENGINE_ECUDA;
    }
    return FENGINE_OK;
}

}  // extern "C"
