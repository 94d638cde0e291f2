// Host side of libfengine: plan state, argument checking and the launch
// sequence of one fengine_process_chunk call. See include/fengine.h for the
// contract of every entry point.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/fengine.h"
#include "fe_device.cuh"
#include "fe_internal.cuh"

using fe::DelaySeg;

namespace {

thread_local std::string g_last_error;

fengine_status fail(fengine_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

fengine_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return FENGINE_ECUDA;
}

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

// Same arithmetic as the device delay table (no contraction: the build
// passes -ffp-contract=off to the host compiler), so c agrees exactly.
long long coarse_delay(const DelaySeg &s, long long t0) {
    const double dt = (double)(t0 - s.t_ref);
    volatile double prod = s.rate * dt;
    const double d = s.d0 + prod;
    return (long long)std::floor(d + 0.5);
}

}  // namespace

struct fengine_plan_s {
    int device = 0;
    int n_ant = 0, n_streams = 0, n = 0, N = 0, T = 0, S = 0, M = 0, N1 = 0, N2 = 0, W = 0, C = 0, R2 = 0;
    int precision = 0;
    int a_elem = 8;                 // bytes per intermediate element
    long long L = 0, D = 0, Dmin = 0, H = 0, chunk_bytes = 0, hist_bytes = 0;
    int E = 0;                      // emission lag (spectra) that makes room for negative delays
    // lost data (Sec. 3.7): received flags of the history heaps, ping-pong with d_hist
    bool lost_ok = false;           // chunk_samples a multiple of the 4096-sample heap
    bool hv_known = true;           // the device history flags describe the current history
    int HV = 0;
    unsigned char *d_hvalid[2] = {nullptr, nullptr};
    // device state
    float *d_w = nullptr;
    float2 *d_tw1 = nullptr, *d_tw2 = nullptr, *d_gains = nullptr, *d_ftab = nullptr, *d_A = nullptr;
    long long *d_gtap = nullptr;    // [stream][kMaxGainSeg] t_apply of each gain set
    int *d_ngs = nullptr;           // [stream] gain sets in use
    unsigned char *d_gsel = nullptr;   // [stream][M] gain set of each spectrum
    unsigned char *d_cchg = nullptr;   // [stream][M] coarse delay changes at this spectrum
    // reduced-precision forms: tensor-core phase-1 operand blocks and per-column epilogue scales
    uint16_t *d_bmat = nullptr;
    float *d_oscale = nullptr;
    uint16_t *d_cols = nullptr;     // FP16 column sequences of history + chunk (per call)
    int cols_rtp = 0;
    float tc_unscale = 1.0f;        // inverse of the FP16 intermediate's scale
    bool tc1 = false;               // phase 1 on tensor cores
    int tc_splits = 1;              // SMs of the device (the tensor-core phase 1 runs one wave)
    uint8_t *d_hist[2] = {nullptr, nullptr};
    int cur = 0;
    DelaySeg *d_seg = nullptr;
    int *d_nseg = nullptr, *d_ctab = nullptr, *d_err = nullptr;
    size_t device_bytes = 0, scratch_bytes = 0;
    // host mirrors, pinned staging
    std::vector<std::vector<DelaySeg>> segs;
    struct GainSet {
        long long t_apply;
        std::vector<float2> g;
    };
    std::vector<std::vector<GainSet>> gsets;   // [stream], sorted by t_apply
    bool delay_dirty = true, gains_dirty = true;
    DelaySeg *h_seg = nullptr;
    int *h_nseg = nullptr;
    float2 *h_gains = nullptr;      // [stream][kMaxGainSeg][n]
    long long *h_gtap = nullptr;
    int *h_ngs = nullptr;
    cudaEvent_t staged = nullptr;
    bool staged_pending = false;
    bool started = false;
    long long next_sample = 0;
    // slab pipeline: phase 1 of slab s+1 overlaps phase 2 of slab s on two
    // internal streams; the intermediate of a slab stays in L2
    int SL = 0, n_slabs = 0;
    cudaStream_t sp[3] = {nullptr, nullptr, nullptr};   // phase 1, phase 2, column unpack
    cudaEvent_t ev_fork = nullptr, ev_p1[2] = {nullptr, nullptr}, ev_p2[2] = {nullptr, nullptr};
    cudaEvent_t ev_u[2] = {nullptr, nullptr};            // column unpack of a slab done
    // optional per-stage timing: (stage, start, end) event records
    bool profiling = false;
    std::vector<cudaEvent_t> prof_events;
    size_t prof_used = 0;
    std::vector<int> prof_stage;
    int prof_calls = 0;
};

namespace {

template <typename P>
cudaError_t dalloc(fengine_plan_s *pl, P **ptr, size_t bytes) {
    cudaError_t e = cudaMalloc((void **)ptr, bytes);
    if (e == cudaSuccess) pl->device_bytes += bytes;
    return e;
}

void release(fengine_plan_s *pl) {
    if (!pl) return;
    cudaFree(pl->d_w);
    cudaFree(pl->d_tw1);
    cudaFree(pl->d_tw2);
    cudaFree(pl->d_bmat);
    cudaFree(pl->d_oscale);
    cudaFree(pl->d_cols);
    cudaFree(pl->d_gains);
    cudaFree(pl->d_ftab);
    cudaFree(pl->d_A);
    cudaFree(pl->d_hist[0]);
    cudaFree(pl->d_hist[1]);
    cudaFree(pl->d_seg);
    cudaFree(pl->d_gtap);
    cudaFree(pl->d_ngs);
    cudaFree(pl->d_gsel);
    cudaFree(pl->d_cchg);
    cudaFree(pl->d_hvalid[0]);
    cudaFree(pl->d_hvalid[1]);
    cudaFree(pl->d_nseg);
    cudaFree(pl->d_ctab);
    cudaFree(pl->d_err);
    cudaFreeHost(pl->h_seg);
    cudaFreeHost(pl->h_nseg);
    cudaFreeHost(pl->h_gains);
    cudaFreeHost(pl->h_gtap);
    cudaFreeHost(pl->h_ngs);
    if (pl->staged) cudaEventDestroy(pl->staged);
    for (cudaEvent_t ev : pl->prof_events) cudaEventDestroy(ev);
    for (int i = 0; i < 2; i++) {
        if (pl->ev_p1[i]) cudaEventDestroy(pl->ev_p1[i]);
        if (pl->ev_p2[i]) cudaEventDestroy(pl->ev_p2[i]);
        if (pl->sp[i]) cudaStreamDestroy(pl->sp[i]);
        if (pl->ev_u[i]) cudaEventDestroy(pl->ev_u[i]);
    }
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    if (pl->sp[2]) cudaStreamDestroy(pl->sp[2]);
    delete pl;
}

void default_weights_fp64(int N, int T, std::vector<double> &w) {
    const long long Mw = (long long)N * T;
    w.resize(Mw);
    double ss = 0.0;
    for (long long u = 0; u < Mw; u++) {
        const double x = ((double)u + 0.5 - (double)Mw / 2.0) / (double)N;
        const double sinc = x == 0.0 ? 1.0 : std::sin(M_PI * x) / (M_PI * x);
        const double h = std::sin(M_PI * ((double)u + 0.5) / (double)Mw);
        w[u] = h * h * sinc;
        ss += w[u] * w[u];
    }
    const double sc = 1.0 / std::sqrt(ss);
    for (auto &v : w) v *= sc;
}

// exp(-2 pi i a / b) with a reduced exactly modulo b first.
float2 unit_root(long long a, long long b) {
    const long long r = ((a % b) + b) % b;
    const double ang = -2.0 * M_PI * (double)r / (double)b;
    return make_float2((float)std::cos(ang), (float)std::sin(ang));
}

// Next profiling event (created on first use, reused across accumulations).
cudaEvent_t prof_event(fengine_plan_s *pl) {
    if (pl->prof_used == pl->prof_events.size()) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
        pl->prof_events.push_back(ev);
    }
    return pl->prof_events[pl->prof_used++];
}

// Profiling: an event pair around one launch of `stage` on stream st.
void prof_begin(fengine_plan_s *pl, int stage, cudaStream_t st) {
    if (!pl->profiling) return;
    cudaEvent_t ev = prof_event(pl);
    if (!ev) return;
    pl->prof_stage.push_back(stage);
    cudaEventRecord(ev, st);
}

void prof_end(fengine_plan_s *pl, cudaStream_t st) {
    if (!pl->profiling || pl->prof_used == 0 || pl->prof_used % 2 == 0) return;
    cudaEvent_t ev = prof_event(pl);
    if (ev) cudaEventRecord(ev, st);
}

}  // namespace

extern "C" {

const char *fengine_strerror(fengine_status st) {
    switch (st) {
        case FENGINE_OK: return "ok";
        case FENGINE_EINVAL: return "invalid argument";
        case FENGINE_ENOMEM: return "out of memory";
        case FENGINE_ECUDA: return "CUDA error";
        case FENGINE_ESEQ: return "chunk timestamp not contiguous with the stream";
        case FENGINE_EBUSY: return "busy: no slot or over budget";
        case FENGINE_ETIMEOUT: return "device wait timed out";
        case FENGINE_EUNSUPPORTED: return "unsupported in this build";
        case FENGINE_EDELAY: return "coarse delay outside [min_delay_samples, max_delay_samples]";
        case FENGINE_EIO: return "host file could not be written";
    }
    return "unknown status";
}

const char *fengine_last_error(void) { return g_last_error.c_str(); }

int32_t fengine_abi_version(void) { return FENGINE_ABI_VERSION; }

int32_t fengine_quantise(float x) { return fe::quant8(x); }

fengine_status fengine_default_weights(int32_t n_channels, int32_t n_taps, float *out) {
    if (!out || !is_pow2(n_channels) || n_taps < 1 || n_taps > 1024)
        return fail(FENGINE_EINVAL, "fengine_default_weights: bad arguments");
    std::vector<double> w;
    default_weights_fp64(2 * n_channels, n_taps, w);
    for (size_t i = 0; i < w.size(); i++) out[i] = (float)w[i];
    return FENGINE_OK;
}

fengine_status fengine_plan_create(const fengine_config *cfg, fengine_plan_t *out) {
    if (!cfg || !out) return fail(FENGINE_EINVAL, "fengine_plan_create: null argument");
    *out = nullptr;
    const int n = cfg->n_channels, T = cfg->n_taps;
    if (cfg->n_antennas < 1) return fail(FENGINE_EINVAL, "n_antennas must be >= 1");
    if (cfg->n_pols != 2) return fail(FENGINE_EINVAL, "n_pols must be 2");
    if (!is_pow2(n) || n < 16 || n > 32768) return fail(FENGINE_EINVAL, "n_channels must be a power of two in [16, 32768]");
    if (!(T == 1 || T == 2 || T == 4 || T == 8 || T == 16 || T == 32))
        return fail(FENGINE_EINVAL, "n_taps must be one of 1, 2, 4, 8, 16, 32");
    const long long N = 2LL * n;
    if (cfg->chunk_samples <= 0 || cfg->chunk_samples % N)
        return fail(FENGINE_EINVAL, "chunk_samples must be a positive multiple of 2 n_channels");
    const long long M = cfg->chunk_samples / N;
    if (M > (1LL << 30)) return fail(FENGINE_EINVAL, "chunk too long");
    // the kernels index a stream's history + chunk with 32-bit sample offsets
    if (cfg->chunk_samples + 2LL * n * T + cfg->max_delay_samples - 2 * cfg->min_delay_samples + 2LL * n + 16 >=
        (1LL << 31))
        return fail(FENGINE_EINVAL, "history + chunk must stay below 2^31 samples per stream");
    if (cfg->max_delay_samples < 0 || cfg->max_delay_samples > (1LL << 30))
        return fail(FENGINE_EINVAL, "max_delay_samples out of range");
    if (cfg->min_delay_samples > 0 || cfg->min_delay_samples < -(1LL << 30))
        return fail(FENGINE_EINVAL, "min_delay_samples must lie in [-2^30, 0]");
    int S = cfg->spectra_per_heap;
    if (S == 0) S = (int)(M < 256 ? M : 256);
    if (S < 1 || S > M) return fail(FENGINE_EINVAL, "spectra_per_heap must be in [1, L/2n]");
    if (cfg->precision != FENGINE_FP32 && cfg->precision != FENGINE_TC_FP16 && cfg->precision != FENGINE_TC_BF16)
        return fail(FENGINE_EINVAL, "unknown precision");
    // four-step split. FP32 form: N1 from the config or the built-in
    // max(8, N / 1024); its phase-1 tiles exist for N1 = 8 (W = min(64, N2))
    // and N1 = 16, 32, 64 (W = 512 / N1 <= N2), the phase-2 kernels for
    // N2 <= 1024. Tensor-core forms: N1 = 8 R (fe::phase1_tc_R), the only split.
    const bool tc1 = cfg->precision != FENGINE_FP32;
    int N1 = cfg->fft_n1 ? cfg->fft_n1 : (int)(N / 1024 > 8 ? N / 1024 : 8);
    if (tc1) {
        if (!fe::phase1_tc_supported((int)N, T, cfg->precision))
            return fail(FENGINE_EUNSUPPORTED, "the tensor-core forms need 32 <= n_channels <= 32768 (and n_taps <= 16 "
                                              "for n_channels >= 32768, or for n_channels = 16384 in BF16)");
        const int n1_tc = 8 * fe::phase1_tc_R((int)N);
        if (cfg->fft_n1 && cfg->fft_n1 != n1_tc)
            return fail(FENGINE_EINVAL, "the tensor-core forms use fft_n1 = " + std::to_string(n1_tc) + " (or 0)");
        N1 = n1_tc;
    } else if (!(N1 == 8 || N1 == 16 || N1 == 32 || N1 == 64) || N % N1 || N / N1 > 1024 || N / N1 < 4 ||
               (N1 > 8 && N / N1 < 512 / N1)) {
        return fail(FENGINE_EINVAL, "fft_n1 must be 8, 16, 32 or 64 with N / fft_n1 <= 1024 (and >= 512 / fft_n1 "
                                    "for fft_n1 > 8)");
    }
    if (cfg->slab_spectra < 0 || cfg->slab_spectra % 32)
        return fail(FENGINE_EINVAL, "slab_spectra must be 0 or a positive multiple of 32");

    fengine_plan_s *pl = new (std::nothrow) fengine_plan_s();
    if (!pl) return fail(FENGINE_ENOMEM, "host allocation");
    cudaGetDevice(&pl->device);
    pl->n_ant = cfg->n_antennas;
    pl->n_streams = 2 * cfg->n_antennas;
    pl->n = n;
    pl->N = (int)N;
    pl->T = T;
    pl->S = S;
    pl->M = (int)M;
    pl->L = cfg->chunk_samples;
    pl->D = cfg->max_delay_samples;
    pl->Dmin = cfg->min_delay_samples;
    pl->E = (int)((-pl->Dmin + N - 1) / N);
    pl->precision = cfg->precision;
    pl->N1 = N1;
    pl->tc1 = tc1;
    pl->N2 = (int)(N / pl->N1);
    pl->W = fe::phase1_W(pl->N1, pl->N2);
    pl->C = pl->N1 * pl->W;
    pl->R2 = fe::phase2_R2(pl->N2);
    // the history reaches back to the earliest window start of the call's
    // first spectrum: N (T - 1 + E) + D samples before the chunk
    long long H = N * (T - 1 + pl->E) + pl->D;
    H = (H + 15) / 16 * 16;     // whole 5-byte groups, and 4-byte aligned rows of packed history
    pl->H = H;
    pl->lost_ok = pl->L % fe::kHeapSamples == 0;
    pl->HV = (int)((H + fe::kHeapSamples - 1) / fe::kHeapSamples) + 1;
    pl->hist_bytes = H / 4 * 5;
    pl->chunk_bytes = pl->L / 4 * 5;

    const int ns = pl->n_streams;
    cudaError_t e = cudaSuccess;
    // Slab of spectra per phase-1 / phase-2 launch pair: built-in, the
    // spectra whose FP32 intermediate (all streams) is about 256 MiB, a
    // multiple of 32 (both phases' tiles). Measured on GB300 (fengine_autotune),
    // launches over more spectra win over keeping a smaller intermediate in
    // L2: the grids then span several waves of CTAs.
    // intermediate element: FP32 (re, im), or FP16 (re, im) in the FP16 form
    pl->a_elem = pl->precision == FENGINE_TC_FP16 ? 4 : 8;
    const size_t per_spec = (size_t)ns * (pl->N1 / 2 + 1) * pl->N2 * pl->a_elem;
    long long SL = cfg->slab_spectra ? cfg->slab_spectra : (long long)((256u << 20) / per_spec) / 32 * 32;
    if (SL < 32) SL = 32;
    const long long M32 = (M + 31) / 32 * 32;
    if (SL > M32) SL = M32;
    pl->SL = (int)SL;
    pl->n_slabs = (int)((M + SL - 1) / SL);
    const int nbuf = pl->n_slabs > 1 ? 2 : 1;
    const size_t a_bytes = (size_t)nbuf * SL * per_spec;
    if ((e = dalloc(pl, &pl->d_w, sizeof(float) * N * T)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_tw1, sizeof(float2) * (pl->N1 / 2 + 1) * pl->N2)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_tw2, sizeof(float2) * pl->N2)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_gains, sizeof(float2) * ns * fe::kMaxGainSeg * n)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_gtap, sizeof(long long) * ns * fe::kMaxGainSeg)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_ngs, sizeof(int) * ns)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_gsel, (size_t)ns * M)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_cchg, (size_t)ns * M)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_hvalid[0], (size_t)ns * pl->HV)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_hvalid[1], (size_t)ns * pl->HV)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_ftab, sizeof(float2) * ns * M)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_ctab, sizeof(int) * ns * M)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_A, a_bytes)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_hist[0], (size_t)pl->hist_bytes * ns + 16)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_hist[1], (size_t)pl->hist_bytes * ns + 16)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_seg, sizeof(DelaySeg) * fe::kMaxSeg * ns)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_nseg, sizeof(int) * ns)) != cudaSuccess ||
        (e = dalloc(pl, &pl->d_err, sizeof(int))) != cudaSuccess) {
        release(pl);
        g_last_error = std::string("device allocation: ") + cudaGetErrorString(e);
        return FENGINE_ENOMEM;
    }
    pl->scratch_bytes = a_bytes + sizeof(float2) * ns * M + sizeof(int) * ns * M;
    if ((e = cudaMallocHost((void **)&pl->h_seg, sizeof(DelaySeg) * fe::kMaxSeg * ns)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&pl->h_nseg, sizeof(int) * ns)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&pl->h_gains, sizeof(float2) * ns * fe::kMaxGainSeg * n)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&pl->h_gtap, sizeof(long long) * ns * fe::kMaxGainSeg)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&pl->h_ngs, sizeof(int) * ns)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&pl->staged, cudaEventDisableTiming)) != cudaSuccess) {
        release(pl);
        g_last_error = std::string("pinned allocation: ") + cudaGetErrorString(e);
        return FENGINE_ENOMEM;
    }
    for (int i = 0; i < 2 && e == cudaSuccess; i++) {
        if ((e = cudaStreamCreateWithFlags(&pl->sp[i], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&pl->ev_p1[i], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&pl->ev_p2[i], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&pl->ev_u[i], cudaEventDisableTiming)) != cudaSuccess)
            break;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->sp[2], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        release(pl);
        return cuda_fail(e, "stream/event creation");
    }

    // weights (Eq. 1's w_{t,j} = w[t + N j])
    std::vector<float> w((size_t)N * T);
    if (cfg->weights) {
        std::memcpy(w.data(), cfg->weights, sizeof(float) * N * T);
    } else {
        std::vector<double> wd;
        default_weights_fp64((int)N, T, wd);
        for (size_t i = 0; i < wd.size(); i++) w[i] = (float)wd[i];
    }
    for (float v : w)
        if (!std::isfinite(v)) {
            release(pl);
            return fail(FENGINE_EINVAL, "weights must be finite");
        }
    // Reduced-precision forms: the tensor-core phase 1's operand blocks
    // (weights x DFT x twiddle, a power-of-two scale per output column) and
    // epilogue scales; the FP16 form stores the second-stage input scaled by
    // a power of two s_int that keeps it inside FP16, undone in phase 2.
    if (tc1) {
        std::vector<uint16_t> bmat;
        std::vector<float> osc;
        float s_int = 1.0f;
        fe::build_phase1_tc_tables((int)N, T, pl->precision, w.data(), bmat, osc, s_int);
        pl->tc_unscale = 1.0f / s_int;
        pl->cols_rtp = fe::unpack_cols_rows(pl->H, pl->L, pl->D, pl->Dmin, (int)N, T);
        // one FP16 plane; the BF16 form keeps hi and lo planes
        const size_t cols_bytes = sizeof(uint16_t) * (size_t)pl->n_streams * (N / 8) * pl->cols_rtp *
                                  (pl->precision == FENGINE_TC_BF16 ? 2 : 1);
        if ((e = dalloc(pl, &pl->d_cols, cols_bytes)) != cudaSuccess) {
            release(pl);
            g_last_error = std::string("device allocation: ") + cudaGetErrorString(e);
            return FENGINE_ENOMEM;
        }
        pl->scratch_bytes += cols_bytes;
        if ((e = dalloc(pl, &pl->d_bmat, sizeof(uint16_t) * bmat.size())) != cudaSuccess ||
            (e = dalloc(pl, &pl->d_oscale, sizeof(float) * osc.size())) != cudaSuccess ||
            (e = cudaMemcpy(pl->d_bmat, bmat.data(), sizeof(uint16_t) * bmat.size(), cudaMemcpyHostToDevice)) !=
                cudaSuccess ||
            (e = cudaMemcpy(pl->d_oscale, osc.data(), sizeof(float) * osc.size(), cudaMemcpyHostToDevice)) !=
                cudaSuccess) {
            release(pl);
            return cuda_fail(e, "tensor-core operand blocks");
        }
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // one wave of two CTAs per SM, each a contiguous, equal share of the
        // (column group, k1-slice, item) passes
        pl->tc_splits = sms > 0 ? sms : 148;
    }
    // twiddles, evaluated in FP64 with exact integer phase reduction
    std::vector<float2> tw1((size_t)(pl->N1 / 2 + 1) * pl->N2), tw2(pl->N2);
    for (int k1 = 0; k1 <= pl->N1 / 2; k1++)
        for (int t2 = 0; t2 < pl->N2; t2++) tw1[(size_t)k1 * pl->N2 + t2] = unit_root((long long)k1 * t2, N);
    for (int q = 0; q < pl->N2; q++) tw2[q] = unit_root(q, pl->N2);
    pl->segs.assign(ns, std::vector<DelaySeg>{DelaySeg{-(1LL << 62), 0, 0.0, 0.0, 0.0, 0.0}});
    pl->gsets.assign(ns, std::vector<fengine_plan_s::GainSet>{
                             fengine_plan_s::GainSet{-(1LL << 62), std::vector<float2>(n, make_float2(1.0f, 0.0f))}});

    if ((e = cudaMemcpy(pl->d_w, w.data(), sizeof(float) * N * T, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(pl->d_tw1, tw1.data(), sizeof(float2) * tw1.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(pl->d_tw2, tw2.data(), sizeof(float2) * tw2.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(pl->d_hist[0], 0, (size_t)pl->hist_bytes * ns + 16)) != cudaSuccess ||
        (e = cudaMemset(pl->d_hist[1], 0, (size_t)pl->hist_bytes * ns + 16)) != cudaSuccess ||
        (e = cudaMemset(pl->d_err, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(pl->d_hvalid[0], 0, (size_t)ns * pl->HV)) != cudaSuccess ||
        (e = cudaMemset(pl->d_hvalid[1], 0, (size_t)ns * pl->HV)) != cudaSuccess) {
        release(pl);
        return cuda_fail(e, "plan upload");
    }
    *out = pl;
    return FENGINE_OK;
}

fengine_status fengine_plan_destroy(fengine_plan_t pl) {
    if (!pl) return fail(FENGINE_EINVAL, "null plan");
    if (pl->staged_pending) cudaEventSynchronize(pl->staged);
    release(pl);
    return FENGINE_OK;
}

fengine_status fengine_get_info(fengine_plan_t pl, fengine_info *info) {
    if (!pl || !info) return fail(FENGINE_EINVAL, "null argument");
    info->n_channels = pl->n;
    info->n_taps = pl->T;
    info->n_antennas = pl->n_ant;
    info->spectra_per_heap = pl->S;
    info->fft_n1 = pl->N1;
    info->fft_n2 = pl->N2;
    info->spectra_per_chunk = pl->M;
    info->history_samples = pl->H;
    info->latency_spectra = pl->T - 1 + pl->E;
    info->out_bytes = (long long)pl->n_ant * pl->M * pl->n * 4;
    info->device_bytes = pl->device_bytes;
    info->scratch_bytes = pl->scratch_bytes;
    info->slab_spectra = pl->SL;
    info->slabs_per_chunk = pl->n_slabs;
    info->heaps_per_chunk = (pl->M + pl->S - 1) / pl->S;
    info->lost_data = pl->lost_ok ? 1 : 0;
    return FENGINE_OK;
}

fengine_status fengine_set_delay(fengine_plan_t pl, int32_t ant, int32_t pol, int64_t t_apply,
                                 int64_t t_ref, double delay, double delay_rate, double phase,
                                 double phase_rate) {
    if (!pl) return fail(FENGINE_EINVAL, "null plan");
    if (ant < 0 || ant >= pl->n_ant || pol < 0 || pol > 1) return fail(FENGINE_EINVAL, "bad stream index");
    if (!std::isfinite(delay) || !std::isfinite(delay_rate) || !std::isfinite(phase) || !std::isfinite(phase_rate))
        return fail(FENGINE_EINVAL, "delay model must be finite");
    auto &v = pl->segs[ant * 2 + pol];
    const DelaySeg s{(long long)t_apply, (long long)t_ref, delay, delay_rate, phase, phase_rate};
    size_t i = 0;
    while (i < v.size() && v[i].t_apply < t_apply) i++;
    if (i < v.size() && v[i].t_apply == t_apply) {
        v[i] = s;
    } else {
        if ((int)v.size() >= fe::kMaxSeg) return fail(FENGINE_EINVAL, "too many pending delay models");
        v.insert(v.begin() + i, s);
    }
    pl->delay_dirty = true;
    return FENGINE_OK;
}

fengine_status fengine_set_gains(fengine_plan_t pl, int32_t ant, int32_t pol, const float *g, int64_t t_apply) {
    if (!pl || !g) return fail(FENGINE_EINVAL, "null argument");
    if (ant < 0 || ant >= pl->n_ant || pol < 0 || pol > 1) return fail(FENGINE_EINVAL, "bad stream index");
    for (int k = 0; k < 2 * pl->n; k++)
        if (!std::isfinite(g[k])) return fail(FENGINE_EINVAL, "gains must be finite");
    auto &v = pl->gsets[ant * 2 + pol];
    fengine_plan_s::GainSet gs{(long long)t_apply, std::vector<float2>(pl->n)};
    for (int k = 0; k < pl->n; k++) gs.g[k] = make_float2(g[2 * k], g[2 * k + 1]);
    size_t i = 0;
    while (i < v.size() && v[i].t_apply < t_apply) i++;
    if (i < v.size() && v[i].t_apply == t_apply) {
        v[i] = std::move(gs);
    } else {
        if ((int)v.size() >= fe::kMaxGainSeg) return fail(FENGINE_EINVAL, "too many pending gain sets");
        v.insert(v.begin() + i, std::move(gs));
    }
    pl->gains_dirty = true;
    return FENGINE_OK;
}

fengine_status fengine_reset(fengine_plan_t pl) {
    if (!pl) return fail(FENGINE_EINVAL, "null plan");
    cudaError_t e;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "reset sync");
    const size_t hb = (size_t)pl->hist_bytes * pl->n_streams + 16;
    if ((e = cudaMemset(pl->d_hist[0], 0, hb)) != cudaSuccess ||
        (e = cudaMemset(pl->d_hist[1], 0, hb)) != cudaSuccess ||
        (e = cudaMemset(pl->d_hvalid[0], 0, (size_t)pl->n_streams * pl->HV)) != cudaSuccess ||
        (e = cudaMemset(pl->d_hvalid[1], 0, (size_t)pl->n_streams * pl->HV)) != cudaSuccess)
        return cuda_fail(e, "reset history");
    pl->hv_known = true;
    pl->started = false;
    return FENGINE_OK;
}

}  // extern "C"

namespace {

// fengine_process_chunk; with def (FP32 form), the phase-1 / phase-2 launches
// are returned in def instead of enqueued (the history tail is then updated
// first: it writes the history buffer this call does not read)
fengine_status process_impl(fengine_plan_t pl, void *cuda_stream, const uint8_t *d_packed, int64_t first_sample,
                            const uint8_t *d_valid, int8_t *d_out, uint8_t *d_heap_flags, float *d_prequant,
                            int32_t *d_window_tap, int64_t *first_spectrum, fe::DeferredCall *def) {
    if (!pl || !d_packed || !d_out) return fail(FENGINE_EINVAL, "null argument");
    if (((uintptr_t)d_packed & 3) || ((uintptr_t)d_out & 3))
        return fail(FENGINE_EINVAL, "d_packed and d_out must be 4-byte aligned");
    if (first_sample % pl->N) return fail(FENGINE_EINVAL, "first_sample must be a multiple of 2 n_channels");
    if (pl->started && first_sample != pl->next_sample)
        return fail(FENGINE_ESEQ, "expected first_sample " + std::to_string(pl->next_sample));
    const bool heap_aligned = pl->lost_ok && first_sample % fe::kHeapSamples == 0;
    if ((d_valid || d_heap_flags) && !heap_aligned)
        return fail(FENGINE_EINVAL, "lost-data flags need chunk_samples and first_sample to be multiples of the "
                                    "4096-sample heap");
    if (d_heap_flags && !pl->hv_known)
        return fail(FENGINE_EINVAL, "the history's received flags are unknown (a call was not heap-aligned); "
                                    "call fengine_reset first");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const long long m0 = first_sample / pl->N - (pl->T - 1) - pl->E;
    const long long t_first = (long long)pl->N * m0, t_last = (long long)pl->N * (m0 + pl->M - 1);

    // Drop delay models that no spectrum from this call on can use, then
    // check that every coarse delay of this call lies in [0, D]. A segment is
    // linear, so its extreme delays over a spectrum range are at the ends.
    for (int s = 0; s < pl->n_streams; s++) {
        auto &v = pl->segs[s];
        while (v.size() > 1 && v[1].t_apply <= t_first) {
            v.erase(v.begin());
            pl->delay_dirty = true;
        }
        for (size_t i = 0; i < v.size(); i++) {
            long long lo = i == 0 ? t_first : (v[i].t_apply > t_first ? v[i].t_apply : t_first);
            long long hi = i + 1 < v.size() ? v[i + 1].t_apply - 1 : t_last;
            if (hi > t_last) hi = t_last;
            // round lo up to a spectrum timestamp
            lo = (lo + pl->N - 1) / pl->N * pl->N;
            if (lo < t_first) lo = t_first;
            if (lo > hi) continue;
            hi = hi / pl->N * pl->N;
            if (hi < lo) continue;
            const long long c0 = coarse_delay(v[i], lo), c1 = coarse_delay(v[i], hi);
            if (c0 < pl->Dmin || c1 < pl->Dmin || c0 > pl->D || c1 > pl->D)
                return fail(FENGINE_EDELAY, "stream " + std::to_string(s) + ": coarse delay " +
                                                std::to_string(c0 < pl->Dmin || c0 > pl->D ? c0 : c1) + " outside [" +
                                                std::to_string(pl->Dmin) + ", " + std::to_string(pl->D) + "]");
        }
    }

    for (int s = 0; s < pl->n_streams; s++) {
        auto &v = pl->gsets[s];
        while (v.size() > 1 && v[1].t_apply <= t_first) {
            v.erase(v.begin());
            pl->gains_dirty = true;
        }
    }

    cudaError_t e;
    if (pl->delay_dirty || pl->gains_dirty) {
        if (pl->staged_pending) {
            if ((e = cudaEventSynchronize(pl->staged)) != cudaSuccess) return cuda_fail(e, "staging wait");
            pl->staged_pending = false;
        }
        if (pl->delay_dirty) {
            for (int s = 0; s < pl->n_streams; s++) {
                pl->h_nseg[s] = (int)pl->segs[s].size();
                for (size_t i = 0; i < pl->segs[s].size(); i++) pl->h_seg[(size_t)s * fe::kMaxSeg + i] = pl->segs[s][i];
            }
            if ((e = cudaMemcpyAsync(pl->d_seg, pl->h_seg, sizeof(DelaySeg) * fe::kMaxSeg * pl->n_streams,
                                     cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(pl->d_nseg, pl->h_nseg, sizeof(int) * pl->n_streams,
                                     cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return cuda_fail(e, "delay upload");
        }
        if (pl->gains_dirty) {
            const int G = fe::kMaxGainSeg;
            for (int s = 0; s < pl->n_streams; s++) {
                const auto &v = pl->gsets[s];
                pl->h_ngs[s] = (int)v.size();
                for (size_t i = 0; i < v.size(); i++) {
                    pl->h_gtap[(size_t)s * G + i] = v[i].t_apply;
                    std::memcpy(pl->h_gains + ((size_t)s * G + i) * pl->n, v[i].g.data(), sizeof(float2) * pl->n);
                }
            }
            if ((e = cudaMemcpyAsync(pl->d_gains, pl->h_gains, sizeof(float2) * pl->n_streams * G * pl->n,
                                     cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(pl->d_gtap, pl->h_gtap, sizeof(long long) * pl->n_streams * G,
                                     cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(pl->d_ngs, pl->h_ngs, sizeof(int) * pl->n_streams, cudaMemcpyHostToDevice,
                                     st)) != cudaSuccess)
                return cuda_fail(e, "gain upload");
        }
        if ((e = cudaEventRecord(pl->staged, st)) != cudaSuccess) return cuda_fail(e, "staging event");
        pl->staged_pending = true;
        pl->delay_dirty = pl->gains_dirty = false;
    }

    fe::DelayTableParams dp{};
    dp.seg = pl->d_seg;
    dp.nseg = pl->d_nseg;
    dp.n_streams = pl->n_streams;
    dp.N = pl->N;
    dp.m0 = m0;
    dp.M = pl->M;
    dp.min_delay = (int)pl->Dmin;
    dp.max_delay = (int)pl->D;
    dp.ctab = pl->d_ctab;
    dp.ftab = pl->d_ftab;
    dp.err = pl->d_err;
    dp.g_tapply = pl->d_gtap;
    dp.n_gsets = pl->d_ngs;
    dp.gsel = pl->d_gsel;
    dp.cchg = pl->d_cchg;
    prof_begin(pl, 0, st);
    if ((e = fe::launch_delay_table(dp, st)) != cudaSuccess) return cuda_fail(e, "delay table launch");
    prof_end(pl, st);

    // Lost data (Sec. 3.7): heap flags of this call and the history heaps'
    // received flags for the next one (kept whenever the call is heap-aligned)
    if (heap_aligned) {
        fe::LostDataParams lp{};
        lp.valid = d_valid;
        lp.hv_in = pl->d_hvalid[pl->cur];
        lp.hv_out = pl->d_hvalid[1 - pl->cur];
        lp.HV = pl->HV;
        lp.heap0 = first_sample / fe::kHeapSamples;
        lp.chunk_heaps = (int)(pl->L / fe::kHeapSamples);
        lp.ctab = pl->d_ctab;
        lp.n_ant = pl->n_ant;
        lp.N = pl->N;
        lp.T = pl->T;
        lp.M = pl->M;
        lp.S = pl->S;
        lp.m0 = m0;
        lp.heap_flags = d_heap_flags;
        if ((e = fe::launch_lost_data(lp, st)) != cudaSuccess) return cuda_fail(e, "lost-data launch");
    } else if (pl->lost_ok) {
        pl->hv_known = false;
    }

    fe::Phase1Params p1{};
    p1.chunk = d_packed;
    p1.hist = pl->d_hist[pl->cur];
    p1.chunk_bytes = pl->chunk_bytes;
    p1.hist_bytes = pl->hist_bytes;
    p1.H = pl->H;
    p1.L = pl->L;
    p1.N = pl->N;
    p1.N2 = pl->N2;
    p1.W = pl->W;
    p1.C = pl->C;
    p1.M = pl->M;
    p1.m0 = m0;
    p1.t_in = first_sample;
    p1.w = pl->d_w;
    p1.tw1 = pl->d_tw1;
    p1.ctab = pl->d_ctab;
    p1.window_tap = d_window_tap;
    p1.a_spectra = pl->SL;
    p1.half_out = 0;

    fe::Phase2Params p2{};
    p2.tw2 = pl->d_tw2;
    p2.gains = pl->d_gains;
    p2.gsel = pl->d_gsel;
    p2.n_gsets_max = fe::kMaxGainSeg;
    p2.ftab = pl->d_ftab;
    p2.N = pl->N;
    p2.N1 = pl->N1;
    p2.M = pl->M;
    p2.S = pl->S;
    p2.R2 = pl->R2;
    p2.out = d_out;
    p2.prequant = reinterpret_cast<float2 *>(d_prequant);
    p2.a_spectra = pl->SL;
    p2.half_in = pl->precision == FENGINE_TC_FP16;   // every form's second stage runs on CUDA cores
    p2.tc_unscale = pl->tc_unscale;

    fe::Phase1TcParams pt{};
    // with several slabs the column unpack goes slab by slab on its own
    // internal stream, ahead of the phase 1 that needs it: the unpack of slab
    // s + 1 runs on the SMs beside the tensor-core phase 1 of slab s (one
    // unpack CTA fits next to it in shared memory and registers)
    const bool split_unpack = pl->tc1 && pl->n_slabs > 1 && (pl->N / 8) % 64 == 0 && !def;
    fe::UnpackColsParams up{};
    if (pl->tc1) {
        // unpack history + chunk into FP16 column sequences (row origin a
        // multiple of 8, so that 16-byte copies of a column stay aligned)
        const long long P = pl->N / 8;
        auto fdiv = [](long long a, long long b) { return a / b - ((a % b != 0 && a < 0) ? 1 : 0); };
        up.chunk = d_packed;
        up.hist = pl->d_hist[pl->cur];
        up.chunk_bytes = pl->chunk_bytes;
        up.hist_bytes = pl->hist_bytes;
        up.H = pl->H;
        up.L = pl->L;
        up.t_in = first_sample;
        up.P = (int)P;
        // pre-delayed by c0 in [Dmin, D]: rows from the history start shifted by Dmin
        up.rb = fdiv(fdiv(first_sample - pl->H + pl->Dmin, P), 8) * 8;
        up.RT = (int)(fdiv(first_sample + pl->L + pl->D, P) + 1 - up.rb);
        up.ctab = pl->d_ctab;
        up.M = pl->M;
        up.RTP = pl->cols_rtp;
        up.cols = pl->d_cols;
        up.n_streams = pl->n_streams;
        up.row_begin = 0;
        up.row_end = pl->cols_rtp;
        up.bf16 = pl->precision == FENGINE_TC_BF16 ? 1 : 0;
        up.plane_elems = (long long)pl->n_streams * (pl->N / 8) * pl->cols_rtp;
        if (!split_unpack) {
            prof_begin(pl, 4, st);
            if ((e = fe::launch_unpack_cols(up, st)) != cudaSuccess) return cuda_fail(e, "unpack launch");
            prof_end(pl, st);
        }
        pt.cols = pl->d_cols;
        pt.plane_elems = up.plane_elems;
        pt.rb = up.rb;
        pt.RTP = pl->cols_rtp;
    }
    pt.N = pl->N;
    pt.N2 = pl->N2;
    pt.M = pl->M;
    pt.m0 = m0;
    pt.a_spectra = pl->SL;
    pt.n_streams = pl->n_streams;
    pt.splits = pl->tc_splits;
    pt.bmat = pl->d_bmat;
    pt.oscale = pl->d_oscale;
    pt.ctab = pl->d_ctab;
    pt.cchg = pl->d_cchg;
    pt.window_tap = d_window_tap;
    pt.err = pl->d_err;

    if (def) {
        const size_t slab_elems = (size_t)pl->n_streams * pl->SL * (pl->N1 / 2 + 1) * pl->N2;
        if ((e = fe::launch_tail_update(pl->d_hist[pl->cur], d_packed, pl->d_hist[1 - pl->cur], pl->hist_bytes,
                                        pl->chunk_bytes, pl->n_streams, st)) != cudaSuccess)
            return cuda_fail(e, "tail launch");
        def->T = pl->T;
        def->N1 = pl->N1;
        def->N2 = pl->N2;
        def->n_streams = pl->n_streams;
        def->n_ant = pl->n_ant;
        def->p1.clear();
        def->p2.clear();
        for (int s = 0; s < pl->n_slabs; s++) {
            float2 *A = reinterpret_cast<float2 *>(reinterpret_cast<char *>(pl->d_A) +
                                                   (size_t)(s & 1) * slab_elems * pl->a_elem);
            const int qb = s * pl->SL;
            const int qc = (pl->M - qb) < pl->SL ? (pl->M - qb) : pl->SL;
            p1.A = A;
            p1.q_begin = qb;
            p1.q_count = qc;
            p2.A = A;
            p2.q_begin = qb;
            p2.q_count = qc;
            def->p1.push_back(p1);
            def->p2.push_back(p2);
        }
        pl->cur = 1 - pl->cur;
        pl->started = true;
        pl->next_sample = first_sample + pl->L;
        if (first_spectrum) *first_spectrum = m0;
        return FENGINE_OK;
    }

    // Slab pipeline: slab s uses intermediate buffer s % 2; phase 1 runs on
    // internal stream 0, phase 2 on internal stream 1, so phase 1 of slab
    // s + 1 overlaps phase 2 of slab s. Buffer reuse waits for phase 2 of
    // slab s - 2. Both internal streams fork from and join back into st.
    const size_t slab_elems = (size_t)pl->n_streams * pl->SL * (pl->N1 / 2 + 1) * pl->N2;
    if ((e = cudaEventRecord(pl->ev_fork, st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(pl->sp[0], pl->ev_fork, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(pl->sp[1], pl->ev_fork, 0)) != cudaSuccess ||
        (split_unpack && (e = cudaStreamWaitEvent(pl->sp[2], pl->ev_fork, 0)) != cudaSuccess))
        return cuda_fail(e, "slab fork");
    int unpacked = 0;   // column rows [0, unpacked) enqueued so far
    for (int s = 0; s < pl->n_slabs; s++) {
        const int b = s & 1;
        float2 *A = reinterpret_cast<float2 *>(reinterpret_cast<char *>(pl->d_A) + (size_t)b * slab_elems * pl->a_elem);
        const int qb = s * pl->SL;
        const int qc = (pl->M - qb) < pl->SL ? (pl->M - qb) : pl->SL;
        if (s >= 2 && (e = cudaStreamWaitEvent(pl->sp[0], pl->ev_p2[b], 0)) != cudaSuccess)
            return cuda_fail(e, "slab wait");
        if (split_unpack) {
            // the rows this slab's passes can read: the last tile's column
            // sequences (8 (127 + T') rows from row 8 (m0 + q0) - rb), moved by
            // at most (D - Dmin) / P + 1 rows for a pass whose delay differs from
            // the unpack's, plus the realigned copy's extra 16-byte chunk
            int hi = pl->cols_rtp;
            if (s + 1 < pl->n_slabs) {
                const long long q_last = qb + (long long)((qc - 1) / 128) * 128;
                const long long shift = (pl->D - pl->Dmin) / (pl->N / 8) + 2;
                const long long rows = 8 * (m0 + q_last) - up.rb + shift + 8LL * (127 + (pl->T < 2 ? 2 : pl->T)) + 16;
                const long long r64 = (rows + 63) / 64 * 64;
                hi = (int)(r64 < pl->cols_rtp ? r64 : pl->cols_rtp);
            }
            if (hi > unpacked) {
                up.row_begin = unpacked;
                up.row_end = hi;
                prof_begin(pl, 4, pl->sp[2]);
                if ((e = fe::launch_unpack_cols(up, pl->sp[2])) != cudaSuccess) return cuda_fail(e, "unpack launch");
                prof_end(pl, pl->sp[2]);
                unpacked = hi;
            }
            if ((e = cudaEventRecord(pl->ev_u[b], pl->sp[2])) != cudaSuccess ||
                (e = cudaStreamWaitEvent(pl->sp[0], pl->ev_u[b], 0)) != cudaSuccess)
                return cuda_fail(e, "unpack handoff");
        }
        p1.A = A;
        p1.q_begin = qb;
        p1.q_count = qc;
        pt.A = A;
        pt.q_begin = qb;
        pt.q_count = qc;
        prof_begin(pl, 1, pl->sp[0]);
        if ((e = pl->tc1 ? fe::launch_phase1_tc(pl->T, pl->precision, pt, pl->sp[0])
                         : fe::launch_phase1(pl->T, pl->N1, p1, pl->n_streams, pl->sp[0])) != cudaSuccess)
            return cuda_fail(e, "phase-1 launch");
        prof_end(pl, pl->sp[0]);
        if ((e = cudaEventRecord(pl->ev_p1[b], pl->sp[0])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(pl->sp[1], pl->ev_p1[b], 0)) != cudaSuccess)
            return cuda_fail(e, "slab handoff");
        p2.A = A;
        p2.q_begin = qb;
        p2.q_count = qc;
        prof_begin(pl, 2, pl->sp[1]);
        if ((e = fe::launch_phase2(pl->N2, p2, pl->n_ant, pl->sp[1])) != cudaSuccess)
            return cuda_fail(e, "phase-2 launch");
        prof_end(pl, pl->sp[1]);
        if ((e = cudaEventRecord(pl->ev_p2[b], pl->sp[1])) != cudaSuccess)
            return cuda_fail(e, "slab event");
    }
    // join: the last phase 2 follows every phase 1 (through the handoff events)
    if ((e = cudaStreamWaitEvent(st, pl->ev_p2[(pl->n_slabs - 1) & 1], 0)) != cudaSuccess)
        return cuda_fail(e, "slab join");

    prof_begin(pl, 3, st);
    if ((e = fe::launch_tail_update(pl->d_hist[pl->cur], d_packed, pl->d_hist[1 - pl->cur], pl->hist_bytes,
                                    pl->chunk_bytes, pl->n_streams, st)) != cudaSuccess)
        return cuda_fail(e, "tail launch");
    prof_end(pl, st);
    if (pl->profiling) pl->prof_calls++;
    pl->cur = 1 - pl->cur;
    pl->started = true;
    pl->next_sample = first_sample + pl->L;
    if (first_spectrum) *first_spectrum = m0;
    return FENGINE_OK;
}

}  // namespace

namespace fe {

bool plan_defers(fengine_plan_t pl) { return pl && !pl->tc1 && pl->precision == FENGINE_FP32; }

fengine_status process_chunk_deferred(fengine_plan_t pl, cudaStream_t st, const uint8_t *d_packed,
                                      int64_t first_sample, const uint8_t *d_valid, int8_t *d_out,
                                      uint8_t *d_heap_flags, int64_t *first_spectrum, DeferredCall *def,
                                      bool *deferred) {
    const bool fp32 = plan_defers(pl);
    *deferred = fp32;
    return process_impl(pl, (void *)st, d_packed, first_sample, d_valid, d_out, d_heap_flags, nullptr, nullptr,
                        first_spectrum, fp32 ? def : nullptr);
}

}  // namespace fe

extern "C" {

fengine_status fengine_process_chunk(fengine_plan_t pl, void *cuda_stream, const uint8_t *d_packed,
                                     int64_t first_sample, const uint8_t *d_valid, int8_t *d_out,
                                     uint8_t *d_heap_flags, float *d_prequant, int32_t *d_window_tap,
                                     int64_t *first_spectrum) {
    return process_impl(pl, cuda_stream, d_packed, first_sample, d_valid, d_out, d_heap_flags, d_prequant,
                        d_window_tap, first_spectrum, nullptr);
}

fengine_status fengine_device_status(fengine_plan_t pl) {
    if (!pl) return fail(FENGINE_EINVAL, "null plan");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "device status");
    int h = 0;
    if ((e = cudaMemcpy(&h, pl->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemset(pl->d_err, 0, sizeof(int))) != cudaSuccess)
        return cuda_fail(e, "device status");
    if (h == 2) return fail(FENGINE_ETIMEOUT, "a bounded wait of the tensor-core phase 1 gave up");
    if (h == 1) return fail(FENGINE_EDELAY, "a coarse delay was clamped on the device");
    return FENGINE_OK;
}

fengine_status fengine_set_profiling(fengine_plan_t pl, int32_t enable) {
    if (!pl) return fail(FENGINE_EINVAL, "null plan");
    pl->profiling = enable != 0;
    return FENGINE_OK;
}

fengine_status fengine_stage_times(fengine_plan_t pl, float *ms, int32_t *calls) {
    if (!pl || !ms || !calls) return fail(FENGINE_EINVAL, "null argument");
    for (int i = 0; i < 5; i++) ms[i] = 0.0f;
    const size_t n_rec = pl->prof_used / 2;
    for (size_t r = 0; r < n_rec; r++) {
        cudaEvent_t a = pl->prof_events[2 * r], b = pl->prof_events[2 * r + 1];
        cudaError_t e = cudaEventSynchronize(b);
        if (e != cudaSuccess) return cuda_fail(e, "stage timing");
        float t = 0.0f;
        if ((e = cudaEventElapsedTime(&t, a, b)) != cudaSuccess) return cuda_fail(e, "stage timing");
        const int stage = r < pl->prof_stage.size() ? pl->prof_stage[r] : 0;
        if (stage >= 0 && stage < 5) ms[stage] += t;
    }
    *calls = pl->prof_calls;
    pl->prof_used = 0;
    pl->prof_stage.clear();
    pl->prof_calls = 0;
    return FENGINE_OK;
}

}  // extern "C"
