/*
 * fengine.h -- C ABI of libfengine, a GB300 (sm_103a) F-engine channelizer.
 *
 * The library implements the data-parallel hot path of the F-engine in
 * B. Merry, "Efficient channelization on a Graphics Processing Unit"
 * (arXiv:2303.09886), Sec. 2.1: unpack 10-bit samples, coarse delay, PFB FIR
 * (Eq. 1), real-to-complex FFT, fine delay and bandpass gain, requantisation
 * to 8-bit Gaussian integers and the channel-major corner turn (Sec. 2.2,
 * Sec. 3.6), for the two polarisations of each antenna (Sec. 2.1, last
 * paragraph).
 *
 * Conventions shared by every entry point:
 *  - N = 2 n is the FFT length for n channels; spectrum m has timestamp
 *    t0 = N m (critically sampled PFB, consecutive spectra N samples apart).
 *  - Packed samples: sample i of a chunk occupies bits [10 i, 10 i + 10) of
 *    the byte stream, most significant bit first, two's complement
 *    (Sec. 2.2 fixes 10 bits per sample without padding; the bit order is
 *    this library's documented choice). A chunk of L samples is 5 L / 4 bytes.
 *  - Pointers named d_* are DEVICE pointers (cudaMalloc / PyTorch CUDA
 *    tensors); all other pointers are host pointers. The caller owns every
 *    buffer it passes; the plan owns its own state (weights, history tails,
 *    delay models, gains, twiddles, scratch) and frees it in
 *    fengine_plan_destroy.
 *  - cuda_stream arguments are cudaStream_t handles passed as void*; NULL is
 *    the legacy default stream. Work is enqueued asynchronously; a device
 *    fault surfaces as FENGINE_ECUDA from a later call.
 *  - Errors are reported only through fengine_status; nothing aborts, traps
 *    the device or throws across the ABI. fengine_last_error() returns a
 *    thread-local message for the last failure on the calling thread.
 */
#ifndef FENGINE_H
#define FENGINE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FENGINE_ABI_VERSION 3
#define FENGINE_MAX_DELAY_SEGMENTS 16
#define FENGINE_MAX_GAIN_SETS 4        /* gain sets per stream pending at once */
#define FENGINE_HEAP_SAMPLES 4096      /* samples per digitiser heap (Sec. 2.2) */

typedef enum {
    FENGINE_OK = 0,
    FENGINE_EINVAL = 1,       /* invalid argument or configuration */
    FENGINE_ENOMEM = 2,       /* device or host allocation failed */
    FENGINE_ECUDA = 3,        /* CUDA runtime error (see fengine_last_error) */
    FENGINE_ESEQ = 4,         /* chunk timestamp not contiguous with the stream */
    FENGINE_EBUSY = 5,        /* no free slot / over the memory budget */
    FENGINE_ETIMEOUT = 6,     /* a bounded device-side wait gave up */
    FENGINE_EUNSUPPORTED = 7, /* valid request this build does not implement */
    FENGINE_EDELAY = 8,       /* a coarse delay of this call leaves [min_delay, max_delay] */
    FENGINE_EIO = 9           /* a host file could not be written */
} fengine_status;

/* Precision forms. The reduced-precision forms run the unpack, the coarse
 * delay, the PFB FIR (Eq. 1) and the first DFT stage (radix 8 R, with its
 * twiddle) as one contraction per FIR column on the tensor cores (tcgen05,
 * FP32 accumulation in tensor memory): the 10-bit samples are exact in FP16;
 * the weights x DFT operand is scaled by a power of two per output column.
 * The BF16 form carries samples and operand as hi + lo BF16 pairs (three
 * products per step). The second DFT stage, delay, gain and requantisation
 * run on CUDA cores in FP32, reading FP16 (FP16 form) or FP32 (BF16 form)
 * pairs. n_channels >= 32 (FENGINE_EUNSUPPORTED otherwise). Pre-quantisation
 * spectra stay within 2e-3 relative RMS of the FP64 oracle (measured: FP16
 * 3-4e-4, BF16 3-4e-6), 8-bit outputs within 1 LSB. */
typedef enum {
    FENGINE_FP32 = 0,    /* FP32 FIR and FFT on CUDA cores */
    FENGINE_TC_FP16 = 1, /* FIR + first DFT stage on tensor cores, FP16 operands, FP32 accumulation */
    FENGINE_TC_BF16 = 2  /* FIR + first DFT stage on tensor cores, BF16 hi + lo operands */
} fengine_precision;

/* Plan configuration (Sec. 2.1: channels and taps; Sec. 3.1: chunks;
 * Sec. 3.3: coarse delay range, which may include negative delays;
 * Sec. 2.2: 256 spectra per output heap). */
typedef struct {
    int32_t n_antennas;        /* >= 1 */
    int32_t n_pols;            /* must be 2 (dual-polarisation F-engine) */
    int32_t n_channels;        /* n: power of two, 16 <= n <= 32768 */
    int32_t n_taps;            /* T: one of 1, 2, 4, 8, 16, 32 */
    int64_t chunk_samples;     /* L per polarisation per call: a positive multiple of 2n */
    int32_t spectra_per_heap;  /* S: 1 <= S <= L/2n; 0 selects min(256, L/2n) */
    int32_t precision;         /* fengine_precision */
    int64_t max_delay_samples; /* D >= 0: every coarse delay must lie in [min_delay_samples, D] */
    const float *weights;      /* host, 2n*T prototype w[t + 2n j] (Eq. 1's w_{t,j});
                                  NULL = built-in Hann-windowed sinc, sum w^2 = 1 */
    /* Tuning knobs (no counterpart in the paper; 0 = built-in choice, see
     * fengine_autotune). They change how the work is split, not what is
     * computed: results agree with the oracle within the same bars. */
    int32_t fft_n1;            /* N1 of the four-step split N = N1 * N2: 8, 16, 32 or 64
                                  with N2 <= 1024 (and N2 >= 512 / N1 for N1 > 8);
                                  built-in: max(8, N / 1024) */
    int32_t slab_spectra;      /* spectra per slab of the two-phase pipeline, a multiple
                                  of 32; built-in: an FP32 intermediate of about 256 MiB */
    int64_t min_delay_samples; /* Dmin in [-2^30, 0]: the most negative coarse delay
                                  (Sec. 3.3 allows negative delays). The plan emits
                                  E = ceil(-Dmin / 2n) spectra later to make room. */
} fengine_config;

typedef struct fengine_plan_s *fengine_plan_t;

/* Read-only facts about a plan. */
typedef struct {
    int32_t n_channels, n_taps, n_antennas, spectra_per_heap;
    int32_t fft_n1, fft_n2;       /* four-step split N = n1 * n2 used on the device */
    int64_t spectra_per_chunk;    /* M = L / 2n: spectra every call emits per stream */
    int64_t history_samples;      /* H = 2n (T - 1) + D rounded up to a multiple of 16 */
    int64_t latency_spectra;      /* T - 1 + E: first spectrum of a call = first_sample/2n - (T-1+E) */
    int64_t out_bytes;            /* bytes of d_out per call: n_antennas * M * n * 4 */
    size_t device_bytes;          /* device memory the plan holds */
    size_t scratch_bytes;         /* part of device_bytes used as per-call scratch */
    int32_t slab_spectra;         /* spectra per slab of the two-phase pipeline (one launch pair) */
    int32_t slabs_per_chunk;      /* slabs (phase-1 + phase-2 launch pairs) per call */
    int32_t heaps_per_chunk;      /* output heaps per antenna per call: ceil(M / S) */
    int32_t lost_data;            /* 1 if lost-data flags are available (chunk_samples a
                                     multiple of FENGINE_HEAP_SAMPLES) */
} fengine_info;

const char *fengine_strerror(fengine_status status);
const char *fengine_last_error(void);
int32_t fengine_abi_version(void);

/* Built-in prototype filter (Sec. 5.2: Hann-windowed sinc), evaluated in FP64
 * and rounded to FP32: for u in [0, M), M = 2n T,
 *   w[u] = sin^2(pi (u + 1/2) / M) sinc((u + 1/2 - M/2) / 2n),
 * scaled so that sum w^2 = 1. out: host array of 2n*T floats. */
fengine_status fengine_default_weights(int32_t n_channels, int32_t n_taps, float *out);

/* The requantiser of one Gaussian-integer component that the kernels apply
 * (Sec. 2.1 step 6, Sec. 3.6): saturate to [-127, 127] and round half away
 * from zero, here evaluated on the host from the same source. */
int32_t fengine_quantise(float x);

/* Create a plan on the current CUDA device (use the plan only while that
 * device is current). Copies cfg->weights. Allocates all
 * device state up front (history tails zeroed: samples before a stream's first
 * chunk read as zero). Delays start at 0, phases at 0, gains at 1. */
fengine_status fengine_plan_create(const fengine_config *cfg, fengine_plan_t *out);
fengine_status fengine_plan_destroy(fengine_plan_t plan);
fengine_status fengine_get_info(fengine_plan_t plan, fengine_info *info);

/* Delay and phase model of one (antenna, pol) stream (Sec. 2.1 steps 2 and 4,
 * Sec. 3.3). From spectrum timestamp t0 >= t_apply on:
 *   d(t0)   = delay + delay_rate * (t0 - t_ref)      samples
 *   phi(t0) = phase + phase_rate * (t0 - t_ref)      radians
 * The spectrum uses coarse delay c = floor(d + 1/2) (window start t0 - c,
 * Eq. 1) and fine delay delta = d - c, applied as the channel rotation
 * exp(i (phi - 2 pi delta k / 2n)). Up to FENGINE_MAX_DELAY_SEGMENTS models
 * per stream are kept, ordered by t_apply; a new model with the same t_apply
 * replaces the old one. Takes effect from the next fengine_process_chunk.
 * Returns FENGINE_EINVAL for a bad index or non-finite parameter. */
fengine_status fengine_set_delay(fengine_plan_t plan, int32_t ant, int32_t pol,
                                 int64_t t_apply, int64_t t_ref, double delay,
                                 double delay_rate, double phase, double phase_rate);

/* Per-channel complex bandpass gains of one stream (Sec. 2.1 step 5): host
 * array of n complex values as interleaved (re, im) floats (copied), used
 * for spectra with timestamp t0 >= t_apply, like a delay model (the paper
 * gives no time rule; this is the library's reading). Up to
 * FENGINE_MAX_GAIN_SETS sets per stream are kept, ordered by t_apply; a set
 * with the same t_apply replaces the old one; sets that no later spectrum
 * can use are dropped at the next call. Use a t_apply far in the past (or
 * the next call's first spectrum timestamp) to apply gains at once.
 * FENGINE_EINVAL for a bad index, non-finite gains or too many pending sets. */
fengine_status fengine_set_gains(fengine_plan_t plan, int32_t ant, int32_t pol,
                                 const float *gains_re_im, int64_t t_apply);

/* Forget the stream history: the next call may start at any first_sample,
 * and samples before it read as zero. */
fengine_status fengine_reset(fengine_plan_t plan);

/* Channelize one chunk of every stream (Sec. 2.1 steps 1-6).
 *   d_packed       device, 4-byte aligned (as is d_out), [antenna][pol][5L/4] bytes: samples
 *                  [first_sample, first_sample + L) of each stream.
 *   first_sample   multiple of 2n; after the first call (or a reset) it must
 *                  equal the previous first_sample + L, else FENGINE_ESEQ.
 *   d_valid        optional (NULL: every heap received) device
 *                  [antenna][pol][L / FENGINE_HEAP_SAMPLES] bytes, nonzero
 *                  where the digitiser heap of samples [first_sample + 4096 i,
 *                  + 4096) arrived (Sec. 3.7). The plan keeps these flags for
 *                  the history; samples no call delivered (before a stream's
 *                  first chunk after creation or a reset) count as missing.
 *   d_heap_flags   optional device [antenna][heaps_per_chunk] bytes out: 1 if
 *                  every spectrum of the output heap is usable in both
 *                  polarisations, 0 if a spectrum's PFB window touches a
 *                  missing heap and the heap should not be transmitted
 *                  (Sec. 3.7). d_out is written either way (missing samples
 *                  are whatever d_packed holds). d_valid and d_heap_flags need
 *                  chunk_samples and first_sample to be multiples of
 *                  FENGINE_HEAP_SAMPLES (FENGINE_EINVAL); a call that is not
 *                  leaves the history's flags unknown until fengine_reset.
 *   d_out          device, n_antennas * M * n * 4 bytes: for each antenna the
 *                  M = L/2n spectra m = first_sample/2n - (T-1+E) + q,
 *                  q in [0, M), as heaps of S spectra (the last heap of a call
 *                  may hold fewer, S_h = min(S, M - h S)); heap h is the
 *                  array [k][s][pol][re, im] of int8 with q = h S + s
 *                  (channel-major within the heap, Sec. 2.2 / Sec. 3.6).
 *                  Values are round-half-away-from-zero, saturated to
 *                  [-127, 127].
 *   d_prequant     optional (NULL to skip) device FP32 [antenna][pol][M][n][re, im]:
 *                  the spectra after fine delay and gain, before quantisation.
 *   d_window_tap   optional (NULL to skip) device int32 [antenna][pol][M][2n]:
 *                  the unpacked, coarse-delayed samples s[2n m - c_m + t],
 *                  t in [0, 2n), that the first FIR tap of spectrum m uses.
 *   first_spectrum optional host out: the m of q = 0.
 * Every spectrum's window [2n m - c_m, 2n m - c_m + 2n T) lies in the data
 * this call and the plan's history hold, for every c_m in [Dmin, D]; a
 * delay model that puts c_m outside [Dmin, D] for a spectrum of this call is
 * refused with FENGINE_EDELAY before anything is enqueued. Asynchronous on
 * cuda_stream; the input may be reused once the stream passes this call. */
fengine_status fengine_process_chunk(fengine_plan_t plan, void *cuda_stream,
                                     const uint8_t *d_packed, int64_t first_sample,
                                     const uint8_t *d_valid, int8_t *d_out, uint8_t *d_heap_flags,
                                     float *d_prequant, int32_t *d_window_tap, int64_t *first_spectrum);

/* Waits for the device (cudaDeviceSynchronize) and reports a device-side
 * condition the plan's kernels recorded since the last call of this
 * function: FENGINE_ETIMEOUT if a bounded wait in a tensor-core kernel gave
 * up, FENGINE_EDELAY if a coarse delay had to be clamped (not reachable
 * after the host-side range check), FENGINE_ECUDA on a CUDA error; clears
 * the record. */
fengine_status fengine_device_status(fengine_plan_t plan);

/* ---- autotuning (no counterpart in the paper) ----
 *
 * Times every valid work split of cfg -- fft_n1 in {8, 16, 32, 64} (the
 * tensor-core forms have one: 8 R) x slab_spectra in {built-in, 32, 64,
 * ..., 2048} (capped at the call's spectra) -- by creating a plan for it and
 * running `calls` calls (after
 * two warm-up calls) on zero-filled input on cuda_stream, timed with CUDA
 * events, and writes cfg with the fastest split into *tuned. The work does
 * not depend on the sample values. Allocates (and frees) a temporary input
 * and output on the current device and synchronises cuda_stream. entries
 * (host, may be NULL) receives up to max_entries measured candidates,
 * *n_entries (may be NULL) their number. */
typedef struct {
    int32_t fft_n1, slab_spectra;   /* the split (slab_spectra as the plan resolved it) */
    float ms_per_call;              /* mean device time of one fengine_process_chunk */
} fengine_tune_entry;

fengine_status fengine_autotune(const fengine_config *cfg, void *cuda_stream, int32_t calls,
                                fengine_config *tuned, fengine_tune_entry *entries, int32_t max_entries,
                                int32_t *n_entries);

/* fengine_autotune with its pick kept in a JSON Lines file (one object per
 * line: device name, SM count, a hash of the library's sources, ABI version,
 * the shape fields of cfg, precision, and the chosen fft_n1, slab_spectra,
 * ms_per_call). A line whose
 * key fields all match cfg on the current device, and whose split still makes
 * a valid plan, is returned without timing anything (*from_cache = 1);
 * otherwise the split is tuned as fengine_autotune does and the file is
 * rewritten with that line replaced or added (written beside the file and
 * renamed over it). cache_path: host path, created if missing; lines of other
 * configurations are kept. Returns fengine_autotune's errors, FENGINE_EINVAL
 * for a NULL or empty path, FENGINE_EIO if the file cannot be written (the
 * tuned split is still returned in *tuned). */
fengine_status fengine_autotune_cached(const fengine_config *cfg, void *cuda_stream, int32_t calls,
                                       const char *cache_path, fengine_config *tuned, int32_t *from_cache);

/* ---- batching: many independent plans per call (uneven streams with
 * different channel counts, tap counts and chunk lengths; engines are
 * independent, Sec. 2.1 last paragraph) ---- */
typedef struct fengine_batch_s *fengine_batch_t;

/* One member of a batch call: the arguments fengine_process_chunk takes. */
typedef struct {
    fengine_plan_t plan;
    const uint8_t *d_packed;
    int64_t first_sample;
    int8_t *d_out;
    const uint8_t *d_valid;     /* optional, as fengine_process_chunk */
    uint8_t *d_heap_flags;      /* optional, as fengine_process_chunk */
} fengine_chunk_desc;

/* A batch owns n_pool (1..64) internal CUDA streams. */
fengine_status fengine_batch_create(int32_t n_pool, fengine_batch_t *out);
fengine_status fengine_batch_destroy(fengine_batch_t batch);

/* Process one chunk of each of n distinct plans as one call on cuda_stream:
 * every member computes exactly what fengine_process_chunk computes for it
 * (Sec. 2.1 steps 1-6). Members in the FP32 form are grouped: their small
 * per-call kernels run spread over the pool's streams, then their phase-1
 * and phase-2 work goes out as one grid per kernel instantiation (members
 * with the same taps and FFT split; up to 64 members per grid), slab by
 * slab, on cuda_stream. Members of the other forms run whole on the pool's
 * streams meanwhile, largest work first onto the least-loaded stream.
 * Everything forks from and joins back into cuda_stream (so the call can be
 * captured into a CUDA graph).
 * first_spectra (host, n entries, may be NULL) receives each member's first
 * spectrum. FENGINE_EINVAL for a repeated or invalid plan; a member that
 * fails validation stops the call with its status, members enqueued before
 * it still run and are joined. */
fengine_status fengine_batch_process(fengine_batch_t batch, void *cuda_stream,
                                     const fengine_chunk_desc *chunks, int32_t n,
                                     int64_t *first_spectra);

/* ---- streaming service: continuous batching of chunk requests (Sec. 3.1:
 * host-to-device copies, computation and device-to-host copies of many
 * chunks overlap) ---- */
typedef struct fengine_service_s *fengine_service_t;

typedef struct {
    int32_t n_streams;          /* CUDA streams requests are spread over (1..64) */
    int64_t hbm_budget_bytes;   /* device memory in-flight chunk buffers may hold */
} fengine_service_config;

typedef struct {
    int64_t admitted, completed, deferred, failed, queued;
    int64_t bytes_in_use, peak_bytes;
    double latency_p50_us, latency_p99_us, latency_max_us;   /* submit -> output on host; the
                                                               percentiles from a histogram of
                                                               1.1 %-wide bins, the maximum exact */
} fengine_service_stats;

/* Start the service on the current device: a dispatcher thread admits queued
 * requests in arrival order once their input and output buffers fit in the
 * budget next to the requests in flight; each plan keeps one CUDA stream, so
 * a plan's chunks run in order while different plans overlap on the device.
 * While a plan is used through a service, call its delay and gain setters
 * only through the service (they are applied in order with its chunks). */
fengine_status fengine_service_create(const fengine_service_config *cfg, fengine_service_t *out);

/* Queue one chunk of `plan` from HOST memory: h_packed holds the plan's
 * [antenna][pol][5L/4] bytes (pinned memory lets the copy run
 * asynchronously), h_out receives info.out_bytes of 8-bit output; h_valid
 * (optional) and h_heap_flags (optional) are host copies of
 * fengine_process_chunk's d_valid and d_heap_flags. All must stay valid
 * until fengine_service_wait returns for the ticket. The result equals
 * fengine_process_chunk's for the same chunk. */
fengine_status fengine_service_submit(fengine_service_t svc, fengine_plan_t plan, const uint8_t *h_packed,
                                      int64_t first_sample, const uint8_t *h_valid, int8_t *h_out,
                                      uint8_t *h_heap_flags, int64_t *ticket);

/* fengine_set_delay / fengine_set_gains, applied in order with the plan's
 * queued chunks. */
fengine_status fengine_service_set_delay(fengine_service_t svc, fengine_plan_t plan, int32_t ant, int32_t pol,
                                         int64_t t_apply, int64_t t_ref, double delay, double delay_rate,
                                         double phase, double phase_rate);
fengine_status fengine_service_set_gains(fengine_service_t svc, fengine_plan_t plan, int32_t ant, int32_t pol,
                                         const float *gains_re_im, int64_t t_apply);

/* Wait up to timeout_ms (-1: no limit) for a chunk request; returns its
 * status (FENGINE_ETIMEOUT if still running; FENGINE_EBUSY if it can never
 * fit the budget) and its latency from submit to output in host memory. A
 * ticket can be waited for once. */
fengine_status fengine_service_wait(fengine_service_t svc, int64_t ticket, int32_t timeout_ms, double *latency_us);
fengine_status fengine_service_get_stats(fengine_service_t svc, fengine_service_stats *out);

/* Finish every queued request, then stop. */
fengine_status fengine_service_destroy(fengine_service_t svc);

/* ---- host ingest: digitiser heaps -> chunks on the device (Sec. 3.1-3.2) ----
 * A digitiser sends each polarisation as heaps of FENGINE_HEAP_SAMPLES
 * samples (FENGINE_HEAP_BYTES packed bytes) with a timestamp; heaps arrive
 * per polarisation, possibly out of order, some not at all. An ingest object
 * takes such heaps in arrival order into a ring of pinned host memory (one
 * host write per byte: the copy a NIC's DMA would make), moves the ring to
 * the device in arrival order on its own CUDA stream as the heaps come
 * (overlapping the processing of earlier chunks), and assembles them there:
 * a kernel places each heap at its position in the chunk of its timestamp
 * ([antenna][pol][5L/4] bytes) and sets the chunk's received-heap flag.
 * A chunk of every stream (both polarisations of every antenna, paired by
 * timestamp) is emitted, in timestamp order, once all its heaps are in or
 * once a heap of a chunk more than reorder_chunks past it arrives (or on a
 * flush);
 * its missing heaps are zero-filled and flagged, and it goes through
 * fengine_process_chunk with those flags (Sec. 3.7: spectra whose window
 * touches a missing heap are unusable, their output heaps flagged). */
#define FENGINE_HEAP_BYTES (FENGINE_HEAP_SAMPLES * 10 / 8)

typedef struct fengine_ingest_s *fengine_ingest_t;

typedef struct {
    int32_t antenna, pol;
    int64_t timestamp;          /* first sample of the heap, a multiple of FENGINE_HEAP_SAMPLES */
    const uint8_t *payload;     /* host, FENGINE_HEAP_BYTES packed samples (10-bit MSB first) */
} fengine_heap;

typedef struct {
    int64_t heaps_accepted;     /* placed in the ring */
    int64_t heaps_late;         /* timestamp of a chunk already emitted (dropped) */
    int64_t heaps_duplicate;    /* a second copy of a heap already in its chunk (dropped) */
    int64_t heaps_outside;      /* timestamp before the first chunk (dropped) */
    int64_t heaps_missing;      /* heaps absent from emitted chunks (zero-filled, flagged) */
    int64_t chunks_emitted;
    int64_t bytes_to_device;    /* ring bytes copied host -> device */
} fengine_ingest_stats;

/* plan: the chunks' plan (chunk_samples and first_sample multiples of
 * FENGINE_HEAP_SAMPLES); the ingest does not own it and must be destroyed
 * first. first_sample: timestamp of the first chunk (the plan's next
 * first_sample). ring_heaps: heap slots of the host and device rings
 * (>= 1); reorder_chunks (0..3): how many chunks past the oldest pending one
 * may receive heaps while it waits; a heap of a later chunk makes the oldest
 * due (emitted with what it has). The device holds reorder_chunks + 1
 * assembly chunks. */
fengine_status fengine_ingest_create(fengine_plan_t plan, int64_t first_sample, int32_t ring_heaps,
                                     int32_t reorder_chunks, fengine_ingest_t *out);
fengine_status fengine_ingest_destroy(fengine_ingest_t ing);

/* Take heaps[0 .. n) in order into the ring; *accepted (host out) = how many
 * were consumed (placed or dropped and counted). It stops early, with
 * FENGINE_EBUSY, at a heap for a chunk beyond the reorder window or when the
 * ring is full: call fengine_ingest_poll, then push the rest. FENGINE_EINVAL
 * for a bad antenna, pol, unaligned timestamp or NULL payload (that heap is
 * not consumed). */
fengine_status fengine_ingest_push(fengine_ingest_t ing, const fengine_heap *heaps, int32_t n, int32_t *accepted);

/* Move the heaps pushed so far to the device and assemble them; then, if the
 * oldest pending chunk is due (complete, a push stopped at a heap past the
 * reorder window, or flush != 0), emit it: zero-fill and flag its missing heaps and run
 * fengine_process_chunk on cuda_stream into d_out / d_heap_flags (as
 * fengine_process_chunk; d_heap_flags may be NULL). *emitted = 1 and
 * *first_sample (its timestamp) / *first_spectrum set when a chunk was
 * emitted, *emitted = 0 otherwise (d_out untouched). One chunk per call. */
fengine_status fengine_ingest_poll(fengine_ingest_t ing, void *cuda_stream, int32_t flush, int8_t *d_out,
                                   uint8_t *d_heap_flags, int32_t *emitted, int64_t *first_sample,
                                   int64_t *first_spectrum);
fengine_status fengine_ingest_get_stats(fengine_ingest_t ing, fengine_ingest_stats *out);

/* ---- narrow-band mode (Sec. 6 names a narrow-band mode with a low-pass
 * filter before the PFB; this is the library's reading of it) ----
 * A down-converter turns the wide-band stream into a real stream at 2/D of
 * its rate whose positive frequencies are the band [fc - 1/(2D),
 * fc + 1/(2D)] (cycles per input sample): per stream,
 *   y[j] = 2 g Re( i^j sum_{u < Lh} h[u] x[j D/2 - u] exp(-2 pi i fc (j D/2 - u)) )
 * (mix the band's centre to 0, low-pass with the real h, move the band's
 * lower edge to 0, real part, keep every (D/2)-th sample), requantised to
 * 10 bits (round half away from zero, saturate to [-511, 511]) and packed
 * like the digitiser's stream (10 bits per sample, MSB first). Input
 * frequency f appears at (f - fc) D/2 + 1/4 cycles per output sample, so an
 * ordinary plan over the output channelizes the band into finer channels;
 * the wide-band plan can run on the same input chunks. */
typedef struct fengine_ddc_s *fengine_ddc_t;

typedef struct {
    int32_t n_antennas;        /* streams = 2 n_antennas */
    int32_t decimation;        /* D: 2, 4, 8, 16 or 32; the band is 1/D of the input rate */
    int32_t taps_per_phase;    /* Th: the low-pass has Lh = D Th taps, 1 <= Th, Lh <= 2048 */
    int32_t reserved;          /* 0 */
    int64_t chunk_samples;     /* L input samples per pol per call: a multiple of 2D and of 16, >= Lh */
    double center_frequency;   /* fc, cycles per input sample, in [0, 0.5) */
    float gain;                /* g, applied before the 10-bit requantisation */
    const float *filter;       /* host, Lh taps h[u]; NULL = built-in Hann-windowed sinc with
                                  cutoff 1/(2D) and unit DC gain (fengine_ddc_default_filter) */
} fengine_ddc_config;

/* The built-in low-pass: h[u] = sin^2(pi (u + 1/2) / Lh) sinc((u + 1/2 - Lh/2) / D),
 * scaled to sum h = 1; out: host, D Th floats. FENGINE_EINVAL for a bad shape. */
fengine_status fengine_ddc_default_filter(int32_t decimation, int32_t taps_per_phase, float *out);

/* The down-converter owns its history (the last Lh samples of every stream,
 * zero before a stream's first chunk) and its filter table on the current
 * device. */
fengine_status fengine_ddc_create(const fengine_ddc_config *cfg, fengine_ddc_t *out);
fengine_status fengine_ddc_destroy(fengine_ddc_t ddc);
/* Forget the history: the next call may start at any first_sample. */
fengine_status fengine_ddc_reset(fengine_ddc_t ddc);

/* One chunk of every stream.
 *   d_packed     device, 4-byte aligned, [antenna][pol][5L/4] bytes: input
 *                samples [first_sample, first_sample + L).
 *   first_sample a multiple of 2D; after the first call (or a reset) the
 *                previous first_sample + L, else FENGINE_ESEQ.
 *   d_out        device, 4-byte aligned, [antenna][pol][5 L' / 4] bytes,
 *                L' = 2L/D: output samples j = 2 first_sample / D + k,
 *                k in [0, L'), packed 10 bits per sample.
 *   d_out_float  optional device FP32 [antenna][pol][L']: y before
 *                requantisation (NULL to skip).
 * Asynchronous on cuda_stream. */
fengine_status fengine_ddc_process(fengine_ddc_t ddc, void *cuda_stream, const uint8_t *d_packed,
                                   int64_t first_sample, uint8_t *d_out, float *d_out_float);

/* ---- no-allocation variant (the paper has no counterpart) ----
 * For callers that cannot allocate device memory: a process whose device
 * memory is handed out in full by another allocator (a framework's caching
 * allocator, a fixed per-process budget), or a latency-critical streaming
 * loop that cannot afford the implicit device synchronisation of
 * cudaMalloc/cudaFree. fengine_process_chunk_noalloc runs the same kernels
 * as fengine_process_chunk without a plan and allocates nothing: the caller
 * passes every input and output in device memory, and the working storage
 * (delay table, twiddle tables, the inter-phase intermediate) lives in one
 * file-scope device array of FENGINE_NOALLOC_SCRATCH_BYTES that every GPU
 * which loads the library holds until the process exits.
 *  - The first call on a device looks up that array's device address (with
 *    the device current); make that first call before any stream capture
 *    (a first call on a stream that is being captured is refused with
 *    FENGINE_EINVAL).
 *  - Every call shares the array and overwrites it: calls whose work
 *    overlaps on the GPU (different streams, or different host threads
 *    without ordering) race; order them on one stream.
 *  - A shape whose working storage exceeds the array (or more than
 *    FENGINE_NOALLOC_MAX_STREAMS streams) is refused with FENGINE_EINVAL. */
#define FENGINE_NOALLOC_SCRATCH_BYTES (64u << 20)
#define FENGINE_NOALLOC_MAX_STREAMS 64

typedef struct {
    int32_t n_antennas, n_channels, n_taps, spectra_per_heap;  /* as fengine_config */
    int64_t chunk_samples, max_delay_samples;                   /* L and D, as fengine_config */
    int64_t first_sample;                                       /* multiple of 2n */
} fengine_noalloc_args;

/* d_history    device [antenna][pol][5H/4] bytes: samples [first_sample - H,
 *              first_sample) of each stream, H = 2n(T-1) + D rounded up to a
 *              multiple of 16 (zeros before a stream starts).
 * d_packed     device [antenna][pol][5L/4] bytes: samples [first_sample, + L).
 * d_weights    device [2n T] prototype w[t + 2n j].
 * d_gains      device [antenna][pol][n] complex gains as (re, im) floats.
 * delay_models host [antenna][pol][5] doubles: delay, delay_rate, phase,
 *              phase_rate, t_ref -- one model per stream, as fengine_set_delay;
 *              all finite and t_ref an integer (FENGINE_EINVAL otherwise).
 *              Coarse delays must stay in [0, D] (no negative delays here).
 * d_out        device, same layout as fengine_process_chunk's.
 * All device buffers 4-byte aligned. The output equals fengine_process_chunk's
 * for the same samples, weights, gains and delay models (within the
 * rounding of the twiddle tables, which are built on the device here).
 * Asynchronous on cuda_stream; FENGINE_EDELAY if a coarse delay of the call
 * leaves [0, D]. */
fengine_status fengine_process_chunk_noalloc(const fengine_noalloc_args *args, const uint8_t *d_history,
                                             const uint8_t *d_packed, const float *d_weights,
                                             const float *d_gains, const double *delay_models,
                                             int8_t *d_out, void *cuda_stream);

/* Per-stage device timing, a profiling aid. While enabled, every
 * fengine_process_chunk records CUDA events on its stream between its
 * kernels. fengine_stage_times waits for those events, writes the summed
 * milliseconds per stage to ms[0..4] = {delay table, phase 1 (FIR + first
 * FFT stage; in the FP32 form also the unpack), phase 2 (second FFT stage +
 * delay/gain + requantise + corner turn), history tail update, column unpack
 * (tensor-core forms; 0 in the FP32 form)}, the number of timed calls to
 * *calls, and starts a new accumulation. ms holds 5 floats. Disabled by
 * default. */
fengine_status fengine_set_profiling(fengine_plan_t plan, int32_t enable);
fengine_status fengine_stage_times(fengine_plan_t plan, float *ms, int32_t *calls);

#ifdef __cplusplus
}
#endif

#endif /* FENGINE_H */
