/*
 * FP64 CPU oracle of the F-engine channelizer hot path described in
 * B. Merry, "Efficient channelization on a Graphics Processing Unit"
 * (arXiv:2303.09886).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline /
 * reference legs of the benchmark load this library. The product library
 * (libfengine) never links, includes or calls it, and this file includes
 * nothing from the product.
 *
 * Everything here is the plain definition, written for a reader to check by
 * eye against the paper. No blocking, fusion or reordering beyond what the
 * definitions state. Steps, in the paper's order (Sec. 2.1, "Channelization"):
 *   1. 10-bit signed samples (Sec. 2.1 step 1; 4096-sample heaps of 5120 bytes,
 *      Sec. 2.2): orc_unpack10.
 *   2. Coarse delay as an index offset per spectrum (Sec. 2.1 step 2, Sec. 3.3):
 *      orc_delay_eval.
 *   3. PFB FIR, Eq. (1): g_t = sum_j s[t0 + t - c + 2n j] w_{t,j}: orc_fir.
 *   4. 2n-point real-to-complex DFT, keep the n non-negative bins, drop
 *      Nyquist (Sec. 2.1 step 3): orc_fft / orc_dft_naive.
 *   5. Fine delay as a frequency-domain phase rotation (Sec. 2.1 step 4) and
 *      per-channel complex gain (Sec. 2.1 step 5).
 *   6. Requantise to 8-bit signed Gaussian integers with rounding and
 *      saturation (Sec. 2.1 step 6, Sec. 3.6) and the channel-major
 *      corner turn within each 256-spectrum heap (Sec. 2.2, Sec. 3.6):
 *      orc_quantise / orc_corner_turn.
 *
 * Readings where the paper is silent (this oracle's and the library's choices):
 *   R1 bit order: sample i occupies bits [10i, 10i+10) of the chunk bit
 *      stream, most significant bit first (bit 0 = MSB of byte 0); the field
 *      is two's complement.
 *   R2 weights: w_{t,j} is the prototype w[t + 2n j] of length 2nT
 *      (the flattening under which the channel response is the Fourier
 *      transform of the weights, Sec. 5.2).
 *   R3 default prototype: Hann window times sinc, normalised to sum w^2 = 1.
 *   R4 delay model: d(t) = d0 + r (t - t_ref) samples, phi(t) = phi0 +
 *      phi_r (t - t_ref) radians, evaluated at the spectrum timestamp
 *      t0 = 2n m; c = floor(d + 1/2), delta = d - c.
 *   R5 DFT sign: X[k] = sum_t g[t] exp(-2 pi i k t / N), unnormalised.
 *   R6 fine delay: Y[k] = G[k] exp(i (phi - 2 pi delta k / N)) X[k].
 *   R7 quantiser: round half away from zero, saturate to [-127, 127].
 *   R8 samples before the first sample of a stream are zero.
 *   R12 a gain update, like a delay update, applies to spectra whose
 *      timestamp t0 is at or after its t_apply.
 *   R13 lost data (Sec. 3.7): a digitiser heap is 4096 samples (Sec. 2.2)
 *      starting at a multiple of 4096; heaps no chunk delivered (before a
 *      stream's first chunk, or flagged missing) are missing.
 *   R15 narrow-band mode (Sec. 6 names it only): a down-converter in front
 *      of the channelizer, described at orc_ddc below.
 * Steps 7-8 (lost data, Sec. 3.7): orc_window_usable / orc_spectrum_flags /
 * orc_heap_flags; gain sets that change at spectrum timestamps:
 * orc_segment_select; the narrow-band front end: orc_ddc_weights / orc_ddc.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- unpack */

/* Step 1 (Sec. 2.1, Sec. 2.2): sample i of the packed stream is the 10-bit
 * field at bits [10 i, 10 i + 10), read most significant bit first (R1),
 * interpreted as two's complement. Read bit by bit: slow and obvious. */
void orc_unpack10(const uint8_t *bytes, int64_t n_samples, int32_t *out)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n_samples; i++) {
        int64_t bit0 = 10 * i;
        int32_t raw = 0;
        for (int b = 0; b < 10; b++) {
            int64_t bit = bit0 + b;
            int v = (bytes[bit / 8] >> (7 - (int)(bit % 8))) & 1;
            raw = raw * 2 + v;
        }
        out[i] = raw >= 512 ? raw - 1024 : raw;
    }
}

/* ------------------------------------------------------------- weights */

/* Default PFB prototype (R3; Sec. 5.2 names a Hann-windowed sinc). For
 * u in [0, M), M = N T:  w[u] = sin^2(pi (u + 1/2) / M) * sinc((u + 1/2 - M/2) / N),
 * sinc(x) = sin(pi x) / (pi x), then scaled so that sum w^2 = 1. */
void orc_pfb_weights(int N, int T, double *w)
{
    int64_t M = (int64_t)N * T;
    double ss = 0.0;
    for (int64_t u = 0; u < M; u++) {
        double x = ((double)u + 0.5 - (double)M / 2.0) / (double)N;
        double sinc = (x == 0.0) ? 1.0 : sin(M_PI * x) / (M_PI * x);
        double h = sin(M_PI * ((double)u + 0.5) / (double)M);
        w[u] = h * h * sinc;
        ss += w[u] * w[u];
    }
    double scale = 1.0 / sqrt(ss);
    for (int64_t u = 0; u < M; u++)
        w[u] *= scale;
}

/* ---------------------------------------------------------- delay model */

/* Piecewise linear delay model (R4; coarse delay Sec. 2.1 step 2 and
 * Sec. 3.3, fine delay Sec. 2.1 step 4). Segment s applies to spectra with
 * timestamp t0 >= t_apply[s]; segments are sorted by t_apply; a timestamp
 * before every segment uses segment 0. */
void orc_delay_eval(int32_t n_seg, const int64_t *t_apply, const int64_t *t_ref,
                    const double *d0, const double *rate, const double *phi0,
                    const double *phi_rate, int64_t t0,
                    int64_t *c_out, double *delta_out, double *phi_out)
{
    int s = 0;
    for (int k = 0; k < n_seg; k++)
        if (t_apply[k] <= t0)
            s = k;
    double dt = (double)(t0 - t_ref[s]);
    double d = d0[s] + rate[s] * dt;
    double c = floor(d + 0.5);
    *c_out = (int64_t)c;
    *delta_out = d - c;
    *phi_out = phi0[s] + phi_rate[s] * dt;
}

/* ------------------------------------------------------------------ FIR */

/* Sample accessor with R8: s(i) = samples[i - first] inside the stream
 * window [first, first + count), zero elsewhere. */
static double sample_at(const int32_t *s, int64_t first, int64_t count, int64_t i)
{
    if (i < first || i >= first + count)
        return 0.0;
    return (double)s[i - first];
}

/* Eq. (1): g[t] = sum_{j<T} s[t0 + t - c + N j] * w[t + N j], 0 <= t < N. */
void orc_fir(const int32_t *s, int64_t first, int64_t count, int N, int T,
             const double *w, int64_t t0, int64_t c, double *g)
{
    for (int t = 0; t < N; t++) {
        double acc = 0.0;
        for (int j = 0; j < T; j++)
            acc += sample_at(s, first, count, t0 + t - c + (int64_t)N * j) *
                   w[t + (int64_t)N * j];
        g[t] = acc;
    }
}

/* ------------------------------------------------------------------ DFT */

/* Direct O(N^2) DFT, R5: X[k] = sum_t x[t] exp(-2 pi i k t / N). Interleaved
 * re/im in and out. The phase k t mod N is reduced exactly in integers. */
void orc_dft_naive(int N, const double *x, double *X)
{
    for (int k = 0; k < N; k++) {
        double re = 0.0, im = 0.0;
        for (int t = 0; t < N; t++) {
            int64_t ph = ((int64_t)k * t) % N;
            double a = -2.0 * M_PI * (double)ph / (double)N;
            double c = cos(a), s = sin(a);
            re += x[2 * t] * c - x[2 * t + 1] * s;
            im += x[2 * t] * s + x[2 * t + 1] * c;
        }
        X[2 * k] = re;
        X[2 * k + 1] = im;
    }
}

/* Radix-2 decimation-in-time FFT, same convention as orc_dft_naive; N a power
 * of two. In place on interleaved re/im. The twiddle exp(-2 pi i j / len) of a
 * stage of length len equals exp(-2 pi i (j N / len) / N), so one table of
 * exp(-2 pi i q / N), q < N/2, evaluated directly with cos/sin, serves all
 * stages. Returns -1 if the table cannot be allocated. */
int orc_fft(int N, double *x)
{
    double *tw = (double *)malloc(sizeof(double) * (N > 1 ? N : 2));
    if (!tw)
        return -1;
    for (int q = 0; q < N / 2; q++) {
        double a = -2.0 * M_PI * (double)q / (double)N;
        tw[2 * q] = cos(a);
        tw[2 * q + 1] = sin(a);
    }
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < N; i++) {
        int bit = N >> 1;
        for (; j & bit; bit >>= 1)
            j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr = x[2 * i], ti = x[2 * i + 1];
            x[2 * i] = x[2 * j];
            x[2 * i + 1] = x[2 * j + 1];
            x[2 * j] = tr;
            x[2 * j + 1] = ti;
        }
    }
    for (int len = 2; len <= N; len <<= 1) {
        int half = len >> 1;
        int step = N / len;
        for (int i = 0; i < N; i += len) {
            for (int j = 0; j < half; j++) {
                double wr = tw[2 * j * step], wi = tw[2 * j * step + 1];
                double *u = x + 2 * (i + j), *v = x + 2 * (i + j + half);
                double vr = v[0] * wr - v[1] * wi;
                double vi = v[0] * wi + v[1] * wr;
                v[0] = u[0] - vr;
                v[1] = u[1] - vi;
                u[0] = u[0] + vr;
                u[1] = u[1] + vi;
            }
        }
    }
    free(tw);
    return 0;
}

/* ------------------------------------------------------------- quantise */

/* R7: round half away from zero (C99 round), then saturate to [-127, 127]
 * (Sec. 2.1 step 6, Sec. 3.6 "rounding and saturation"). */
int32_t orc_quantise(double x)
{
    double r = round(x);
    if (r > 127.0)
        r = 127.0;
    if (r < -127.0)
        r = -127.0;
    return (int32_t)r;
}

/* ------------------------------------------------------ whole hot path */

/* Channelize spectra m_first .. m_first + m_count - 1 of one (antenna, pol)
 * stream. Spectrum m has timestamp t0 = N m (N = 2n, critically sampled).
 *   s, first, count : the stream's samples as integers (R8 outside).
 *   w               : N*T prototype (R2).
 *   delay model     : n_seg segments (R4).
 *   gains           : n complex (interleaved re/im), Sec. 2.1 step 5.
 *   prequant        : out, m_count * n complex, Y before quantisation.
 *   q               : out, m_count * n * 2 int8 (re, im), may be NULL.
 *   coarse          : out, m_count coarse delays, may be NULL.
 * Parallel over spectra with OpenMP. Returns 0, or -1 on allocation failure. */
int orc_channelize(const int32_t *s, int64_t first, int64_t count, int N, int T,
                   const double *w, int32_t n_seg, const int64_t *t_apply,
                   const int64_t *t_ref, const double *d0, const double *rate,
                   const double *phi0, const double *phi_rate,
                   const double *gains, int64_t m_first, int64_t m_count,
                   double *prequant, int8_t *q, int64_t *coarse)
{
    int n = N / 2;
    int err = 0;
    int64_t mi;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (mi = 0; mi < m_count; mi++) {
        double *g = (double *)malloc(sizeof(double) * N);
        double *X = (double *)malloc(sizeof(double) * 2 * N);
        if (!g || !X) {
            free(g);
            free(X);
            err |= 1;
            continue;
        }
        int64_t m = m_first + mi;
        int64_t t0 = (int64_t)N * m;
        int64_t c;
        double delta, phi;
        orc_delay_eval(n_seg, t_apply, t_ref, d0, rate, phi0, phi_rate, t0, &c,
                       &delta, &phi);
        if (coarse)
            coarse[mi] = c;
        orc_fir(s, first, count, N, T, w, t0, c, g);
        for (int t = 0; t < N; t++) {
            X[2 * t] = g[t];
            X[2 * t + 1] = 0.0;
        }
        if (orc_fft(N, X) != 0) {
            free(g);
            free(X);
            err |= 1;
            continue;
        }
        /* keep k = 0 .. n-1; Nyquist (k = n) and negative bins dropped */
        for (int k = 0; k < n; k++) {
            double a = phi - 2.0 * M_PI * delta * (double)k / (double)N;
            double rr = cos(a), ri = sin(a);
            double gr = gains[2 * k], gi = gains[2 * k + 1];
            /* (gr + i gi)(rr + i ri) */
            double fr = gr * rr - gi * ri, fi = gr * ri + gi * rr;
            double xr = X[2 * k], xi = X[2 * k + 1];
            double yr = fr * xr - fi * xi, yi = fr * xi + fi * xr;
            double *yp = prequant + 2 * ((int64_t)mi * n + k);
            yp[0] = yr;
            yp[1] = yi;
            if (q) {
                q[2 * ((int64_t)mi * n + k)] = (int8_t)orc_quantise(yr);
                q[2 * ((int64_t)mi * n + k) + 1] = (int8_t)orc_quantise(yi);
            }
        }
        free(g);
        free(X);
    }
    return err ? -1 : 0;
}

/* Corner turn (Sec. 2.2: a heap is a channels x spectra x pols array of
 * Gaussian integers; Sec. 3.6: channel-major within each heap). Input q_pol
 * for pol p is [m][k][re,im] for M spectra; output for one antenna is
 * out[h][k][s][p][re,im] with m = h S + s; the last heap holds
 * S_h = min(S, M - h S) spectra. */
void orc_corner_turn(const int8_t *q_pol0, const int8_t *q_pol1, int64_t M,
                     int n, int S, int8_t *out)
{
    const int8_t *qp[2] = {q_pol0, q_pol1};
    for (int64_t m = 0; m < M; m++) {
        int64_t h = m / S, s = m % S;
        int64_t Sh = (M - h * S) < S ? (M - h * S) : S;
        for (int k = 0; k < n; k++)
            for (int p = 0; p < 2; p++)
                for (int c = 0; c < 2; c++) {
                    int64_t off = h * (int64_t)S * n * 4 + (int64_t)k * Sh * 4 +
                                  s * 4 + p * 2 + c;
                    out[off] = qp[p][2 * (m * n + k) + c];
                }
    }
}

/* ------------------------------------------------------------ lost data */

/* floor(a / b) for b > 0, also for negative a. */
static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0)
        q -= 1;
    return q;
}

/* Lost data (Sec. 3.7): the receiver flags which digitiser heaps arrived;
 * a heap holds heap_len consecutive samples of one polarisation (4096,
 * Sec. 2.2), heap h holding samples [h heap_len, (h + 1) heap_len).
 * received[i] describes heap heap_first + i for i < n_heaps; every heap
 * outside that range counts as missing (so do samples before a stream's
 * first chunk). A window [start, start + len) is usable iff every heap it
 * touches was received. Returns 1 (usable) or 0. */
int orc_window_usable(const uint8_t *received, int64_t heap_first, int64_t n_heaps,
                      int64_t heap_len, int64_t start, int64_t len)
{
    int64_t h0 = floor_div(start, heap_len);
    int64_t h1 = floor_div(start + len - 1, heap_len);
    for (int64_t h = h0; h <= h1; h++) {
        if (h < heap_first || h >= heap_first + n_heaps)
            return 0;
        if (!received[h - heap_first])
            return 0;
    }
    return 1;
}

/* Sec. 3.7: the output spectrum m is flagged unusable if the window of input
 * samples of its PFB, [t0 - c, t0 - c + N T) with t0 = N m and c the coarse
 * delay of the delay model (orc_delay_eval), has any missing data.
 * usable[i] (i < m_count) is 1 or 0 for spectrum m_first + i. */
void orc_spectrum_flags(const uint8_t *received, int64_t heap_first, int64_t n_heaps,
                        int64_t heap_len, int N, int T, int32_t n_seg,
                        const int64_t *t_apply, const int64_t *t_ref, const double *d0,
                        const double *rate, const double *phi0, const double *phi_rate,
                        int64_t m_first, int64_t m_count, uint8_t *usable)
{
    for (int64_t i = 0; i < m_count; i++) {
        int64_t t0 = (int64_t)N * (m_first + i);
        int64_t c;
        double delta, phi;
        orc_delay_eval(n_seg, t_apply, t_ref, d0, rate, phi0, phi_rate, t0, &c, &delta, &phi);
        usable[i] = (uint8_t)orc_window_usable(received, heap_first, n_heaps, heap_len,
                                                t0 - c, (int64_t)N * T);
    }
}

/* Sec. 3.7 with Sec. 2.1 (an output heap carries both polarisations of an
 * antenna): output heap h of a call, spectra h S .. h S + S_h - 1 with
 * S_h = min(S, M - h S) (the heap layout of orc_corner_turn), is transmitted
 * (heap_ok[h] = 1) only if all of its spectra are usable in both
 * polarisations; otherwise heap_ok[h] = 0. */
void orc_heap_flags(const uint8_t *usable_pol0, const uint8_t *usable_pol1, int64_t M, int S,
                    uint8_t *heap_ok)
{
    int64_t n_heaps = (M + S - 1) / S;
    for (int64_t h = 0; h < n_heaps; h++) {
        int ok = 1;
        for (int64_t m = h * S; m < M && m < (h + 1) * S; m++)
            if (!usable_pol0[m] || !usable_pol1[m])
                ok = 0;
        heap_ok[h] = (uint8_t)ok;
    }
}

/* --------------------------------------------------------- gain updates */

/* Bandpass gains change at spectrum timestamps like the delay model (Sec. 2.1
 * step 5 gives the per-channel correction; the time it applies from is this
 * library's reading R12): gain set s applies to spectra with timestamp
 * t0 >= t_apply[s], sets sorted by t_apply, a timestamp before every set uses
 * set 0. Returns the index of the set that spectrum timestamp t0 uses. */
int32_t orc_segment_select(int32_t n_seg, const int64_t *t_apply, int64_t t0)
{
    int32_t s = 0;
    for (int32_t k = 0; k < n_seg; k++)
        if (t_apply[k] <= t0)
            s = k;
    return s;
}

/* ------------------------------------------------------ narrow-band mode */

/* Narrow-band front end. The paper names a narrow-band mode (Sec. 6: a
 * low-pass filter before the PFB) without specifying it; this is the
 * library's reading R15 of it, a digital down-converter that turns the
 * wide-band stream into a real stream at a lower rate which the same
 * channelizer then takes:
 *   band        [fc - 1/(2D), fc + 1/(2D)] of the input (D a power of two),
 *   mix         m[i] = x[i] exp(-2 pi i fc i),
 *   low-pass    z[i] = sum_{u < Lh} h[u] m[i - u]  (real h, cutoff 1/(2D)),
 *   shift       the band's lower edge to 0: z[i] exp(+2 pi i i / (2D)),
 *   real part   y = 2 g Re(.), which keeps the band's amplitudes,
 *   decimate    keep every (D/2)-th sample: y[j] at input sample j D / 2.
 * Output j therefore holds 2 g Re(exp(2 pi i j / 4) sum_u h[u] x[j D/2 - u]
 * exp(-2 pi i fc (j D/2 - u))); the band appears at output frequencies
 * [0, 1/2) cycles per output sample, input frequency f at (f - fc) D / 2 +
 * 1/4. The output is requantised to 10 bits (round half away from zero,
 * saturate to [-511, 511]) so that the channelizer reads it like a
 * digitiser stream.
 *
 * Default low-pass (R15): Lh = D Th taps, h[u] = sin^2(pi (u + 1/2) / Lh) *
 * sinc((u + 1/2 - Lh/2) / D), scaled to unit DC gain (sum h = 1). */
void orc_ddc_weights(int D, int Th, double *h)
{
    int64_t L = (int64_t)D * Th;
    double s = 0.0;
    for (int64_t u = 0; u < L; u++) {
        double x = ((double)u + 0.5 - (double)L / 2.0) / (double)D;
        double sinc = (x == 0.0) ? 1.0 : sin(M_PI * x) / (M_PI * x);
        double w = sin(M_PI * ((double)u + 0.5) / (double)L);
        h[u] = w * w * sinc;
        s += h[u];
    }
    for (int64_t u = 0; u < L; u++)
        h[u] /= s;
}

/* R15 requantiser: round half away from zero, saturate to [-511, 511]. */
int32_t orc_quantise10(double x)
{
    double r = round(x);
    if (r > 511.0)
        r = 511.0;
    if (r < -511.0)
        r = -511.0;
    return (int32_t)r;
}

/* Outputs j = j0 .. j0 + n_out - 1 of the down-converter for one stream.
 *   x, first, count : input samples (zero outside, R8).
 *   D, Lh, h        : decimation (even) and low-pass taps.
 *   fc, g           : centre frequency (cycles per input sample) and gain.
 *   y               : out, n_out doubles before requantisation.
 *   q               : out, n_out 10-bit values, may be NULL. */
void orc_ddc(const int32_t *x, int64_t first, int64_t count, int D, int Lh, const double *h,
             double fc, double g, int64_t j0, int64_t n_out, double *y, int32_t *q)
{
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < n_out; k++) {
        int64_t j = j0 + k;
        int64_t i0 = j * (D / 2);
        double re = 0.0, im = 0.0;
        for (int u = 0; u < Lh; u++) {
            int64_t i = i0 - u;
            double v = (i >= first && i < first + count) ? (double)x[i - first] : 0.0;
            /* the mixing phase fc i, reduced to one cycle before the
             * trigonometry (fc i can be large) */
            double ph = fc * (double)i;
            ph -= floor(ph);
            re += h[u] * v * cos(2.0 * M_PI * ph);
            im -= h[u] * v * sin(2.0 * M_PI * ph);
        }
        /* exp(2 pi i j / 4) = i^j: a quarter turn per output sample */
        int64_t r = ((j % 4) + 4) % 4;
        double out_re = r == 0 ? re : r == 1 ? -im : r == 2 ? -re : im;
        y[k] = 2.0 * g * out_re;
        if (q)
            q[k] = orc_quantise10(y[k]);
    }
}
