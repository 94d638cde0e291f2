"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-derived
golden bytes, a library FFT, closed forms of the PFB for tones, invariants
(shift, Parseval, linearity) and the exact quantiser definition.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_09886_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dtft(w, f):
    """W(f) = sum_u w[u] exp(-2 pi i f u), a library-free closed-form helper."""
    u = np.arange(w.size)
    return np.sum(w * np.exp(-2j * np.pi * f * u))


# ----------------------------------------------------------------- unpack

def test_unpack_golden():
    with open(os.path.join(GOLDEN, "unpack10_msb.txt")) as fh:
        lines = [l for l in fh if l.strip() and not l.startswith("#")]
    assert len(lines) == 3
    for line in lines:
        hexpart, vals = line.split(";")
        b = np.array([int(x, 16) for x in hexpart.split()], np.uint8)
        expect = np.array([int(v) for v in vals.split()], np.int32)
        got = O.unpack10(b, expect.size)
        np.testing.assert_array_equal(got, expect)


def test_unpack_pack_roundtrip_all_values_all_offsets():
    # every 10-bit value at every one of the 4 positions of a 5-byte group
    vals = np.arange(-512, 512, dtype=np.int32)
    for shift in range(4):
        s = np.roll(np.tile(vals, 4), shift)
        got = O.unpack10(synth.pack10(s), s.size)
        np.testing.assert_array_equal(got, s)


def test_pack10_known_bytes():
    # the generator's packer against the same hand-derived bytes
    np.testing.assert_array_equal(synth.pack10(np.array([-512, -1, 0, 511])),
                                  np.array([0x80, 0x3F, 0xF0, 0x01, 0xFF], np.uint8))


# -------------------------------------------------------------------- DFT

@pytest.mark.parametrize("N", [1, 2, 4, 8, 16, 64, 256])
def test_fft_matches_naive_dft(N):
    g = np.random.default_rng(N)
    x = g.standard_normal(N) + 1j * g.standard_normal(N)
    a, b = O.fft(x), O.dft_naive(x)
    assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("N", [32, 1024, 16384, 65536])
def test_fft_matches_library(N):
    g = np.random.default_rng(N)
    x = g.standard_normal(N) + 1j * g.standard_normal(N)
    a, b = O.fft(x), np.fft.fft(x)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_dft_sign_and_closed_forms():
    N = 16
    delta1 = np.zeros(N, complex)
    delta1[1] = 1.0
    k = np.arange(N)
    # a delayed impulse transforms to exp(-2 pi i k / N): fixes the sign (R5)
    np.testing.assert_allclose(O.dft_naive(delta1), np.exp(-2j * np.pi * k / N), atol=1e-13)
    np.testing.assert_allclose(O.fft(delta1), np.exp(-2j * np.pi * k / N), atol=1e-13)
    const = np.ones(N, complex)
    expect = np.zeros(N, complex)
    expect[0] = N
    np.testing.assert_allclose(O.fft(const), expect, atol=1e-12)


def test_parseval_real_input():
    N = 2048
    g = np.random.default_rng(7).standard_normal(N)
    X = O.fft(g.astype(complex))
    lhs = np.sum(g * g)
    rhs = (abs(X[0]) ** 2 + abs(X[N // 2]) ** 2 + 2 * np.sum(np.abs(X[1:N // 2]) ** 2)) / N
    assert abs(lhs - rhs) <= 1e-10 * lhs


# ---------------------------------------------------------------- weights

@pytest.mark.parametrize("N,T", [(64, 4), (2048, 16), (16384, 16)])
def test_default_weights_shape(N, T):
    w = O.pfb_weights(N, T)
    assert w.size == N * T
    assert np.max(np.abs(w - w[::-1])) < 1e-15          # linear phase
    assert abs(np.sum(w * w) - 1.0) < 1e-12               # R3 normalisation
    W0 = abs(_dtft(w, 0.0))
    # sinc cut-off at half a channel: adjacent channels cross near -6 dB
    half = 20 * np.log10(abs(_dtft(w, 0.5 / N)) / W0)
    assert -6.5 < half < -5.5
    # stopband at the next channel centre
    assert 20 * np.log10(abs(_dtft(w, 1.0 / N)) / W0) < (-40 if T < 8 else -75)


# ----------------------------------------------------- delay model (R4)

@pytest.mark.parametrize("d,c,delta", [(7.3, 7, 0.3), (7.5, 8, -0.5), (-0.2, 0, -0.2),
                                       (-0.5, 0, -0.5), (-0.7, -1, 0.3), (0.0, 0, 0.0)])
def test_delay_split(d, c, delta):
    cc, dd, ph = O.DelayModel.constant(delay=d, phase=0.25).eval(12345)
    assert cc == c and abs(dd - delta) < 1e-12 and ph == 0.25


def test_delay_rate_and_segments():
    m = O.DelayModel([(-(2 ** 62), 0, 1.0, 1e-3, 0.0, 0.01), (5000, 5000, 100.0, 0.0, 1.0, 0.0)])
    c, dl, ph = m.eval(1000)            # d = 1 + 1e-3 * 1000 = 2
    assert c == 2 and abs(dl) < 1e-12 and abs(ph - 10.0) < 1e-12
    c, dl, ph = m.eval(5000)            # second segment
    assert c == 100 and dl == 0.0 and ph == 1.0


# ------------------------------------------------ FIR + DFT composition

def test_pfb_closed_form_composition():
    """Eq. 1 followed by the DFT equals one sum over the whole window:
    X[k] = sum_{u < N T} w[u] s[t0 - c + u] exp(-2 pi i k u / N)."""
    N, T = 64, 4
    n = N // 2
    g = np.random.default_rng(3)
    s = g.integers(-512, 512, size=4096).astype(np.int32)
    w = g.standard_normal(N * T)           # arbitrary weights: checks the index map
    c = 5
    m = 20
    pre, _, co = O.channelize(s, 0, N, T, w, O.DelayModel.constant(delay=c), np.ones(n), m, 1)
    assert co[0] == c
    u = np.arange(N * T)
    win = s[N * m - c + u].astype(np.float64)
    k = np.arange(n)[:, None]
    X = np.sum(w * win * np.exp(-2j * np.pi * ((k * u) % N) / N), axis=1)
    np.testing.assert_allclose(pre[0], X, rtol=0, atol=1e-9 * np.max(np.abs(X)))


def test_fir_missing_samples_are_zero():
    N, T = 16, 2
    s = np.arange(1, 33, dtype=np.int32)       # samples at absolute 100..131
    w = np.ones(N * T)
    g = O.fir(s, 100, N, T, w, t0=96, c=0)     # window [96, 128)
    # t covers [96,112) and [112,128): sums of in-range samples only
    expect = np.array([(s[t - 4] if t >= 4 else 0) + s[t + 12] for t in range(N)], float)
    np.testing.assert_array_equal(g, expect)


# --------------------------------------------------------- tone responses

def _tone(N, total, f, A, psi, start=0):
    i = np.arange(start, start + total, dtype=np.float64)
    return A * np.cos(2 * np.pi * f * i + psi)


def test_bin_centred_tone_lands_in_one_channel():
    """Channel response is the Fourier transform of the weights (Sec. 5.2):
    a bin-centred tone gives (A/2) W(0) in its channel plus one image term."""
    N, T, k0, A = 256, 8, 19, 1000.0
    n = N // 2
    w = O.pfb_weights(N, T)
    s = np.rint(_tone(N, N * 64, k0 / N, A, 0.4)).astype(np.int32)
    # the closed form holds for the unrounded tone; the oracle sees the rounded
    # one, which differs by at most half a unit per sample
    s_exact = _tone(N, N * 64, k0 / N, A, 0.4)
    m = 10
    pre, _, _ = O.channelize(s, 0, N, T, w, O.DelayModel.constant(), np.ones(n), m, 1)
    P = np.abs(pre[0]) ** 2
    assert P[k0] / P.sum() > 0.999
    # closed form on the exact tone (quantisation of the tone adds white noise)
    t0 = N * m
    u = np.arange(N * T)
    X_exact = np.sum(w * s_exact[t0 + u] * np.exp(-2j * np.pi * k0 * u / N))
    W0 = _dtft(w, 0.0)
    Wimg = _dtft(w, 2 * k0 / N)
    theta = 2 * np.pi * k0 * t0 / N + 0.4
    main = 0.5 * A * W0 * np.exp(1j * theta)
    assert abs(X_exact - main) <= 0.5 * A * abs(Wimg) * (1 + 1e-9) + 1e-9
    # rounding the tone to integers moves the channel by at most the
    # rounding noise bound sum |w| * 0.5
    assert abs(pre[0][k0] - X_exact) <= 0.5 * np.sum(np.abs(w))
    # every other channel: below the stopband given by W at >= 1 channel
    others = np.delete(P, k0) / P[k0]
    assert 10 * np.log10(others.max()) < -60


def test_sub_channel_tone_response_matches_weight_transform():
    """Sec. 5.2: the channel response follows |W(f - k/N)| (sub-channel sweep)."""
    N, T, A = 128, 8, 1.0e4
    n = N // 2
    w = O.pfb_weights(N, T)
    k0 = 23
    for frac in (0.0, 0.2, 0.5, 0.8):
        f = (k0 + frac) / N
        s = np.rint(_tone(N, N * 40, f, A, 1.1)).astype(np.int32)
        pre, _, _ = O.channelize(s, 0, N, T, w, O.DelayModel.constant(), np.ones(n), 12, 1)
        for k in (k0 - 1, k0, k0 + 1, k0 + 2):
            expect = 0.5 * A * abs(_dtft(w, f - k / N))
            bound = 0.5 * A * abs(_dtft(w, f + k / N)) + 0.5 * np.sum(np.abs(w))
            assert abs(abs(pre[0][k]) - expect) <= bound


# ----------------------------------------------------------- delays

def test_integer_delay_is_a_sample_shift():
    N, T = 64, 4
    n = N // 2
    g = np.random.default_rng(11)
    s = g.integers(-512, 512, size=8192).astype(np.int32)
    w = O.pfb_weights(N, T)
    c = 5
    shifted = np.concatenate([np.zeros(c, np.int32), s[:-c]])   # s'[i] = s[i - c]
    a, _, _ = O.channelize(s, 0, N, T, w, O.DelayModel.constant(delay=c), np.ones(n), 3, 20)
    b, _, _ = O.channelize(shifted, 0, N, T, w, O.DelayModel.constant(), np.ones(n), 3, 20)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("d", [0.3, 0.7, 1.0, 7.3, 12.49])
def test_fine_and_coarse_delay_compose(d):
    """A total delay d (split into coarse c and fine delta, R4/R6) delays a
    bin-centred tone: Y_d[k0] = Y_0[k0] exp(-2 pi i k0 d / N), up to the
    image term."""
    N, T, k0, A = 256, 8, 37, 3000.0
    n = N // 2
    w = O.pfb_weights(N, T)
    s = _tone(N, N * 64, k0 / N, A, 0.2)
    si = np.rint(s * 1000).astype(np.int64)   # keep the tone almost exact
    assert np.abs(si).max() < 2 ** 31
    si = si.astype(np.int32)
    y0, _, _ = O.channelize(si, 0, N, T, w, O.DelayModel.constant(), np.ones(n), 20, 1)
    yd, _, _ = O.channelize(si, 0, N, T, w, O.DelayModel.constant(delay=d), np.ones(n), 20, 1)
    img = 0.5 * A * 1000 * abs(_dtft(w, 2 * k0 / N))
    noise = 0.5 * np.sum(np.abs(w))
    expect = y0[0][k0] * np.exp(-2j * np.pi * k0 * d / N)
    assert abs(yd[0][k0] - expect) <= 2 * (img + noise) + 1e-6 * abs(expect)


def test_phase_and_gain():
    N, T = 64, 4
    n = N // 2
    g = np.random.default_rng(5)
    s = g.integers(-512, 512, size=4096).astype(np.int32)
    w = O.pfb_weights(N, T)
    base, _, _ = O.channelize(s, 0, N, T, w, O.DelayModel.constant(delay=2.3), np.ones(n), 4, 8)
    ph, _, _ = O.channelize(s, 0, N, T, w, O.DelayModel.constant(delay=2.3, phase=0.1), np.ones(n), 4, 8)
    np.testing.assert_allclose(ph, base * np.exp(0.1j), rtol=1e-12, atol=1e-9)
    two, _, _ = O.channelize(s, 0, N, T, w, O.DelayModel.constant(delay=2.3), 2 * np.ones(n), 4, 8)
    np.testing.assert_array_equal(two, 2 * base)
    G = np.exp(1j * np.linspace(0, 3, n))
    rot, _, _ = O.channelize(s, 0, N, T, w, O.DelayModel.constant(delay=2.3), G, 4, 8)
    np.testing.assert_allclose(rot, base * G, rtol=1e-12, atol=1e-9)


# ----------------------------------------------------------- quantiser

@pytest.mark.parametrize("x,q", [(0.0, 0), (0.49999999, 0), (0.5, 1), (-0.5, -1), (1.5, 2),
                                 (2.5, 3), (-2.5, -3), (126.4, 126), (126.5, 127), (127.5, 127),
                                 (-127.5, -127), (-128.0, -127), (1e6, 127), (-1e6, -127)])
def test_quantiser_half_away_and_saturate(x, q):
    assert O.quantise(x) == q


def test_saturating_tone_never_minus_128():
    N, T, k0 = 2048, 16, 192      # tone in channel 192 of 1024, as in Sec. 3.5.1
    n = N // 2
    w = O.pfb_weights(N, T)
    s = np.clip(np.rint(_tone(N, N * 24, k0 / N, 100.0, 0.3)), -512, 511).astype(np.int32)
    pre, q, _ = O.channelize(s, 0, N, T, w, O.DelayModel.constant(), np.ones(n), 2, 4)
    assert np.abs(pre[:, k0]).max() > 1000          # far beyond full scale
    assert q.min() >= -127 and q.max() <= 127
    tone = q[:, k0, :]
    assert np.all(np.abs(tone).max(axis=1) == 127)


# ----------------------------------------------------------- corner turn

def test_corner_turn_golden():
    with open(os.path.join(GOLDEN, "corner_turn_small.txt")) as fh:
        lines = [l for l in fh if l.strip() and not l.startswith("#")]
    hdr = dict(kv.split("=") for kv in lines[0].split())
    M, n, S = int(hdr["M"]), int(hdr["n"]), int(hdr["S"])
    expect = np.array([int(v) for v in lines[1].split()], np.int8)
    q0 = np.empty((M, n, 2), np.int8)
    for m in range(M):
        for k in range(n):
            q0[m, k] = (10 * m + 2 * k + 1, 10 * m + 2 * k + 2)
    out = O.corner_turn(q0, -q0, S)
    np.testing.assert_array_equal(out, expect)


# -------------------------------------------------------------- lost data

def _golden_lost():
    with open(os.path.join(GOLDEN, "lost_data_small.txt")) as fh:
        return [l.strip() for l in fh if l.strip() and not l.startswith("#")]


def test_lost_data_golden():
    rec = [np.ones(20, np.uint8), np.ones(20, np.uint8)]
    rec[0][5] = 0
    rec[1][9] = 0
    usable = {}
    for line in _golden_lost():
        head, tail = line.split(";")
        expect = [int(v) for v in tail.split()]
        if head.startswith("heaps"):
            got = O.heap_flags(usable[(0, 0)], usable[(1, 0)], 4)
            np.testing.assert_array_equal(got, np.array(expect, np.uint8))
            continue
        pol, c = (int(v) for v in head.split())
        f = O.spectrum_flags(rec[pol], 0, 2048, 4, O.DelayModel.constant(float(c)), 0, 20)
        usable[(pol, c)] = f
        np.testing.assert_array_equal(np.where(f == 0)[0], np.array(expect))


@pytest.mark.parametrize("seed", range(6))
def test_lost_data_brute_force_per_sample(seed):
    # sample-by-sample definition on tiny streams: a spectrum is usable iff no
    # sample of its window lies in a missing heap (or before the stream)
    g = np.random.default_rng(seed)
    heap = int(g.choice([16, 32, 64]))
    N, T = int(g.choice([8, 16, 32])), int(g.choice([1, 2, 4]))
    n_heaps = 24
    rec = (g.random(n_heaps) > 0.25).astype(np.uint8)
    first = int(g.integers(0, 3))          # heaps before `first` are missing
    d = float(g.uniform(-40, 40))
    rate = float(g.choice([0.0, 0.01]))
    dm = O.DelayModel.constant(d, rate=rate)
    M = (n_heaps * heap) // N
    f = O.spectrum_flags(rec[first:], first, N, T, dm, 0, M, heap_len=heap)
    ok_sample = np.zeros(n_heaps * heap + 4096, bool)
    for h in range(first, n_heaps):
        ok_sample[h * heap:(h + 1) * heap] = bool(rec[h])
    for m in range(M):
        c, _, _ = dm.eval(N * m)
        idx = N * m - c + np.arange(N * T)
        expect = bool(np.all(idx >= 0) and np.all(ok_sample[np.clip(idx, 0, None)]))
        assert bool(f[m]) == expect, (seed, m)


def test_heap_flags_partial_last_heap():
    u0 = np.array([1, 1, 1, 1, 1, 1, 1, 0], np.uint8)    # last (partial) heap: spectrum 7 unusable
    u1 = np.array([1, 0, 1, 1, 1, 1, 1, 1], np.uint8)
    np.testing.assert_array_equal(O.heap_flags(u0, u1, 3), [0, 1, 0])
    np.testing.assert_array_equal(O.heap_flags(u1, u1, 3), [0, 1, 1])


# ----------------------------------------------------------- gain updates

def test_gain_set_applies_from_t_apply():
    # a second gain set equal to twice the first, applied from spectrum 5 on:
    # spectra 0..4 keep the first set, 5.. are exactly doubled (power-of-two
    # scaling is exact), and the switch is at t0 >= t_apply, not after it
    N, T = 64, 4
    g = np.random.default_rng(3)
    s = g.integers(-300, 300, 4096).astype(np.int32)
    w = O.pfb_weights(N, T)
    G0 = g.uniform(0.5, 2, N // 2) * np.exp(2j * np.pi * g.random(N // 2))
    dm = O.DelayModel.constant(3.25, phase=0.4)
    base, _, _ = O.channelize(s, 0, N, T, w, dm, G0, 4, 12)
    sched, _, _ = O.channelize(s, 0, N, T, w, dm, [(-(2 ** 62), G0), (N * 5, 2 * G0)], 4, 12)
    np.testing.assert_array_equal(sched[:1], base[:1])            # m = 4 < 5
    np.testing.assert_array_equal(sched[1:], 2 * base[1:])         # m >= 5
    assert O.segment_select([-(2 ** 62), N * 5], N * 5) == 1
    assert O.segment_select([-(2 ** 62), N * 5], N * 5 - 1) == 0
    assert O.segment_select([100, 200], 50) == 0                  # before every set: set 0


# --------------------------------------------------------- negative delays

@pytest.mark.parametrize("c", [1, 7, 300])
def test_negative_integer_delay_is_a_shift_the_other_way(c):
    # Sec. 3.3 allows negative delays: delay -c on stream s equals delay 0 on
    # the stream advanced by c samples (s'[i] = s[i + c]), exactly
    N, T = 128, 4
    g = np.random.default_rng(c)
    s = g.integers(-512, 512, 40 * N).astype(np.int32)
    w = O.pfb_weights(N, T)
    neg, qn, cn = O.channelize(s, 0, N, T, w, O.DelayModel.constant(-float(c), phase=0.2), np.ones(N // 2), 2, 20)
    adv, qa, _ = O.channelize(s[c:], 0, N, T, w, O.DelayModel.constant(0.0, phase=0.2), np.ones(N // 2), 2, 20)
    assert np.all(cn == -c)
    np.testing.assert_array_equal(neg, adv)
    np.testing.assert_array_equal(qn, qa)


# ------------------------------------------------ narrow-band front end (R15)

def test_ddc_weights_lowpass_shape():
    """Unit DC gain, symmetric, -6 dB at the cutoff 1/(2D), flat passband and
    a stopband below -40 dB one transition width past the cutoff."""
    for D, Th in ((4, 16), (8, 16), (16, 8)):
        h = O.ddc_weights(D, Th)
        assert h.size == D * Th
        assert abs(h.sum() - 1.0) < 1e-12
        np.testing.assert_allclose(h, h[::-1], atol=1e-15)
        F = 1 << 16
        H = np.abs(np.fft.fft(h, F))
        f = np.arange(F) / F
        edge = 20 * np.log10(H[int(round(F / (2 * D)))])
        assert abs(edge + 6.02) < 0.2
        if Th >= 16:   # the transition narrows with the taps: Th = 16 is the default
            pb = H[f < 0.8 / (2 * D)]
            assert 20 * np.log10(pb.max() / pb.min()) < 0.15
            assert 20 * np.log10(H[(f > 1.25 / (2 * D)) & (f < 0.5)].max()) < -40.0


def _ddc_stepwise(x, first, D, h, fc, g, j0, n_out):
    """The down-converter's steps one after another at the full rate (mix,
    low-pass by np.convolve, shift the band edge to 0, real part, keep every
    (D/2)-th sample): an independent formulation of the fused sum."""
    lo = j0 * (D // 2) - h.size + 1
    hi = (j0 + n_out - 1) * (D // 2) + 1
    i = np.arange(lo, hi)
    v = np.zeros(i.size)
    inside = (i >= first) & (i < first + x.size)
    v[inside] = x[i[inside] - first]
    m = v * np.exp(-2j * np.pi * fc * i.astype(np.float64))
    z = np.convolve(m, h)[h.size - 1:h.size - 1 + i.size - h.size + 1]   # z at i = lo + Lh - 1 ...
    iz = i[h.size - 1:]
    s = z * np.exp(2j * np.pi * iz / (2 * D))
    y_full = 2 * g * s.real
    keep = (iz % (D // 2) == 0)
    return y_full[keep][:n_out]


def test_ddc_matches_stepwise_pipeline():
    g = np.random.default_rng(5)
    for D, Th, fc in ((8, 8, 0.2), (4, 16, 0.37), (16, 4, 0.05)):
        x = g.integers(-512, 512, 6000).astype(np.int32)
        h = O.ddc_weights(D, Th)
        first, j0, n_out = 1000, 0, 900     # outputs from before the stream: zeros there
        y, q = O.ddc(x, first, D, h, fc, 1.7, j0, n_out)
        ref = _ddc_stepwise(x, first, D, h, fc, 1.7, j0, n_out)
        np.testing.assert_allclose(y, ref, rtol=1e-9, atol=1e-9)
        np.testing.assert_array_equal(q, [O.quantise10(v) for v in y])


def test_ddc_tone_closed_form():
    """A tone A cos(2 pi f i + psi) comes out as 2 g Re(i^j (A/2) [e^{i psi}
    e^{2 pi i (f - fc) i} H(f - fc) + e^{-i psi} e^{-2 pi i (f + fc) i} H(-f - fc)])
    at i = j D / 2, H the transform of the low-pass; only the input's
    rounding to integers is left (|error| <= g sum |h|)."""
    D, Th, fc, g = 8, 16, 0.21, 0.8
    h = O.ddc_weights(D, Th)
    u = np.arange(h.size)
    Hf = lambda nu: np.sum(h * np.exp(-2j * np.pi * nu * u))
    for f, A, psi in ((0.21 + 0.02, 400.0, 0.4), (0.21 - 0.045, 300.0, 2.0), (0.21, 450.0, -1.0)):
        n = 1 << 14
        i = np.arange(n)
        x = np.rint(A * np.cos(2 * np.pi * f * i + psi)).astype(np.int32)
        j0 = h.size          # windows inside the stream
        n_out = 2000
        y, _ = O.ddc(x, 0, D, h, fc, g, j0, n_out)
        j = np.arange(j0, j0 + n_out)
        t = j * (D // 2)
        zz = (A / 2) * (np.exp(1j * psi) * np.exp(2j * np.pi * (f - fc) * t) * Hf(f - fc)
                        + np.exp(-1j * psi) * np.exp(-2j * np.pi * (f + fc) * t) * Hf(-f - fc))
        pred = 2 * g * (1j ** (j % 4) * zz).real
        assert np.max(np.abs(y - pred)) <= g * np.sum(np.abs(h)) + 1e-9


def test_quantise10_ties_and_saturation():
    for x, q in ((10.5, 11), (-10.5, -11), (10.49, 10), (0.5, 1), (-0.5, -1), (510.5, 511),
                 (511.5, 511), (-600.0, -511), (1e9, 511)):
        assert O.quantise10(x) == q
