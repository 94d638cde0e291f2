"""Why the tensor-core second stage splits its operands (no GPU needed).

The reduced-precision forms compute the 1024-point DFT of a class sequence
as two 32-point DFT contractions (t2 = 32 a + b, k2 = c + 32 d):
Y = W32 . B, Y' = twiddle * Y, F = Y' . W32^T. This model replays that order
in numpy with FP16 rounding at the points the kernel rounds (the FP16
intermediate B, the DFT matrices, the data between the contractions) and
measures the largest error of F relative to the largest channel of the
sequence, for sequences that hold two strong tones over weak noise (a strong
tone dominates its class sequence in the workloads). With single FP16
operands the error reaches ~1e-4 of the tone: an 8-bit output next to a
tone of amplitude 1e4 is then off by more than 1 LSB. Carrying the DFT
matrices and the mid data as hi + lo pairs (2 products in contraction 1,
3 in contraction 2) leaves the FP16 intermediate's own rounding, a few 1e-5.
"""
import numpy as np

n = np.arange(32)
W = np.exp(-2j * np.pi * np.outer(n, n) / 32)
TW = np.exp(-2j * np.pi * np.outer(n, n) / 1024) / 32


def h16(x):
    return x.real.astype(np.float16).astype(np.float64) + 1j * x.imag.astype(np.float16).astype(np.float64)


def split(x):
    hi = h16(x)
    return hi, h16(x - hi)


def single(x):
    X = h16(x).reshape(32, 32)            # [a][b]
    Y = h16(h16(W) @ X * TW)
    F = Y @ h16(W).T
    return (32 * F).T.reshape(-1)        # k2 = c + 32 d


def split_form(x):
    X = h16(x).reshape(32, 32)
    Wh, Wl = split(W)
    Yh, Yl = split((Wh @ X + Wl @ X) * TW)
    F = Yh @ Wh.T + Yh @ Wl.T + Yl @ Wh.T
    return (32 * F).T.reshape(-1)


def _errors(seeds):
    t = np.arange(1024)
    out = []
    for seed in seeds:
        g = np.random.default_rng(seed)
        x = g.normal(size=1024) + 1j * g.normal(size=1024)
        for k, A in zip(g.uniform(0, 1024, 2), (58.0, 96.0)):
            x = x + A * np.exp(2j * np.pi * k * t / 1024 + 1j * g.uniform(0, 2 * np.pi))
        ref = np.fft.fft(x)
        top = np.abs(ref).max()
        out.append((np.abs(single(x) - ref).max() / top, np.abs(split_form(x) - ref).max() / top))
    return np.array(out)


def test_contraction_order_reproduces_the_fft():
    x = np.random.default_rng(0).normal(size=1024) + 0j
    Y = (W @ x.reshape(32, 32)) * TW
    F = (32 * (Y @ W.T)).T.reshape(-1)
    np.testing.assert_allclose(F, np.fft.fft(x), rtol=0, atol=1e-9)


def test_single_fp16_operands_miss_the_8bit_bar_next_to_tones_and_split_operands_meet_it():
    e = _errors(range(40))
    # single FP16 operands: errors of the order of 1e-4 of the strongest channel
    assert e[:, 0].max() > 1e-4
    assert np.median(e[:, 0]) > 5e-5
    # split operands: only the FP16 intermediate's rounding is left
    assert e[:, 1].max() < 5e-5
    assert np.all(e[:, 1] < e[:, 0] / 2)
