"""Where the FP16 tensor-core form's error comes from (no GPU needed).

The FP16 form computes the FIR and the first DFT stage as one contraction
per output column t2, B[k1][t2] = sum_k x[t2 + P k] W_t2[k][k1], with the
data exact in FP16 (10-bit integers), the operand block W_t2 (weights x DFT
x twiddle) rounded to FP16 after a power-of-two scale of its own, FP32
accumulation, and B stored as FP16 after one global power-of-two scale;
the second stage is FP32. This model replays those roundings in numpy on a
1024-channel, 16-tap PFB (N1 = 8, N2 = 256) and checks that

  * the relative RMS error of the spectra sits far inside the 2e-3 bar,
    at the level the GPU measures for the FP16 form (a few 1e-4);
  * the two FP16 roundings contribute errors of the same order, and
    neither scale leaves the FP16 range;
  * the BF16 form's hi + lo split of data and operands (three products)
    brings the contraction's error down by more than an order of magnitude.
"""
import numpy as np

from oracle import oracle as O

N, T, N1 = 2048, 16, 8
P, N2 = N // 8, N // N1
n = N // 2


def _f16(a):
    return a.astype(np.float16).astype(np.float64)


def _bf16(a):
    """Round to BF16 (8 significant bits), nearest even, via the FP32 bit pattern."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _operands():
    w = O.pfb_weights(N, T)
    k = np.arange(8 * T)
    Wt = np.empty((P, 8 * T, N1), np.complex128)
    for t in range(P):
        ph = np.outer(P * (k % 8) + t, np.arange(N1)) / N
        Wt[t] = w[t + P * k][:, None] * np.exp(-2j * np.pi * ph)
    return w, Wt


def _spectra(x, Wt, mode):
    """Spectra k < n of windows x[m] (rows: spectra) in one of the forms."""
    M = x.shape[0]
    k = np.arange(8 * T)
    A = np.stack([x[:, t + P * k] for t in range(P)], axis=1)       # [m][t][k]
    if mode == "exact":
        B = np.einsum("mtk,tkc->mct", A, Wt)
    else:
        # per-column power of two: the block's largest entry just below 2^15
        bmax = np.max(np.abs(np.concatenate([Wt.real, Wt.imag], axis=1)), axis=(1, 2))
        sB = 2.0 ** np.floor(np.log2(32768.0 / bmax))
        Ws = Wt * sB[:, None, None]
        if mode == "fp16":
            Wq = _f16(Ws.real) + 1j * _f16(Ws.imag)
            B = np.einsum("mtk,tkc->mct", A, Wq) / sB[None, None, :]
            # the FP16 intermediate, one global power of two from |B| <= 512 sum |w|
            bound = 512.0 * np.max(np.sum(np.abs(Wt), axis=1))
            s_int = 2.0 ** np.floor(np.log2(32768.0 / bound))
            assert np.max(np.abs(Ws)) < 65504 and np.max(np.abs(B)) * s_int < 65504
            B = (_f16(B.real * s_int) + 1j * _f16(B.imag * s_int)) / s_int
        elif mode == "fp16_operands_only":
            Wq = _f16(Ws.real) + 1j * _f16(Ws.imag)
            B = np.einsum("mtk,tkc->mct", A, Wq) / sB[None, None, :]
        else:   # bf16: x = x_hi + x_lo, W = W_hi + W_lo, three products
            xh = _bf16(A)
            xl = A - xh
            Wh = _bf16(Ws.real) + 1j * _bf16(Ws.imag)
            Wl = (_bf16(Ws.real - Wh.real) + 1j * _bf16(Ws.imag - Wh.imag))
            B = (np.einsum("mtk,tkc->mct", xh, Wh) + np.einsum("mtk,tkc->mct", xl, Wh)
                 + np.einsum("mtk,tkc->mct", xh, Wl)) / sB[None, None, :]
    # second stage (exact here): X[k1 + N1 k2] = sum_t2 exp(-2 pi i k2 t2 / N2) B[k1][t2]
    X = np.fft.fft(B, axis=2)                                       # [m][k1][k2]
    X = X.transpose(0, 2, 1).reshape(M, N)                          # index k1 + N1 k2
    return X[:, :n]


def test_fp16_form_error_budget():
    g = np.random.default_rng(3)
    M = 24
    i = np.arange(M * N + N * T)
    sig = 40 * g.standard_normal(i.size) + 90 * np.cos(2 * np.pi * 0.1234 * i)
    s = np.clip(np.rint(sig), -512, 511)
    x = np.stack([s[m * N:m * N + N * T] for m in range(M)])
    w, Wt = _operands()
    ref = _spectra(x, Wt, "exact")
    # the exact contraction is the PFB + DFT itself (closed form of Eq. 1 + DFT)
    g_fir = np.stack([np.sum((w * x[m]).reshape(T, N), axis=0) for m in range(M)])
    np.testing.assert_allclose(ref, np.fft.fft(g_fir, axis=1)[:, :n], rtol=0, atol=1e-8 * np.abs(ref).max())

    def rel(a):
        return np.sqrt(np.sum(np.abs(a - ref) ** 2) / np.sum(np.abs(ref) ** 2))

    e16, e_op, ebf = rel(_spectra(x, Wt, "fp16")), rel(_spectra(x, Wt, "fp16_operands_only")), \
        rel(_spectra(x, Wt, "bf16"))
    print(f"[precision model] FP16 form {e16:.3g} (operand rounding alone {e_op:.3g}), BF16 form {ebf:.3g}")
    assert 3e-5 < e16 < 5e-4                     # the GPU measures 2e-4 .. 3e-4; the bar is 2e-3
    assert 0.2 < e_op / e16 < 0.95               # both roundings matter, neither alone explains it
    assert ebf < e16 / 10
