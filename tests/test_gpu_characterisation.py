"""Precision and channel-response characterisation of the three forms on the
GPU, through the C ABI, after the paper's two experiments.

Spur test (Sec. 3.5, FFT precision): a tone in channel 192 of 1024 is
quantised to 10 bits with a uniform dither and channelized many times; the
complex spectra are averaged in FP64 and squared to power. Dither noise
averages down with the number of spectra, while rounding errors of the
arithmetic that are data-dependent (non-zero mean) stay and show up as
spurs. Each form's averaged spectrum is compared with the oracle's on the
same bytes: their difference is the coherent error the form adds, in dB
relative to the tone's power (the paper saw harmonics at about -75 dB with
an FP16 FFT).

Channel response (Sec. 5.2): a common full-scale tone in both
polarisations with independent dither, swept in sub-channel steps;
cross-correlating the two polarisations removes the dither noise from the
average, and the power in channel k is compared with (A/2)^2 |W(k/N - f)|^2,
W the Fourier transform of the PFB weights (computed from the same weights
in FP64), for 1024 and 32768 channels with 16 taps."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_09886_gb300 import fengine, synth
from tests.fe_harness import default_delays, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

FORMS = {"fp32": fengine.FP32, "fp16": fengine.TC_FP16, "bf16": fengine.TC_BF16}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_09886_gb300 import build
    build.build()
    fengine.load()


def _db(x):
    return 10.0 * np.log10(np.maximum(x, 1e-300))


def test_spur_level_of_each_form():
    n, T, k0, A = 1024, 16, 192, 500.0
    N = 2 * n
    n_ant, M = 2, 1024
    L = N * M
    f = k0 / N                              # bin-centred: every spectrum sees the same tone phase
    s = np.stack([np.stack([synth.dithered_tone(synth.SEED_BASE + 300 + 2 * a + p, L, f, A, 0.3)
                            for p in range(2)]) for a in range(n_ant)])
    w = O.pfb_weights(N, T).astype(np.float32)
    delays = default_delays(n_ant)
    avg, m0 = {}, None
    for name, prec in FORMS.items():
        res, M_, _ = run_gpu(s, n, T, L, 1, delays, None, weights=w, taps=False, precision=prec)
        m0 = res[0]["m0"]
        keep = slice(-m0, None)             # spectra whose window lies after sample 0
        avg[name] = res[0]["pre"][:, :, keep].astype(np.complex128).reshape(-1, n).mean(axis=0)
    pre_o, _, _ = run_oracle(s, n, T, delays, None, m0, M, weights=w.astype(np.float64))
    avg["oracle"] = pre_o[:, :, -m0:].reshape(-1, n).mean(axis=0)
    p_tone = np.abs(avg["oracle"][k0]) ** 2
    # the channels the tone's own response reaches above -130 dB are not spurs
    W = np.abs(np.fft.fft(O.pfb_weights(N, T))) ** 2
    lobe = np.array([W[(k - k0) * T % (N * T)] / W[0] for k in range(n)]) > 1e-13
    floor = {}
    for name, a in avg.items():
        lvl = _db(np.abs(a) ** 2 / p_tone)
        floor[name] = float(np.max(lvl[~lobe]))
    coherent = {name: float(np.max(_db(np.abs(avg[name] - avg["oracle"]) ** 2 / p_tone)))
                for name in FORMS}
    iters = n_ant * 2 * (M + m0)
    print(f"[spur] tone ch {k0}/{n}, A={A}, {iters} averaged spectra; largest level outside the "
          f"tone's response (dB): " + ", ".join(f"{k} {v:.1f}" for k, v in floor.items()))
    print("[spur] coherent error against the oracle, largest channel (dB): "
          + ", ".join(f"{k} {v:.1f}" for k, v in coherent.items()))
    # the FP32 form sits at the oracle's dither floor; its own rounding is far below it
    assert abs(floor["fp32"] - floor["oracle"]) < 1.0
    assert coherent["fp32"] < -135.0
    # the tensor-core forms: 20 dB (FP16) and 45 dB (BF16) below the spurs the
    # paper saw with an FP16 FFT (about -75 dB); measured -95 and -125 dB
    assert coherent["fp16"] < -90.0
    assert coherent["bf16"] < -115.0


@pytest.mark.parametrize("n,L", [(1024, 1 << 22), (32768, 1 << 22)])
def test_channel_response_sub_channel_sweep(n, L):
    T, A, steps = 16, 500.0, 16      # the weights' FFT (N T points) samples W every 1/T channel
    assert steps == T
    N = 2 * n
    k0 = n // 4                                # image of the tone far outside the compared channels
    K = 24                                     # channels compared on each side of k0
    w = O.pfb_weights(N, T)
    # |W(nu)|^2 on a grid of 1/16 channel: the FFT of the N T weights has that spacing for T = 16
    Wp = np.abs(np.fft.fft(w)) ** 2
    ks = np.arange(k0 - K, k0 + K + 1)
    delays = default_delays(1)
    worst = {name: {60: 0.0, 90: 0.0} for name in FORMS}
    for j in range(steps):
        f = (k0 + j / steps) / N
        s = np.stack([np.stack([synth.dithered_tone(synth.SEED_BASE + 400 + 2 * j + p, L, f, A, 0.7)
                                for p in range(2)])])
        # nu = k/N - f = (steps (k - k0) - j) / (steps N)
        pred = (A / 2) ** 2 * Wp[(steps * (ks - k0) - j) % (N * T)]
        pred_db = _db(pred / ((A / 2) ** 2 * Wp[0]))
        for name, prec in FORMS.items():
            res, M_, _ = run_gpu(s, n, T, L, 1, delays, None, weights=w.astype(np.float32), taps=False,
                                 precision=prec)
            x = res[0]["pre"][0, :, -res[0]["m0"]:, :].astype(np.complex128)
            c = np.abs(np.mean(x[0][:, ks] * np.conj(x[1][:, ks]), axis=0))
            dev = np.abs(_db(c) - _db(pred))
            for lim in (60, 90):
                sel = pred_db >= -lim
                worst[name][lim] = max(worst[name][lim], float(np.max(dev[sel])))
    print(f"[response] n={n}: largest |measured - |W|^2| in dB over {steps} sub-channel offsets x "
          f"{2 * K + 1} channels, where the response is above -60 / -90 dB: "
          + ", ".join(f"{k} {v[60]:.3f} / {v[90]:.3f}" for k, v in worst.items()))
    # measured: FP32 0.003 / 0.16 dB, FP16 0.014 / 0.38, BF16 0.003 / 0.16 (the
    # -90 dB figures are the dither noise left in the cross-correlation)
    assert worst["fp32"][60] < 0.02 and worst["fp32"][90] < 0.3
    for name in ("fp16", "bf16"):
        assert worst[name][60] < 0.05 and worst[name][90] < 0.6
