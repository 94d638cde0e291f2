"""GPU parity of the narrow-band front end (the library's reading of the
narrow-band mode Sec. 6 names: mix, low-pass, shift the band's lower edge to
0, real part, decimate by D/2, requantise to 10 bits) against the FP64
oracle, and of the narrow-band channelizer built from it.

Bars: the output before requantisation within relative RMS 1e-5 of the
oracle (the FP32 bar of the channelizer); the 10-bit codes within 1 LSB
(exact fraction printed) and exactly the requantiser (R15) of the GPU's own
FP32 output; the packed bytes exactly the 10-bit packing of those codes;
bit-identical output for different chunk lengths (the history carries the
low-pass's window across calls)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_09886_gb300 import fengine, synth
from tests.fe_harness import streams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_09886_gb300 import build
    build.build()
    fengine.load()


def _run(samples, D, Th, L, fc, g, n_chunks, filt=None):
    """Chunks of `samples` [ant, pol, n] through one DDC; returns per chunk
    (packed bytes [ant, pol, 5L'/4], float [ant, pol, L'])."""
    import torch
    n_ant = samples.shape[0]
    ddc = fengine.DDC(n_ant, D, Th, L, fc, g, filter=filt)
    Lo = ddc.out_samples
    res = []
    for c in range(n_chunks):
        pk = np.stack([np.stack([synth.pack10(samples[a, p, c * L:(c + 1) * L]) for p in range(2)])
                       for a in range(n_ant)])
        d_out = torch.empty((n_ant, 2, Lo * 5 // 4), dtype=torch.uint8, device="cuda")
        d_f = torch.empty((n_ant, 2, Lo), dtype=torch.float32, device="cuda")
        ddc.process(torch.from_numpy(pk).cuda(), c * L, d_out, d_f)
        torch.cuda.synchronize()
        res.append((d_out.cpu().numpy(), d_f.cpu().numpy()))
    ddc.close()
    return res


@pytest.mark.parametrize("D,Th,fc,g", [(8, 16, 0.2, 0.9), (4, 16, 0.37, 2.0), (32, 4, 0.05, 1.0),
                                       (2, 64, 0.25, 0.5), (16, 8, 0.4375, 3.0)])
def test_down_converter_matches_oracle(D, Th, fc, g):
    n_ant, L, n_chunks = 2, 1 << 15, 3
    s = streams(synth.SEED_BASE + 900 + D, n_ant, n_chunks * L, 40.0,
                tones=[(fc + 0.3 / D, 120.0, 0.2), (fc - 0.1 / D, 60.0, 1.0), (0.11, 80.0, 0.0)])
    res = _run(s, D, Th, L, fc, g, n_chunks)
    h = O.ddc_weights(D, Th)
    Lo = 2 * L // D
    exact = total = 0
    worst = 0.0
    for c, (packed, yf) in enumerate(res):
        for a in range(n_ant):
            for p in range(2):
                y_o, q_o = O.ddc(s[a, p].astype(np.int32), 0, D, h, fc, g, c * Lo, Lo)
                y = yf[a, p].astype(np.float64)
                rel = np.sqrt(np.sum((y - y_o) ** 2) / np.sum(y_o ** 2))
                worst = max(worst, rel)
                assert rel <= 1e-5, f"chunk {c} stream {a},{p}: relative RMS {rel:.3g}"
                q = O.unpack10(packed[a, p], Lo)
                np.testing.assert_array_equal(q, [O.quantise10(v) for v in yf[a, p]],
                                              err_msg="requantiser / packing of the GPU's own output")
                d = np.abs(q - q_o)
                assert d.max() <= 1
                exact += int(np.sum(d == 0))
                total += d.size
    print(f"[narrow-band] D={D} Th={Th} fc={fc}: rel_rms={worst:.3g} exact_10bit={exact / total:.6f}")


def test_down_converter_chunking_invariance():
    D, Th, fc = 8, 16, 0.3
    L = 1 << 14
    s = streams(synth.SEED_BASE + 950, 1, 8 * L, 50.0, tones=[(0.31, 100.0, 0.5)])
    small = np.concatenate([r[0] for r in _run(s, D, Th, L, fc, 1.0, 8)], axis=-1)
    large = np.concatenate([r[0] for r in _run(s, D, Th, 4 * L, fc, 1.0, 2)], axis=-1)
    np.testing.assert_array_equal(small, large)


def test_narrow_band_channelizer_puts_a_tone_in_its_channel():
    """Down-converter + an ordinary 1024-channel plan on its output: a tone at
    input frequency f appears at (f - fc) D/2 + 1/4 cycles per output sample,
    i.e. in narrow-band channel ((f - fc) D/2 + 1/4) N', and nowhere else
    above the PFB's own leakage."""
    import torch
    D, Th, fc, n_nb, T = 8, 16, 0.2, 1024, 16
    N = 2 * n_nb
    k_tone = 300
    f = fc + (k_tone / N - 0.25) * 2 / D            # bin-centred in the narrow band
    L = 1 << 20
    s = streams(synth.SEED_BASE + 960, 1, 2 * L, 8.0, tones=[(f, 200.0, 0.3)])
    res = _run(s, D, Th, L, fc, 1.0, 2)
    Lo = 2 * L // D
    plan = fengine.Plan(1, n_nb, T, Lo, max_delay_samples=0)
    pre = []
    for c, (packed, _) in enumerate(res):
        d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
        d_pre = torch.empty(2 * plan.M * n_nb * 2, dtype=torch.float32, device="cuda")
        plan.process(torch.from_numpy(packed).cuda(), c * Lo, d_out, d_pre)
        torch.cuda.synchronize()
        pre.append(d_pre.cpu().numpy().view(np.complex64).reshape(2, plan.M, n_nb))
    plan.close()
    power = np.mean(np.abs(pre[1]) ** 2, axis=(0, 1))          # second chunk: history filled
    assert int(np.argmax(power)) == k_tone
    others = np.delete(power, [k_tone - 1, k_tone, k_tone + 1])
    ratio = 10 * np.log10(others.max() / power[k_tone])
    print(f"[narrow-band] tone in channel {k_tone}: next strongest channel {ratio:.1f} dB")
    assert ratio < -30.0
