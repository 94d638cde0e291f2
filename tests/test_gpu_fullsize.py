"""Full size: the seeded workloads at their own sizes, on the GPU, in the
launch configuration bench.py times, compared with the FP64 oracle in full
-- every spectrum of every stream:

  * config 1 (1 antenna x 2 pol x 2^20 samples/pol, 1024 channels, 16 taps,
    a bin-centred tone of amplitude 100 that saturates its channel, coarse
    delay 7, fine delay 0.3, phase 0.1) in every precision;
  * config 2 (4 antennas x 2 pol x 2^25 samples/pol, 8192 channels, 16 taps,
    3 tones, random delays and gains) with the whole chunk in one slab (the
    split the autotuner picks for it) and fft_n1 = 16 and 64 in the FP32
    form, in every precision;
  * config 3 (1 antenna x 2 pol x 2^28 samples/pol, 32768 channels, a chirp
    across the chunk, delay rate 5e-9 so that the coarse delay steps twice
    inside the chunk) with built-in slabs and the whole chunk in one slab.

Per form: pre-quantisation relative RMS within the form's bar, int8 within
1 LSB with the exact fraction printed, and the int8 output exactly the
requantiser of the GPU's own spectra."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_09886_gb300 import fengine, synth
from paper_2303_09886_gb300.workloads import WORKLOADS
from tests.fe_harness import REL_RMS_FP32, REL_RMS_REDUCED, oracle_model, Seg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_09886_gb300 import build
    build.build()
    fengine.load()


_cache = {}


def _workload(index):
    if index not in _cache:
        _cache.clear()
        wl = WORKLOADS[index]
        samples = np.stack([np.stack([wl.samples(a, p) for p in range(2)]) for a in range(wl.n_antennas)])
        packed = np.stack([np.stack([synth.pack10(samples[a, p]) for p in range(2)]) for a in range(wl.n_antennas)])
        _cache[index] = (wl, samples, packed)
    return _cache[index]


def _check(index, precision, fft_n1=0, slab=0):
    import torch
    wl, samples, packed = _workload(index)
    n, N, T, L = wl.n_channels, wl.N, wl.n_taps, wl.chunk_samples
    plan = fengine.Plan(wl.n_antennas, n, T, L, spectra_per_heap=wl.spectra_per_heap,
                        max_delay_samples=wl.max_delay, precision=precision, fft_n1=fft_n1, slab_spectra=slab)
    segs = {}
    for a, p, d, r, ph, pr in wl.delays():
        plan.set_delay(a, p, d, r, ph, pr)
        segs[(a, p)] = [Seg(delay=d, rate=r, phase=ph, phase_rate=pr)]
    g = wl.gains()
    if g is not None:
        for a in range(wl.n_antennas):
            for p in range(2):
                plan.set_gains(a, p, g[a, p])
    M, S = plan.M, plan.S
    d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
    d_pre = torch.empty(wl.n_antennas * 2 * M * n * 2, dtype=torch.float32, device="cuda")
    m0 = plan.process(torch.from_numpy(packed).cuda(), 0, d_out, d_pre)
    plan.device_status()
    info = plan.info
    plan.close()
    out = d_out.view(wl.n_antennas, -1).cpu().numpy()
    del d_out

    w = O.pfb_weights(N, T)
    bar = REL_RMS_FP32 if precision == fengine.FP32 else REL_RMS_REDUCED
    num = den = 0.0
    exact = total = 0
    worst = (0.0, None)
    max_lsb = 0
    for a in range(wl.n_antennas):
        q = []
        for p in range(2):
            gp = np.ones(n) if g is None else g[a, p]
            ref, qo, _ = O.channelize(samples[a, p].astype(np.int32), 0, N, T, w, oracle_model(segs[(a, p)]),
                                      gp, m0, M)
            got = d_pre[(2 * a + p) * M * n * 2:(2 * a + p + 1) * M * n * 2].cpu().numpy().astype(np.float64)
            got = (got[0::2] + 1j * got[1::2]).reshape(M, n)
            num += float(np.sum(np.abs(got - ref) ** 2))
            den += float(np.sum(np.abs(ref) ** 2))
            err = np.maximum(np.abs(got.real - ref.real), np.abs(got.imag - ref.imag))
            k = np.unravel_index(int(np.argmax(err)), err.shape)
            if err[k] > worst[0]:
                worst = (float(err[k]), (a, p, m0 + int(k[0]), int(k[1]), complex(ref[k]), complex(got[k])))
            # the requantiser: the int8 output is R7 of the GPU's own spectra
            comp = np.stack([got.real, got.imag], axis=-1)
            rq = np.clip(np.where(comp >= 0, np.floor(comp + 0.5), -np.floor(-comp + 0.5)), -127, 127)
            q.append((qo, rq.astype(np.int8)))
            del ref, got, err, comp, rq
        ref_heaps = O.corner_turn(q[0][0], q[1][0], S)
        d = np.abs(out[a].astype(np.int16) - ref_heaps.astype(np.int16))
        max_lsb = max(max_lsb, int(d.max()))
        exact += int(np.sum(d == 0))
        total += d.size
        np.testing.assert_array_equal(out[a], O.corner_turn(q[0][1], q[1][1], S), err_msg=f"requantiser ant {a}")
        del q, ref_heaps, d
    rel = np.sqrt(num / den)
    print(f"[parity] {wl.name} full size, every spectrum ({M} per stream), precision {precision}, "
          f"split (n1 {info.fft_n1}, slab {info.slab_spectra}): rel_rms={rel:.3g} exact_int8={exact / total:.6f} "
          f"max_component_error={worst[0]:.3g} at (ant, pol, spectrum, channel, oracle, gpu)={worst[1]}")
    assert rel <= bar
    assert max_lsb <= 1, f"int8 output differs by {max_lsb} LSB"


@pytest.mark.parametrize("precision", [fengine.FP32, fengine.TC_FP16, fengine.TC_BF16])
def test_config1_full_size_every_spectrum(precision):
    _check(1, precision)


@pytest.mark.parametrize("precision,fft_n1", [(fengine.FP32, 16), (fengine.FP32, 64), (fengine.TC_FP16, 0),
                                              (fengine.TC_BF16, 0)])
def test_config2_full_size_every_spectrum(precision, fft_n1):
    _check(2, precision, fft_n1=fft_n1, slab=2048)


@pytest.mark.parametrize("precision,slab", [(fengine.FP32, 0), (fengine.FP32, 4096), (fengine.TC_FP16, 0),
                                            (fengine.TC_BF16, 0)])
def test_config3_full_size_every_spectrum(precision, slab):
    _check(3, precision, fft_n1=64 if precision == fengine.FP32 else 0, slab=slab)
