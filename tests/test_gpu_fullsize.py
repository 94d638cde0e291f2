"""Full size: the seeded workloads at their own sizes, on the GPU, in the
launch configuration bench.py times, against the FP64 oracle on sampled
spectra.

  * config 2 (4 antennas x 2 pol x 2^25 samples/pol, 8192 channels, 16 taps,
    3 tones, random delays and gains) with the work splits the autotuner
    picks for it (fft_n1 = 16 and 64, the whole chunk in one slab), in every
    precision;
  * config 3 (1 antenna x 2 pol x 2^28 samples/pol, 32768 channels, a chirp
    across the chunk, delay rate 5e-9 so that the coarse delay steps twice
    inside the chunk) with fft_n1 = 64 (the built-in split, and the one the
    tensor-core second stage takes for N = 65536), built-in slabs and the
    whole chunk in one slab.

Sampled spectra of every stream -- the first ones (windows reaching into the
zero history), tile and slab boundaries, both sides of every coarse-delay
step and the last -- are recomputed one by one by the oracle: pre-quantisation
relative RMS within the form's bar, int8 within 1 LSB (the exact fraction is
printed), and the int8 output is exactly the requantiser of the GPU's own
spectra."""
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


def _coarse_steps(wl):
    """Spectra m at which the coarse delay of some stream differs from m - 1."""
    out = set()
    m = np.arange(wl.chunk_samples // wl.N + 1)
    for a, p, d, r, ph, pr in wl.delays():
        c = np.floor(d + r * wl.N * m + 0.5)
        out.update(int(x) + 1 for x in np.nonzero(np.diff(c))[0])
    return sorted(out)


def _check(index, precision, fft_n1=0, slab=0, sampled=()):
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
    torch.cuda.synchronize()
    info = plan.info
    plan.close()

    # sampled spectra (relative to the first one emitted): the fixed list plus
    # both sides of every coarse-delay step inside the chunk
    qs = {q for q in sampled if 0 <= q < M} | {M - 1}
    for m in _coarse_steps(wl):
        qs.update(q for q in (m - 1 - m0, m - m0) if 0 <= q < M)
    qs = sorted(qs)
    pre = d_pre.view(wl.n_antennas, 2, M, n, 2)[:, :, qs].cpu().numpy().astype(np.float64)
    pre = pre[..., 0] + 1j * pre[..., 1]
    out = d_out.view(wl.n_antennas, -1).cpu().numpy()
    del d_out, d_pre

    w = O.pfb_weights(N, T)
    bar = REL_RMS_FP32 if precision == fengine.FP32 else REL_RMS_REDUCED
    num = den = 0.0
    exact = total = 0
    worst = (0.0, None)
    lsb = []
    for a in range(wl.n_antennas):
        for p in range(2):
            gp = np.ones(n) if g is None else g[a, p]
            for i, q in enumerate(qs):
                # only the samples around the window [N m - c, N m - c + N T)
                lo = max(0, N * (m0 + q) - 2 * wl.max_delay - N)
                hi = min(L, N * (m0 + q) + N * T + 2 * wl.max_delay + N)
                ref, qo, _ = O.channelize(samples[a, p, lo:hi].astype(np.int32), lo, N, T, w,
                                          oracle_model(segs[(a, p)]), gp, m0 + q, 1)
                got = pre[a, p, i]
                num += np.sum(np.abs(got - ref[0]) ** 2)
                den += np.sum(np.abs(ref[0]) ** 2)
                err = np.maximum(np.abs(got.real - ref[0].real), np.abs(got.imag - ref[0].imag))
                k = int(np.argmax(err))
                if err[k] > worst[0]:
                    worst = (float(err[k]), (a, p, m0 + q, k, complex(ref[0][k]), complex(got[k])))
                # the heap cells of spectrum q, pol p: out[heap][k][s][pol][re, im]
                h, s_ = divmod(q, S)
                Sh = min(S, M - h * S)
                cells = out[a][h * S * n * 4:h * S * n * 4 + n * Sh * 4].reshape(n, Sh, 2, 2)[:, s_, p, :]
                d = np.abs(cells.astype(np.int16) - qo[0].astype(np.int16))
                lsb.append(int(d.max()))
                exact += int(np.sum(d == 0))
                total += d.size
                comp = np.stack([got.real, got.imag], axis=-1)
                rq = np.clip(np.where(comp >= 0, np.floor(comp + 0.5), -np.floor(-comp + 0.5)), -127, 127)
                np.testing.assert_array_equal(cells, rq.astype(np.int8))
    rel = np.sqrt(num / den)
    print(f"[parity] {wl.name} full size, precision {precision}, split (n1 {info.fft_n1}, slab {info.slab_spectra}), "
          f"{len(qs)} spectra/stream: rel_rms={rel:.3g} exact_int8={exact / total:.6f} "
          f"max_component_error={worst[0]:.3g} at (ant, pol, spectrum, channel, oracle, gpu)={worst[1]}")
    assert rel <= bar
    assert max(lsb) <= 1, f"int8 output differs by {max(lsb)} LSB"


@pytest.mark.parametrize("precision,fft_n1", [(fengine.FP32, 16), (fengine.FP32, 64), (fengine.TC_FP16, 16),
                                              (fengine.TC_BF16, 16)])
def test_config2_full_size_sampled_against_the_oracle(precision, fft_n1):
    _check(2, precision, fft_n1=fft_n1, slab=2048, sampled=[0, 1, 14, 15, 31, 32, 33, 1023, 1024, 2046])


@pytest.mark.parametrize("precision,slab", [(fengine.FP32, 0), (fengine.FP32, 4096), (fengine.TC_FP16, 0),
                                            (fengine.TC_BF16, 0)])
def test_config3_full_size_sampled_against_the_oracle(precision, slab):
    _check(3, precision, fft_n1=64, slab=slab, sampled=[0, 1, 31, 32, 2047, 2048])
