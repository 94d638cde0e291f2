"""Full size, in the launch configuration bench.py times: config 2 (4 antennas
x 2 pol x 2^25 samples/pol, 8192 channels, 16 taps, random delays and gains,
the seeded workload of the bench) with the work split the autotuner picks for
it (fft_n1 = 16, the whole chunk in one slab). Sampled spectra of every
stream -- the first ones (windows reaching into the zero history), slab-tile
boundaries and the last -- are recomputed one by one by the FP64 oracle:
pre-quantisation relative RMS within the form's bar, int8 within 1 LSB, and
the int8 output is exactly the requantiser of the GPU's own spectra."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_09886_gb300 import fengine, synth
from paper_2303_09886_gb300.workloads import WORKLOADS
from tests.fe_harness import REL_RMS_FP32, REL_RMS_REDUCED, oracle_model, Seg

pytestmark = pytest.mark.gpu

SAMPLED = [0, 1, 14, 15, 31, 32, 33, 1023, 1024, 2046, 2047]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_09886_gb300 import build
    build.build()
    fengine.load()


@pytest.fixture(scope="module")
def workload():
    wl = WORKLOADS[2]
    samples = np.stack([np.stack([wl.samples(a, p) for p in range(2)]) for a in range(wl.n_antennas)])
    packed = np.stack([np.stack([synth.pack10(samples[a, p]) for p in range(2)]) for a in range(wl.n_antennas)])
    return wl, samples, packed


@pytest.mark.parametrize("precision", [fengine.FP32, fengine.TC_FP16, fengine.TC_BF16])
def test_config2_full_size_sampled_against_the_oracle(workload, precision):
    import torch
    wl, samples, packed = workload
    n, N, T, L = wl.n_channels, wl.N, wl.n_taps, wl.chunk_samples
    plan = fengine.Plan(wl.n_antennas, n, T, L, spectra_per_heap=wl.spectra_per_heap,
                        max_delay_samples=wl.max_delay, precision=precision, fft_n1=16, slab_spectra=2048)
    assert plan.info.slabs_per_chunk == 1
    segs = {}
    for a, p, d, r, ph, pr in wl.delays():
        plan.set_delay(a, p, d, r, ph, pr)
        segs[(a, p)] = [Seg(delay=d, rate=r, phase=ph, phase_rate=pr)]
    g = wl.gains()
    for a in range(wl.n_antennas):
        for p in range(2):
            plan.set_gains(a, p, g[a, p])
    M, S = plan.M, plan.S
    d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
    d_pre = torch.empty(wl.n_antennas * 2 * M * n * 2, dtype=torch.float32, device="cuda")
    m0 = plan.process(torch.from_numpy(packed).cuda(), 0, d_out, d_pre)
    torch.cuda.synchronize()
    out = d_out.cpu().numpy().reshape(wl.n_antennas, -1)
    pre = d_pre.cpu().numpy().view(np.complex64).reshape(wl.n_antennas, 2, M, n)
    plan.close()

    w = O.pfb_weights(N, T)
    bar = REL_RMS_FP32 if precision == fengine.FP32 else REL_RMS_REDUCED
    num = den = 0.0
    exact = total = 0
    worst = (0.0, None)
    lsb = []
    for a in range(wl.n_antennas):
        heaps = out[a]
        for p in range(2):
            for q in SAMPLED:
                ref, qo, _ = O.channelize(samples[a, p].astype(np.int32), 0, N, T, w, oracle_model(segs[(a, p)]),
                                          g[a, p], m0 + q, 1)
                got = pre[a, p, q].astype(np.complex128)
                num += np.sum(np.abs(got - ref[0]) ** 2)
                den += np.sum(np.abs(ref[0]) ** 2)
                err = np.maximum(np.abs(got.real - ref[0].real), np.abs(got.imag - ref[0].imag))
                k = int(np.argmax(err))
                if err[k] > worst[0]:
                    worst = (float(err[k]), (a, p, q, k, complex(ref[0][k]), complex(got[k])))
                # the heap cells of spectrum q, pol p: out[heap][k][s][pol][re, im]
                h, s_ = divmod(q, S)
                Sh = min(S, M - h * S)
                cells = heaps[h * S * n * 4:h * S * n * 4 + n * Sh * 4].reshape(n, Sh, 2, 2)[:, s_, p, :]
                d = np.abs(cells.astype(np.int16) - qo[0].astype(np.int16))
                lsb.append(int(d.max()))
                exact += int(np.sum(d == 0))
                total += d.size
                comp = np.stack([got.real, got.imag], axis=-1)
                rq = np.clip(np.where(comp >= 0, np.floor(comp + 0.5), -np.floor(-comp + 0.5)), -127, 127)
                np.testing.assert_array_equal(cells, rq.astype(np.int8))
    rel = np.sqrt(num / den)
    print(f"[parity] config 2 full size, precision {precision}: rel_rms={rel:.3g} exact_int8={exact / total:.6f} "
          f"max_component_error={worst[0]:.3g} at (ant, pol, spectrum, channel, oracle, gpu)={worst[1]}")
    assert rel <= bar
    assert max(lsb) <= 1, f"int8 output differs by {max(lsb)} LSB"
