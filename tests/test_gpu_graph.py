"""CUDA graph capture of the hot path: once a plan's delay models and gains
are on the device (staged by an earlier call), a fengine_process_chunk call
and a fengine_batch_process call enqueue only kernels and event edges, so
they can be captured into a CUDA graph; replaying the graph gives output
bit-identical to the same call made directly."""
import numpy as np
import pytest

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


def _plan(n_ant, n, T, m, seed, precision=fengine.FP32):
    L = 2 * n * m
    s = streams(seed, n_ant, 2 * L, 30.0, tones=[(0.2, 40.0, 0.1)])
    plan = fengine.Plan(n_ant, n, T, L, spectra_per_heap=min(16, m), max_delay_samples=64, precision=precision)
    gains = synth.random_gains(seed, 2 * n_ant, n).reshape(n_ant, 2, n)
    for a in range(n_ant):
        for p in range(2):
            plan.set_delay(a, p, 12.3 + p, rate=1e-7, phase=0.2 * (a + 1))
            plan.set_gains(a, p, gains[a, p])
    return plan, s, L


def _packed(s, lo, L):
    import torch
    pk = np.stack([np.stack([synth.pack10(s[a, p, lo:lo + L]) for p in range(2)]) for a in range(s.shape[0])])
    return torch.from_numpy(pk).cuda()


@pytest.mark.parametrize("shape,precision", [((2, 8192, 16, 40), fengine.FP32), ((1, 8192, 16, 37), fengine.TC_FP16),
                                             ((1, 1024, 8, 70), fengine.FP32)])
def test_process_chunk_replays_from_a_graph(shape, precision):
    import torch
    direct, s, L = _plan(*shape, seed=synth.SEED_BASE + 70, precision=precision)
    captured, _, _ = _plan(*shape, seed=synth.SEED_BASE + 70, precision=precision)
    c0, c1 = _packed(s, 0, L), _packed(s, L, L)
    out_d0 = torch.empty(direct.info.out_bytes, dtype=torch.int8, device="cuda")
    out_d1 = torch.empty_like(out_d0)
    out_c0 = torch.empty_like(out_d0)
    out_c1 = torch.zeros_like(out_d0)
    direct.process(c0, 0, out_d0)
    direct.process(c1, L, out_d1)
    captured.process(c0, 0, out_c0)   # stages the models and fills the history
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
        captured.process(c1, L, out_c1, stream=side)
    assert int(out_c1.abs().sum().item()) == 0      # capturing ran nothing
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out_c1.cpu().numpy(), out_d1.cpu().numpy())
    direct.close()
    captured.close()


def test_batch_replays_from_a_graph():
    import torch
    shapes = [(1, 1024, 16, 40), (2, 4096, 8, 20), (1, 256, 4, 300)]
    made_d = [_plan(*sh, seed=synth.SEED_BASE + 80 + i) for i, sh in enumerate(shapes)]
    made_c = [_plan(*sh, seed=synth.SEED_BASE + 80 + i) for i, sh in enumerate(shapes)]
    ins = [(_packed(s, 0, L), _packed(s, L, L)) for _, s, L in made_d]
    outs_d = [torch.empty(p.info.out_bytes, dtype=torch.int8, device="cuda") for p, _, _ in made_d]
    outs_c = [torch.zeros_like(o) for o in outs_d]
    scratch = [torch.empty_like(o) for o in outs_d]
    batch_d, batch_c = fengine.Batch(4), fengine.Batch(4)
    # chunk 0 directly on both (stages models, fills histories), chunk 1 directly / captured
    batch_d.process([(p, ins[i][0], 0, scratch[i]) for i, (p, _, _) in enumerate(made_d)])
    batch_d.process([(p, ins[i][1], L, outs_d[i]) for i, (p, _, L) in enumerate(made_d)])
    batch_c.process([(p, ins[i][0], 0, scratch[i]) for i, (p, _, _) in enumerate(made_c)])
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
        batch_c.process([(p, ins[i][1], L, outs_c[i]) for i, (p, _, L) in enumerate(made_c)], stream=side)
    g.replay()
    torch.cuda.synchronize()
    for od, oc in zip(outs_d, outs_c):
        np.testing.assert_array_equal(oc.cpu().numpy(), od.cpu().numpy())
    batch_d.close()
    batch_c.close()
    for p, _, _ in made_d + made_c:
        p.close()
