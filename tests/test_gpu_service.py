"""Streaming service (continuous batching): every chunk's result is the same
alone and in the mix, per-plan order holds, a small HBM budget defers
requests without changing results, an impossible request fails cleanly, and
delay updates applied through the service match the same updates applied to
a plan processed alone."""
import numpy as np
import pytest

from paper_2303_09886_gb300 import fengine, synth
from tests.fe_harness import streams

pytestmark = pytest.mark.gpu

SHAPES = [(1024, 16, 32), (4096, 8, 16), (256, 4, 200)]   # (channels, taps, spectra per chunk)
N_CHUNKS = 3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_09886_gb300 import build
    build.build()
    fengine.load()


def _pinned(nbytes, dtype):
    import torch
    return torch.empty(nbytes, dtype=dtype, pin_memory=True).numpy()


def _setup():
    import torch
    plans, chunks = [], []
    for i, (n, T, m) in enumerate(SHAPES):
        L = 2 * n * m
        plan = fengine.Plan(1, n, T, L, spectra_per_heap=min(16, m), max_delay_samples=64)
        s = streams(synth.SEED_BASE + 60 + i, 1, N_CHUNKS * L, 30.0, tones=[(0.2, 40.0, 0.5)])
        cs = []
        for c in range(N_CHUNKS):
            pk = np.stack([synth.pack10(s[0, p, c * L:(c + 1) * L]) for p in range(2)]).reshape(-1)
            h = _pinned(pk.size, torch.uint8)
            h[:] = pk
            cs.append(h)
        plans.append(plan)
        chunks.append(cs)
    return plans, chunks


def _alone(plans, chunks, delay_updates=None):
    import torch
    ref = []
    for i, plan in enumerate(plans):
        outs = []
        for c in range(N_CHUNKS):
            if delay_updates and (i, c) in delay_updates:
                plan.set_delay(0, 0, *delay_updates[(i, c)])
            d_in = torch.from_numpy(chunks[i][c]).cuda().view(1, 2, -1)
            d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
            plan.process(d_in, c * plan.chunk_samples, d_out)
            outs.append(d_out.cpu().numpy())
        ref.append(outs)
        plan.reset()
        plan.set_delay(0, 0, 0.0)
    torch.cuda.synchronize()
    return ref


def test_service_results_equal_alone_and_in_order():
    import torch
    plans, chunks = _setup()
    ref = _alone(plans, chunks)
    svc = fengine.Service(n_streams=3, hbm_budget_bytes=1 << 30)
    outs = [[_pinned(p.info.out_bytes, torch.int8) for _ in range(N_CHUNKS)] for p in plans]
    tickets = []
    for c in range(N_CHUNKS):                       # interleave the plans
        for i, plan in enumerate(plans):
            tickets.append(svc.submit(plan, chunks[i][c], c * plan.chunk_samples, outs[i][c]))
    lat = [svc.wait(t, 60000) for t in tickets]
    st = svc.stats()
    print(f"[service] completed={st['completed']} p50={st['latency_p50_us']:.0f}us "
          f"p99={st['latency_p99_us']:.0f}us peak={st['peak_bytes']}")
    assert st["completed"] == len(tickets) and st["failed"] == 0
    assert all(x > 0 for x in lat)
    for i in range(len(plans)):
        for c in range(N_CHUNKS):
            np.testing.assert_array_equal(outs[i][c], ref[i][c], err_msg=f"plan {i} chunk {c}")
    svc.close()
    for p in plans:
        p.close()


def test_small_budget_defers_but_keeps_results():
    import torch
    plans, chunks = _setup()
    ref = _alone(plans, chunks)
    biggest = max(p.info.out_bytes + p.n_antennas * 2 * p.chunk_samples * 5 // 4 for p in plans)
    svc = fengine.Service(n_streams=2, hbm_budget_bytes=biggest + 1)   # one request at a time
    outs = [[_pinned(p.info.out_bytes, torch.int8) for _ in range(N_CHUNKS)] for p in plans]
    tickets = [svc.submit(plan, chunks[i][c], c * plan.chunk_samples, outs[i][c])
               for c in range(N_CHUNKS) for i, plan in enumerate(plans)]
    for t in tickets:
        svc.wait(t, 60000)
    st = svc.stats()
    assert st["deferred"] > 0 and st["peak_bytes"] <= biggest + 1
    for i in range(len(plans)):
        for c in range(N_CHUNKS):
            np.testing.assert_array_equal(outs[i][c], ref[i][c])
    svc.close()
    for p in plans:
        p.close()


def test_request_over_budget_fails_cleanly():
    import torch
    plans, chunks = _setup()
    svc = fengine.Service(n_streams=1, hbm_budget_bytes=1024)
    out = _pinned(plans[0].info.out_bytes, torch.int8)
    t = svc.submit(plans[0], chunks[0][0], 0, out)
    with pytest.raises(fengine.FEngineError) as e:
        svc.wait(t, 60000)
    assert e.value.status == 5
    assert svc.stats()["failed"] == 1
    svc.close()
    for p in plans:
        p.close()


def test_delay_updates_through_the_service():
    import torch
    plans, chunks = _setup()
    upd = {(0, 1): (12.4, 1e-5, 0.7), (2, 2): (3.3, 0.0, -1.0)}
    ref = _alone(plans, chunks, upd)
    svc = fengine.Service(n_streams=3, hbm_budget_bytes=1 << 30)
    outs = [[_pinned(p.info.out_bytes, torch.int8) for _ in range(N_CHUNKS)] for p in plans]
    tickets = []
    for c in range(N_CHUNKS):
        for i, plan in enumerate(plans):
            if (i, c) in upd:
                svc.set_delay(plan, 0, 0, *upd[(i, c)])
            tickets.append(svc.submit(plan, chunks[i][c], c * plan.chunk_samples, outs[i][c]))
    for t in tickets:
        svc.wait(t, 60000)
    for i in range(len(plans)):
        for c in range(N_CHUNKS):
            np.testing.assert_array_equal(outs[i][c], ref[i][c], err_msg=f"plan {i} chunk {c}")
    svc.close()
    for p in plans:
        p.close()
