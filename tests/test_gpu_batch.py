"""Batched call over uneven streams: every member's output in one
fengine_batch_process equals (bit for bit) what the same plan produces alone,
and every member, alone, matches the FP64 oracle in both chunks
(pre-quantisation spectra and 8-bit output)."""
import numpy as np
import pytest

from paper_2303_09886_gb300 import fengine, synth
from tests.fe_harness import Seg, compare_call, streams

pytestmark = pytest.mark.gpu

MEMBERS = [  # (n_antennas, n_channels, n_taps, spectra per chunk, delay)
    (1, 1024, 16, 40, 7.3), (2, 4096, 8, 20, 120.6), (1, 8192, 16, 36, 1999.2),
    (1, 256, 4, 300, 3.0), (1, 32768, 4, 9, 40.4), (3, 2048, 16, 17, 0.0),
]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_09886_gb300 import build
    build.build()
    fengine.load()


def _make(i, n_ant, n, T, m, d):
    L = 2 * n * m
    s = streams(synth.SEED_BASE + 40 + i, n_ant, 2 * L, 20.0 + 7 * i, tones=[(0.1 + 0.05 * i, 50.0, 0.1)])
    plan = fengine.Plan(n_ant, n, T, L, spectra_per_heap=min(16, m), max_delay_samples=int(d) + 8)
    gains = synth.random_gains(500 + i, 2 * n_ant, n).reshape(n_ant, 2, n)
    for a in range(n_ant):
        for p in range(2):
            plan.set_delay(a, p, d + 0.1 * p, rate=1e-7, phase=0.3 * i)
            plan.set_gains(a, p, gains[a, p])
    return plan, s, gains


def _packed(s, lo, L):
    import torch
    pk = np.stack([np.stack([synth.pack10(s[a, p, lo:lo + L]) for p in range(2)]) for a in range(s.shape[0])])
    return torch.from_numpy(pk).cuda()


def test_batch_equals_alone_and_oracle():
    import torch
    made = [_make(i, *m) for i, m in enumerate(MEMBERS)]
    # alone, every member against the oracle in both chunks
    alone = []
    for k, (plan, s, gains) in enumerate(made):
        n_ant, n, T, m, d = MEMBERS[k]
        delays = [[[Seg(delay=d + 0.1 * p, rate=1e-7, phase=0.3 * k)] for p in range(2)] for _ in range(n_ant)]
        outs = []
        for c in range(2):
            L = plan.chunk_samples
            d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
            d_pre = torch.empty(n_ant * 2 * plan.M * n * 2, dtype=torch.float32, device="cuda")
            m0 = plan.process(_packed(s, c * L, L), c * L, d_out, d_pre)
            torch.cuda.synchronize()
            call = dict(m0=m0, out=d_out.cpu().numpy(), tap=None,
                        pre=d_pre.cpu().numpy().view(np.complex64).reshape(n_ant, 2, plan.M, n))
            st = compare_call(s, call, plan.M, plan.S, n, T, delays,
                              [[gains[a, p] for p in range(2)] for a in range(n_ant)])
            print(f"[parity] batch member {k} chunk {c}: rel_rms={st['rel_rms']:.3g} "
                  f"exact_int8={st['exact_fraction']:.6f}")
            outs.append(call["out"])
        alone.append(outs)
        plan.reset()
    # batched, same plans after a reset (same delays and gains)
    batch = fengine.Batch(4)
    got = [[None, None] for _ in made]
    firsts = []
    for c in range(2):
        members = []
        for k, (plan, s, _) in enumerate(made):
            L = plan.chunk_samples
            d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
            members.append((plan, _packed(s, c * L, L), c * L, d_out))
        firsts.append(batch.process(members))
        torch.cuda.synchronize()
        for k, mem in enumerate(members):
            got[k][c] = mem[3].cpu().numpy()
    for k in range(len(made)):
        for c in range(2):
            np.testing.assert_array_equal(got[k][c], alone[k][c], err_msg=f"member {k} chunk {c}")
    batch.close()
    for plan, _, _ in made:
        plan.close()


def test_batch_rejects_repeated_plan():
    import torch
    plan, s, _ = _make(0, *MEMBERS[0])
    L = plan.chunk_samples
    d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
    batch = fengine.Batch(2)
    pk = _packed(s, 0, L)
    with pytest.raises(fengine.FEngineError) as e:
        batch.process([(plan, pk, 0, d_out), (plan, pk, 0, d_out)])
    assert e.value.status == 1
    batch.close()
    plan.close()


def test_grouped_launches_with_shared_shapes_slabs_and_other_forms():
    """Members that share a kernel instantiation go out as one grid per
    phase: five 1024-channel plans (16 taps, one of them in several slabs), three
    8192-channel plans (the persistent 1024-point second stage, one with two
    antennas), a 256-channel plan, and two tensor-core plans that run whole
    beside the grids. Every member's bytes equal its plan alone, in three
    consecutive chunks (history carried through the grouped path)."""
    import torch
    specs = [  # (n_antennas, n_channels, n_taps, spectra per chunk, delay, precision, slab_spectra)
        (1, 1024, 16, 40, 7.3, fengine.FP32, 0), (1, 1024, 16, 70, 30.0, fengine.FP32, 0),
        (2, 1024, 16, 33, 100.2, fengine.FP32, 0), (1, 1024, 16, 100, 2.5, fengine.FP32, 32),
        (1, 1024, 16, 64, 0.0, fengine.FP32, 0),
        (1, 8192, 16, 36, 1999.2, fengine.FP32, 0), (2, 8192, 16, 20, 50.7, fengine.FP32, 0),
        (1, 8192, 16, 50, 5.5, fengine.FP32, 0),
        (1, 256, 4, 300, 3.0, fengine.FP32, 0),
        (1, 8192, 16, 40, 60.1, fengine.TC_FP16, 0), (1, 1024, 8, 45, 9.9, fengine.TC_BF16, 0),
    ]
    made = []
    for i, (n_ant, n, T, m, d, prec, sl) in enumerate(specs):
        L = 2 * n * m
        s = streams(synth.SEED_BASE + 60 + i, n_ant, 3 * L, 25.0, tones=[(0.07 + 0.03 * i, 40.0, 0.2)])
        plans = []
        for _ in range(2):   # one to run alone, one in the batch
            p = fengine.Plan(n_ant, n, T, L, spectra_per_heap=min(16, m), max_delay_samples=int(d) + 8,
                             precision=prec, slab_spectra=sl)
            g = synth.random_gains(700 + i, 2 * n_ant, n).reshape(n_ant, 2, n)
            for a in range(n_ant):
                for pol in range(2):
                    p.set_delay(a, pol, d + 0.2 * pol, rate=1e-7, phase=0.1 * i)
                    p.set_gains(a, pol, g[a, pol])
            plans.append(p)
        made.append((plans, s))
    assert made[3][0][0].info.slabs_per_chunk > 1
    batch = fengine.Batch(4)
    for c in range(3):
        members, alone = [], []
        for plans, s in made:
            L = plans[0].chunk_samples
            pk = _packed(s, c * L, L)
            d_a = torch.empty(plans[0].info.out_bytes, dtype=torch.int8, device="cuda")
            m0 = plans[0].process(pk, c * L, d_a)
            alone.append((m0, d_a))
            members.append((plans[1], pk, c * L, torch.empty_like(d_a)))
        firsts = batch.process(members)
        torch.cuda.synchronize()
        for k, (mem, (m0, d_a)) in enumerate(zip(members, alone)):
            assert firsts[k] == m0
            np.testing.assert_array_equal(mem[3].cpu().numpy(), d_a.cpu().numpy(),
                                          err_msg=f"member {k} chunk {c}")
    batch.close()
    for plans, _ in made:
        for p in plans:
            p.device_status()
            p.close()


def test_grouped_batch_with_lost_data_flags():
    """Grouped members carrying received-heap flags (Sec. 3.7): the output
    and the output-heap flags of every member equal its plan alone."""
    import torch
    HS = fengine.HEAP_SAMPLES
    specs = [(1, 2048, 16, 64), (2, 2048, 16, 128), (1, 8192, 16, 32), (1, 8192, 16, 64)]
    g = np.random.default_rng(11)
    made = []
    for i, (n_ant, n, T, m) in enumerate(specs):
        L = 2 * n * m
        s = streams(synth.SEED_BASE + 90 + i, n_ant, 2 * L, 30.0, tones=[(0.2 + 0.01 * i, 70.0, 0.0)])
        plans = [fengine.Plan(n_ant, n, T, L, spectra_per_heap=16, max_delay_samples=100) for _ in range(2)]
        for p in plans:
            for a in range(n_ant):
                for pol in range(2):
                    p.set_delay(a, pol, 10.0 + a + pol, rate=1e-7)
        valid = [(g.random((n_ant, 2, L // HS)) > 0.15).astype(np.uint8) for _ in range(2)]
        made.append((plans, s, valid))
    batch = fengine.Batch(3)
    for c in range(2):
        members, alone = [], []
        for plans, s, valid in made:
            L = plans[0].chunk_samples
            pk = _packed(s, c * L, L)
            v = torch.from_numpy(valid[c]).cuda()
            d_a = torch.empty(plans[0].info.out_bytes, dtype=torch.int8, device="cuda")
            f_a = torch.empty((plans[0].n_antennas, plans[0].heaps), dtype=torch.uint8, device="cuda")
            plans[0].process(pk, c * L, d_a, valid=v, heap_flags=f_a)
            d_b, f_b = torch.empty_like(d_a), torch.empty_like(f_a)
            alone.append((d_a, f_a))
            members.append((plans[1], pk, c * L, d_b, v, f_b))
        batch.process(members)
        torch.cuda.synchronize()
        for k, (mem, (d_a, f_a)) in enumerate(zip(members, alone)):
            np.testing.assert_array_equal(mem[3].cpu().numpy(), d_a.cpu().numpy(), err_msg=f"member {k} chunk {c}")
            np.testing.assert_array_equal(mem[5].cpu().numpy(), f_a.cpu().numpy(), err_msg=f"flags {k} chunk {c}")
            assert f_a.cpu().numpy().min() == 0          # some heaps were flagged
    batch.close()
    for plans, _, _ in made:
        for p in plans:
            p.close()
