"""GPU tests of the host ingest path (Sec. 3.1-3.2, 3.7): digitiser heaps of
4096 samples pushed per polarisation in a shuffled arrival order, with lost,
duplicated and late heaps, come out of fengine_ingest_poll as the chunks a
direct fengine_process_chunk call gives for the same samples (missing heaps
zero-filled, received-heap flags set from what arrived): 8-bit output and
output-heap flags bit-identical, counters exact, and the flags equal to the
oracle's for the heaps that were lost."""
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


def _plan(n_ant, n, T, L, precision=fengine.FP32):
    p = fengine.Plan(n_ant, n, T, L, spectra_per_heap=16, max_delay_samples=300, precision=precision)
    for a in range(n_ant):
        for pol in range(2):
            p.set_delay(a, pol, 17.3 + 40 * a + 9 * pol, 1e-6, 0.2 * pol)
    return p


@pytest.mark.parametrize("reorder,precision", [(0, fengine.FP32), (1, fengine.FP32), (2, fengine.FP32),
                                               (1, fengine.TC_FP16)])
def test_shuffled_heaps_with_losses_equal_direct_chunks(reorder, precision):
    import torch
    n_ant, n, T = 2, 1024, 8
    N = 2 * n
    L = N * 64                       # 32 heaps per stream per chunk
    hpc = L // fengine.HEAP_SAMPLES
    n_chunks = 5
    s = streams(synth.SEED_BASE + 500, n_ant, n_chunks * L, 30.0, tones=[(0.137, 60.0, 0.4)])
    packed = [[synth.pack10(s[a, p]) for p in range(2)] for a in range(n_ant)]
    g = np.random.default_rng(77)
    # lost heaps: (chunk, stream, heap); chunk 3 loses every heap of stream 3 (antenna 1, pol 1)
    lost = {(0, 0, 0), (1, 0, 5), (1, 2, 31), (2, 1, 16)} | {(3, 3, h) for h in range(hpc)}
    received = np.ones((n_chunks, 2 * n_ant, hpc), np.uint8)
    for c, st, h in lost:
        received[c, st, h] = 0

    def heap(c, st, h):
        a, pol = divmod(st, 2)
        ts = c * L + h * fengine.HEAP_SAMPLES
        b0 = ts * 5 // 4
        return (a, pol, ts, packed[a][pol][b0:b0 + fengine.HEAP_BYTES])

    # arrival order: chunk by chunk, each chunk's heaps shuffled, and within
    # the reorder window the next chunk's heaps interleaved with the current one's
    order = []
    for c in range(n_chunks):
        hs = [(c, st, h) for st in range(2 * n_ant) for h in range(hpc) if (c, st, h) not in lost]
        g.shuffle(hs)
        order.extend(hs)
    if reorder > 0:
        # move a few heaps of chunk c + 1 ahead of the last heaps of chunk c
        for c in range(n_chunks - 1):
            first_next = next(i for i, x in enumerate(order) if x[0] == c + 1)
            for k in range(3):
                order.insert(first_next - 5 * (k + 1), order.pop(first_next + k))
    dup = order[10]
    order.insert(40, dup)                          # a duplicate of a heap of chunk 0
    heaps = [heap(*x) for x in order]
    late = heap(0, 1, 3)                           # chunk 0 again, after it has been emitted

    plan = _plan(n_ant, n, T, L, precision)
    ing = fengine.Ingest(plan, first_sample=0, ring_heaps=48, reorder_chunks=reorder)
    d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
    d_flags = torch.empty((n_ant, plan.heaps), dtype=torch.uint8, device="cuda")
    got = []

    def drain(flush=False):
        while True:
            em, t0, m0 = ing.poll(d_out, d_flags, flush=flush)
            if not em:
                return
            torch.cuda.synchronize()
            got.append((t0, m0, d_out.cpu().numpy().copy(), d_flags.cpu().numpy().copy()))
            if flush:
                return

    i = 0
    sent_late = False
    while i < len(heaps):
        k = ing.push(heaps[i:i + 7])
        i += k
        drain()
        if got and not sent_late:
            assert ing.push([late]) == 1
            sent_late = True
    while len(got) < n_chunks:
        drain(flush=True)
    st = ing.stats()
    ing.close()
    plan.close()

    # the same chunks through fengine_process_chunk, missing heaps zeroed
    ref = _plan(n_ant, n, T, L, precision)
    r_out = torch.empty_like(d_out)
    r_flags = torch.empty_like(d_flags)
    for c in range(n_chunks):
        chunk = np.stack([np.stack([packed[a][p][c * L * 5 // 4:(c + 1) * L * 5 // 4] for p in range(2)])
                          for a in range(n_ant)]).copy()
        for cc, stn, h in lost:
            if cc == c:
                a, pol = divmod(stn, 2)
                chunk[a, pol, h * fengine.HEAP_BYTES:(h + 1) * fengine.HEAP_BYTES] = 0
        valid = torch.from_numpy(received[c].reshape(n_ant, 2, hpc).copy()).cuda()
        m0 = ref.process(torch.from_numpy(chunk).cuda(), c * L, r_out, valid=valid, heap_flags=r_flags)
        torch.cuda.synchronize()
        t0, gm0, out, flags = got[c]
        assert (t0, gm0) == (c * L, m0)
        np.testing.assert_array_equal(out, r_out.cpu().numpy(), err_msg=f"chunk {c} output")
        np.testing.assert_array_equal(flags, r_flags.cpu().numpy(), err_msg=f"chunk {c} heap flags")
        # output-heap flags against the oracle's reading of Sec. 3.7
        info = ref.info
        for a in range(n_ant):
            usable = []
            for pol in range(2):
                rec = received[:c + 1, 2 * a + pol].reshape(-1)
                dm = O.DelayModel([(-(2 ** 62), 0, 17.3 + 40 * a + 9 * pol, 1e-6, 0.2 * pol, 0.0)])
                usable.append(O.spectrum_flags(rec, 0, N, T, dm, m0, info.spectra_per_chunk))
            np.testing.assert_array_equal(flags[a], O.heap_flags(usable[0], usable[1], 16),
                                          err_msg=f"chunk {c} antenna {a} oracle flags")
    ref.close()
    n_lost = len(lost)
    assert st["chunks_emitted"] == n_chunks
    assert st["heaps_missing"] == n_lost
    assert st["heaps_duplicate"] == 1
    assert st["heaps_late"] == 1
    assert st["heaps_accepted"] == n_chunks * 2 * n_ant * hpc - n_lost
    assert st["bytes_to_device"] >= st["heaps_accepted"] * fengine.HEAP_BYTES
