"""GPU parity of the boundary's time-dependent inputs against the oracle:
lost-data flags (Sec. 3.7: a spectrum whose PFB window touches a missing
4096-sample heap is unusable, an output heap holding one is not sent), gain
sets that switch at spectrum timestamps, and negative coarse delays
(Sec. 3.3), in the FP32 form and the tensor-core forms."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_09886_gb300 import fengine, synth
from tests.fe_harness import REL_RMS_FP32, REL_RMS_REDUCED, Seg, compare_call, oracle_model, run_gpu, streams

pytestmark = pytest.mark.gpu

HEAP = O.HEAP_SAMPLES
FORMS = [fengine.FP32, fengine.TC_FP16, fengine.TC_BF16]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_09886_gb300 import build
    build.build()
    fengine.load()


def _bar(precision):
    return REL_RMS_FP32 if precision == fengine.FP32 else REL_RMS_REDUCED


def _oracle_flags(valids, L, n_ant, N, T, delays, m0, M, S, n_calls_before):
    """Heap flags of one call from the oracle: the received flags of every
    heap delivered so far (heaps before the first chunk are missing)."""
    rec = np.concatenate([v for v in valids[:n_calls_before + 1]], axis=2)   # [ant, pol, heaps]
    out = np.empty((n_ant, (M + S - 1) // S), np.uint8)
    for a in range(n_ant):
        u = [O.spectrum_flags(rec[a, p], 0, N, T, oracle_model(delays[a][p]), m0, M) for p in range(2)]
        out[a] = O.heap_flags(u[0], u[1], S)
    return out


@pytest.mark.parametrize("precision", FORMS)
def test_lost_data_flags_hand_case(precision):
    # n = 1024, T = 4, one spectrum per heap (S = 1: heap flags = spectrum
    # flags of both pols); missing heaps at a chunk edge, mid-window and in
    # the second chunk; delays 0, 3 and -5 samples (the oracle's hand case)
    n, T, M = 1024, 4, 20
    N, L = 2 * n, 2 * n * 20
    s = streams(synth.SEED_BASE + 200, 3, 2 * L, 30.0)
    valids = [np.ones((3, 2, L // HEAP), np.uint8) for _ in range(2)]
    valids[0][:, 0, 5] = 0          # pol 0, heap 5: samples [20480, 24576)
    valids[0][:, 1, 9] = 0          # pol 1, heap 9: the chunk's last heap
    valids[1][0, 0, 0] = 0          # antenna 0, first heap of the second chunk
    delays = [[[Seg(delay=float(c))], [Seg(delay=float(c))]] for c in (0, 3, -5)]
    res, M2, S = run_gpu(s, n, T, L, 2, delays, None, S=1, D=8, Dmin=-5, precision=precision,
                         valids=valids, flags=True)
    for k, c in enumerate(res):
        st = compare_call(s, c, M2, S, n, T, delays, None, rel_rms=_bar(precision))
        want = _oracle_flags(valids, L, 3, N, T, delays, c["m0"], M2, S, k)
        np.testing.assert_array_equal(c["flags"], want, err_msg=f"call {k}")
    assert res[0]["flags"].min() == 0 and res[0]["flags"].max() == 1


@pytest.mark.parametrize("precision", FORMS)
def test_lost_data_random_heaps_and_delay_steps(precision):
    # 8192 channels, 16 taps, heaps of 64 spectra, three calls, a tenth of the
    # heaps missing at random, delays with a rate that steps the coarse delay
    n, T, M = 8192, 16, 64
    N, L = 2 * n, 2 * n * 64
    g = np.random.default_rng(7)
    s = streams(synth.SEED_BASE + 201, 2, 3 * L, 40.0, tones=[(0.17, 70.0, 0.3)])
    valids = [(g.random((2, 2, L // HEAP)) > 0.1).astype(np.uint8) for _ in range(3)]
    delays = [[[Seg(delay=float(g.uniform(-900, 900)), rate=3e-6, phase=0.2)] for _ in range(2)] for _ in range(2)]
    res, M2, S = run_gpu(s, n, T, L, 3, delays, None, S=16, D=1000, Dmin=-1000, precision=precision,
                         valids=valids, flags=True, taps=False)
    for k, c in enumerate(res):
        compare_call(s, c, M2, S, n, T, delays, None, rel_rms=_bar(precision))
        want = _oracle_flags(valids, L, 2, N, T, delays, c["m0"], M2, S, k)
        np.testing.assert_array_equal(c["flags"], want, err_msg=f"call {k}")


def test_lost_data_needs_heap_aligned_calls():
    import torch
    plan = fengine.Plan(1, 1024, 4, 2048 * 2, max_delay_samples=0)     # L = 4096: one heap
    d_in = torch.zeros(plan.n_antennas * 2 * plan.chunk_samples * 5 // 4, dtype=torch.uint8, device="cuda")
    d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
    flags = torch.empty((1, plan.heaps), dtype=torch.uint8, device="cuda")
    plan.process(d_in, 0, d_out, heap_flags=flags)
    plan.reset()
    plan.process(d_in, 2048, d_out)                       # not heap-aligned: history flags unknown
    with pytest.raises(fengine.FEngineError) as e:
        plan.process(d_in, 2048 + 4096, d_out, heap_flags=flags)
    assert e.value.status == 1
    plan.reset()
    plan.process(d_in, 8192, d_out, heap_flags=flags)      # known again after a reset
    torch.cuda.synchronize()
    assert int(flags.cpu().numpy().max()) == 0             # every window reaches before the first chunk
    odd = fengine.Plan(1, 1024, 4, 2048 * 3)                # L = 6144: not a multiple of 4096
    assert odd.info.lost_data == 0
    with pytest.raises(fengine.FEngineError):
        odd.process(torch.zeros(2 * 6144 * 5 // 4, dtype=torch.uint8, device="cuda"), 0,
                    torch.empty(odd.info.out_bytes, dtype=torch.int8, device="cuda"),
                    heap_flags=torch.empty((1, odd.heaps), dtype=torch.uint8, device="cuda"))
    plan.close()
    odd.close()


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("n", [1024, 8192])
def test_gain_sets_switch_at_spectrum_timestamps(precision, n):
    # three gain sets per stream: from the start, from a spectrum inside the
    # first call (not on a tile or heap boundary), and from one inside the
    # second call; pol 1 switches one spectrum later than pol 0
    T, M = 16, 75
    N, L = 2 * n, 2 * n * M
    g = np.random.default_rng(n)
    s = streams(synth.SEED_BASE + 202, 1, 2 * L, 35.0, tones=[(0.23, 60.0, 0.1)])
    G = synth.random_gains(203, 6, n).reshape(3, 2, n)
    m_first = -(T - 1)
    sched = [[(fengine.FAR_PAST, G[0, p]), (N * (m_first + 37 + p), G[1, p]),
              (N * (m_first + M + 11 + p), G[2, p])] for p in range(2)]
    delays = [[[Seg(delay=float(g.uniform(0, 500)), rate=1e-7, phase=0.7)] for _ in range(2)]]
    res, M2, S = run_gpu(s, n, T, L, 2, delays, [sched], S=16, D=600, precision=precision, taps=False)
    for c in res:
        compare_call(s, c, M2, S, n, T, delays, [sched], rel_rms=_bar(precision))


@pytest.mark.parametrize("precision", FORMS)
def test_negative_coarse_delays(precision):
    # delays from -2500 to +1500 samples (Sec. 3.3: "even negative"), a rate
    # that crosses zero inside the call; the emission lag E = ceil(2500 / N)
    n, T, M = 1024, 16, 90
    N, L = 2 * n, 2 * n * M
    s = streams(synth.SEED_BASE + 204, 2, 2 * L, 40.0, tones=[(0.31, 80.0, 0.4)])
    delays = [[[Seg(delay=-2500.0)], [Seg(delay=-40.0, rate=1e-3)]],
              [[Seg(delay=1500.0)], [Seg(delay=-1.49, phase=1.0)]]]
    res, M2, S = run_gpu(s, n, T, L, 2, delays, None, D=1600, Dmin=-2500, precision=precision)
    E = -(-2500 // N)
    assert res[0]["m0"] == -(T - 1) - E
    assert res[1]["m0"] == M - (T - 1) - E
    for c in res:
        compare_call(s, c, M2, S, n, T, delays, None, rel_rms=_bar(precision))


def test_delay_outside_the_range_is_refused():
    import torch
    plan = fengine.Plan(1, 1024, 4, 2048 * 4, max_delay_samples=10, min_delay_samples=-10)
    d_in = torch.zeros(2 * plan.chunk_samples * 5 // 4, dtype=torch.uint8, device="cuda")
    d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
    plan.set_delay(0, 0, -10.4)
    plan.process(d_in, 0, d_out)
    plan.set_delay(0, 1, -10.6)                           # rounds to -11
    with pytest.raises(fengine.FEngineError) as e:
        plan.process(d_in, plan.chunk_samples, d_out)
    assert e.value.status == 8
    plan.close()
