"""Work splits and the autotuner: every four-step split (fft_n1) and slab size
a plan can be given computes the same channelizer within the parity bars;
fengine_autotune times the valid splits and returns one of them; the
tensor-core forms run for every channel count with a 1024-point second
stage (4096 ... 32768 channels)."""
import numpy as np
import pytest

from paper_2303_09886_gb300 import fengine, synth
from tests.fe_harness import REL_RMS_REDUCED, Seg, compare_call, run_gpu, streams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_09886_gb300 import build
    build.build()
    fengine.load()


def _report(name, st):
    print(f"[parity] {name}: rel_rms={st.get('rel_rms', float('nan')):.3g} exact_int8={st['exact_fraction']:.6f}")


@pytest.mark.parametrize("n,T,M,n1,sl", [(8192, 16, 70, 32, 0), (8192, 16, 70, 64, 32), (8192, 16, 70, 16, 64),
                                         (1024, 8, 100, 16, 32), (1024, 8, 100, 32, 0), (1024, 8, 100, 64, 0),
                                         (4096, 4, 45, 8, 32)])
def test_work_splits_match_the_oracle(n, T, M, n1, sl):
    L = 2 * n * M
    s = streams(synth.SEED_BASE + 90, 1, 2 * L, 35.0, tones=[(0.31, 60.0, 0.2)])
    delays = [[[Seg(delay=17.4 + p, rate=2e-7, phase=0.4)] for p in range(2)]]
    gains = synth.random_gains(91, 2, n).reshape(1, 2, n)
    gains = [[gains[0, p] for p in range(2)]]
    res, M2, S = run_gpu(s, n, T, L, 2, delays, gains, S=10, D=40, fft_n1=n1, slab_spectra=sl)
    for c in res:
        _report(f"split n={n} n1={n1} slab={sl}", compare_call(s, c, M2, S, n, T, delays, gains))


@pytest.mark.parametrize("n,precision", [(4096, fengine.TC_FP16), (32768, fengine.TC_BF16), (32768, fengine.TC_FP16),
                                         (16384, fengine.TC_BF16)])
def test_tensor_core_forms_for_every_1024_point_second_stage(n, precision):
    T, M = 16, 12
    L = 2 * n * M
    s = streams(synth.SEED_BASE + 95, 1, 2 * L, 24.0, chirp=(0.05, 0.45, 60.0, 0.0, 2 * L))
    delays = [[[Seg(delay=30.2 + 3 * p, rate=5e-9, phase=1.1)] for p in range(2)]]
    gains = synth.random_gains(96, 2, n).reshape(1, 2, n)
    gains = [[gains[0, p] for p in range(2)]]
    res, M2, S = run_gpu(s, n, T, L, 2, delays, gains, S=4, D=64, precision=precision, taps=False)
    for c in res:
        _report(f"tensor-core n={n} precision {precision}",
                compare_call(s, c, M2, S, n, T, delays, gains, rel_rms=REL_RMS_REDUCED))


@pytest.mark.parametrize("n,precision", [(8192, fengine.FP32), (8192, fengine.TC_FP16), (2048, fengine.FP32)])
def test_autotune_returns_a_measured_valid_split(n, precision):
    T, M = 16, 96
    L = 2 * n * M
    best, table = fengine.autotune(1, n, T, L, max_delay_samples=64, precision=precision, calls=3)
    assert table, "no candidate was measured"
    assert (best["fft_n1"], best["slab_spectra"]) in {(a, b) for a, b, _ in table}
    assert all(ms > 0 for _, _, ms in table)
    fastest = min(table, key=lambda e: e[2])
    assert (best["fft_n1"], best["slab_spectra"]) == fastest[:2]
    if precision != fengine.FP32:
        assert {a for a, _, _ in table} == {2 * n // 1024}
    print(f"[autotune] n={n} precision={precision}: {table} -> {best}")
    # the tuned plan computes the channelizer
    s = streams(synth.SEED_BASE + 97, 1, 2 * L, 30.0, tones=[(0.2, 50.0, 0.0)])
    delays = [[[Seg(delay=5.5)] for _ in range(2)]]
    res, M2, S = run_gpu(s, n, T, L, 1, delays, None, S=16, D=64, precision=precision,
                         fft_n1=best["fft_n1"], slab_spectra=best["slab_spectra"], taps=False)
    bar = 1e-5 if precision == fengine.FP32 else REL_RMS_REDUCED
    _report(f"autotuned n={n}", compare_call(s, res[0], M2, S, n, T, delays, None, rel_rms=bar))


def test_autotune_cache_round_trip(tmp_path):
    """fengine_autotune_cached: the first call tunes and writes one line; the
    same configuration then comes from the file without timing; another
    shape adds its own line and keeps the first; a line whose split no
    longer makes a plan is ignored and replaced."""
    import json
    path = str(tmp_path / "tune.jsonl")
    kw = dict(spectra_per_heap=0, max_delay_samples=0, calls=1)
    best, hit = fengine.autotune_cached(path, 1, 1024, 8, 2048 * 64, **kw)
    assert not hit
    lines = [json.loads(x) for x in open(path)]
    assert len(lines) == 1 and lines[0]["fft_n1"] == best["fft_n1"] and lines[0]["n_channels"] == 1024
    again, hit = fengine.autotune_cached(path, 1, 1024, 8, 2048 * 64, **kw)
    assert hit and again == best
    other, hit = fengine.autotune_cached(path, 1, 2048, 8, 4096 * 32, **kw)
    assert not hit
    assert len(open(path).readlines()) == 2
    # a stale split (fft_n1 = 3 makes no plan) is ignored and the line replaced
    first = json.loads(open(path).readline())
    first["fft_n1"] = 3
    rest = open(path).readlines()[1:]
    with open(path, "w") as f:
        f.write(json.dumps(first) + "\n" + "".join(rest))
    fresh, hit = fengine.autotune_cached(path, 1, 1024, 8, 2048 * 64, **kw)
    assert not hit and fresh["fft_n1"] != 3
    assert len(open(path).readlines()) == 2
