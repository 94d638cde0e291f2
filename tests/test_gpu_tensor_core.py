"""GPU parity of the reduced-precision forms, whose phase 1 (unpack, coarse
delay, PFB FIR of Eq. 1 and the first DFT stage with its twiddle) runs as one
tcgen05 tensor-core contraction per FIR column, against the FP64 oracle:
bit-exact window taps (unpack + coarse delay), pre-quantisation relative RMS
<= 2e-3, 8-bit output within 1 LSB.

The cases cover every first-stage radix the kernel has (N1 = 8 R, R = 1, 2,
4, 8), every tap count (T = 1 pads the contraction to K = 16), ragged last
tiles (spectra per call not a multiple of the 128-spectrum tile), several
slabs per call, windows that straddle the history and the chunk, delay
steps inside a tile (one pass per run of equal delay) and chunking
invariance (bit-identical output for different chunk lengths)."""
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


def _report(name, stats):
    print(f"[tensor-core] {name}: rel_rms={stats.get('rel_rms', float('nan')):.3g} "
          f"exact_int8={stats['exact_fraction']:.6f}")


def _case(n, T, M, chunks, precision, seed, rate=1e-9, slab=0, n_ant=1, taps=True, D=2100):
    N = 2 * n
    L = N * M
    g = np.random.default_rng(seed)
    tones = [(f, a, 0.3) for f, a in zip(g.uniform(0.01, 0.49, 3), g.uniform(20, 100, 3))]
    s = streams(synth.SEED_BASE + seed, n_ant, chunks * L, 40.0, tones=tones)
    delays = [[[Seg(delay=float(g.uniform(0, D - 100)), rate=rate, phase=float(g.uniform(0, 6.28)))]
               for _ in range(2)] for _ in range(n_ant)]
    gains = synth.random_gains(seed, 2 * n_ant, n).reshape(n_ant, 2, n)
    gains = [[gains[a, p] for p in range(2)] for a in range(n_ant)]
    res, M_, S = run_gpu(s, n, T, L, chunks, delays, gains, D=D, precision=precision, slab_spectra=slab,
                         taps=taps)
    for c in res:
        st = compare_call(s, c, M_, S, n, T, delays, gains, rel_rms=REL_RMS_REDUCED)
        _report(f"n={n} T={T} M={M} prec={precision}", st)
    return res


@pytest.mark.parametrize("precision", [fengine.TC_FP16, fengine.TC_BF16])
@pytest.mark.parametrize("n,T,M", [
    (32, 4, 130),        # N = 64: R = 1, N2 = 8; two tiles, the second of 2 spectra
    (1024, 16, 200),     # R = 1, N2 = 256
    (4096, 8, 131),      # R = 1, N2 = 1024
    (8192, 16, 129),     # R = 2 (the 8192-channel workload's split)
    (16384, 4, 40),      # R = 4
    (32768, 2, 12),      # R = 8
    (512, 1, 150),       # T = 1: the contraction padded to K = 16 with zero weights
    (256, 32, 140),      # T = 32: K = 256
])
def test_every_radix_and_tap_count(n, T, M, precision):
    _case(n, T, M, 2, precision, seed=40 + n % 97 + T)


@pytest.mark.parametrize("precision", [fengine.TC_FP16, fengine.TC_BF16])
def test_slabs_and_two_antennas(precision):
    # 200 spectra in 64-spectrum slabs: four phase-1 / phase-2 launch pairs,
    # tiles of 64 rows, two antennas (four streams)
    _case(2048, 16, 200, 2, precision, seed=61, slab=64, n_ant=2)


@pytest.mark.parametrize("precision", [fengine.TC_FP16, fengine.TC_BF16])
def test_delay_steps_inside_tiles(precision):
    # a delay rate of 0.02 samples/sample steps the coarse delay every ~25
    # samples of timestamp, i.e. every spectrum or two: a tile is many passes
    n, T, M = 64, 8, 160
    N = 2 * n
    L = N * M
    s = streams(synth.SEED_BASE + 70, 1, 2 * L, 40.0, tones=[(0.13, 80.0, 0.1)])
    delays = [[[Seg(delay=5.0 + 3 * p, rate=0.003 * (p + 1), phase=0.4)] for p in range(2)]]
    res, M_, S = run_gpu(s, n, T, L, 2, delays, None, D=300, precision=precision)
    for c in res:
        st = compare_call(s, c, M_, S, n, T, delays, None, rel_rms=REL_RMS_REDUCED)
        _report(f"delay steps prec={precision}", st)


@pytest.mark.parametrize("precision", [fengine.TC_FP16, fengine.TC_BF16])
def test_chunking_invariance(precision):
    """The same stream in chunks of 128, 256 or 512 spectra gives the same
    bytes: each spectrum's contraction does not depend on where its row sits
    in a tile, or on whether its window was decoded from history."""
    n, T = 1024, 16
    N = 2 * n
    total = 1024 * N
    s = streams(synth.SEED_BASE + 80, 1, total, 40.0, tones=[(0.21, 90.0, 0.2)])
    delays = [[[Seg(delay=123.4, rate=2e-6, phase=0.3)] for _ in range(2)]]
    outs = {}
    for M in (128, 256, 512):
        L = N * M
        res, M_, S = run_gpu(s, n, T, L, total // L, delays, None, S=128, D=200, precision=precision,
                             taps=False, prequant=False)
        outs[M] = np.concatenate([r["out"] for r in res])
    np.testing.assert_array_equal(outs[128], outs[256])
    np.testing.assert_array_equal(outs[128], outs[512])
