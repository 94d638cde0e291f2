"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded bytes (bit-exact unpack + coarse delay, pre-quantisation relative
RMS <= 1e-5, 8-bit output within 1 LSB), over several tiles, ragged tails,
every FFT split the library uses, delay steps inside a tile, delay-model
segments, chunking invariance and the error paths."""
import numpy as np
import pytest

from paper_2303_09886_gb300 import fengine, synth
from tests.fe_harness import Seg, compare_call, default_delays, run_gpu, streams

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
    print(f"[parity] {name}: rel_rms={stats.get('rel_rms', float('nan')):.3g} "
          f"exact_int8={stats['exact_fraction']:.6f}")


def test_config1_shape_tone_and_saturation():
    """1 ant x 2 pol, 1024 channels, 16 taps, sigma 32 + bin-centred tone of
    amplitude 100 at channel 192, coarse 7 + fine 0.3, phase 0.1, unit gains."""
    n, T, L = 1024, 16, 2048 * 32
    s = streams(synth.SEED_BASE + 1, 1, 3 * L, 32.0, tones=[(192 / 2048, 100.0, 0.7)])
    delays = default_delays(1, [Seg(delay=7.3, phase=0.1)])
    res, M, S = run_gpu(s, n, T, L, 3, delays, None, D=16)
    for c in res:
        st = compare_call(s, c, M, S, n, T, delays, None)
        _report("cfg1-shape", st)
    # the tone channel saturates at +-127 and never reaches -128
    assert res[-1]["out"].min() >= -127


def test_config2_shape_random_delays_and_gains():
    """8192 channels, 16 taps, 2 antennas, delays 0-2000 with rate 1e-9,
    random gains |g| in [0.5, 2], ragged heaps (S = 16, M = 40)."""
    n, T, L = 8192, 16, 16384 * 40
    g = np.random.default_rng(5)
    tones = [(f, a, 0.3) for f, a in zip(g.uniform(0.01, 0.49, 3), g.uniform(20, 100, 3))]
    s = streams(synth.SEED_BASE + 2, 2, 2 * L, 40.0, tones=tones)
    delays = [[[Seg(delay=float(g.uniform(0, 2000)), rate=1e-9, phase=float(g.uniform(0, 6.28)))]
               for _ in range(2)] for _ in range(2)]
    gains = synth.random_gains(99, 4, n).reshape(2, 2, n)
    gains = [[gains[a, p] for p in range(2)] for a in range(2)]
    res, M, S = run_gpu(s, n, T, L, 2, delays, gains, S=16, D=2100)
    for c in res:
        _report("cfg2-shape", compare_call(s, c, M, S, n, T, delays, gains))


def test_persistent_second_stage_with_several_items_per_cta():
    """The FP32 1024-point second stage is persistent (at most two CTAs per
    SM, each taking every gridDim-th work item of 4 spectra x 2 pols of one
    class k1). n = 4096 (N1 = 8: 5 classes) with 3 antennas and 257 spectra
    per call gives 3 x 5 x 65 = 975 items, more than the resident CTAs, so
    CTAs run several items with the next item's sequences prefetched, and
    the last group of each class is ragged (1 spectrum)."""
    n, T, M = 4096, 16, 257
    L = 2 * n * M
    g = np.random.default_rng(11)
    s = streams(synth.SEED_BASE + 12, 3, 2 * L, 30.0, tones=[(0.3173, 80.0, 0.2)])
    delays = [[[Seg(delay=float(g.uniform(0, 60)), rate=3e-9, phase=float(g.uniform(0, 6.28)))] for _ in range(2)]
              for _ in range(3)]
    gains = synth.random_gains(13, 6, n).reshape(3, 2, n)
    gains = [[gains[a, p] for p in range(2)] for a in range(3)]
    res, M2, S = run_gpu(s, n, T, L, 2, delays, gains, S=64, D=64, taps=False)
    for c in res:
        _report("persistent second stage, 975 items", compare_call(s, c, M2, S, n, T, delays, gains))


@pytest.mark.parametrize("n,T,M", [(32768, 4, 12), (16384, 8, 20), (4096, 16, 33), (2048, 32, 9)])
def test_other_fft_splits(n, T, M):
    L = 2 * n * M
    s = streams(synth.SEED_BASE + 3, 1, 2 * L, 24.0, tones=[(0.1234, 60.0, 0.0)])
    delays = default_delays(1, [Seg(delay=3.6, rate=2e-7, phase=-1.0, phase_rate=1e-4)])
    res, M2, S = run_gpu(s, n, T, L, 2, delays, None, D=64)
    for c in res:
        _report(f"n={n} T={T}", compare_call(s, c, M2, S, n, T, delays, None))


@pytest.mark.parametrize("n,T", [(16, 2), (16, 1), (32, 8), (64, 32), (128, 4)])
def test_tiny_transforms(n, T):
    L = 2 * n * 70
    s = streams(synth.SEED_BASE + 4, 2, 2 * L, 50.0)
    delays = default_delays(2, [Seg(delay=1.2)])
    res, M, S = run_gpu(s, n, T, L, 2, delays, None, S=7, D=8)
    for c in res:
        _report(f"tiny n={n} T={T}", compare_call(s, c, M, S, n, T, delays, None))


def test_coarse_delay_steps_inside_tiles():
    """Delay rate of 2e-3 samples/sample: the coarse delay changes every few
    spectra, so phase-1 tiles hold several constant-delay runs."""
    n, T, L = 256, 4, 512 * 96
    s = streams(synth.SEED_BASE + 5, 1, 3 * L, 30.0)
    delays = default_delays(1, [Seg(delay=5.0, rate=2e-3, phase=0.5, phase_rate=3e-3)])
    res, M, S = run_gpu(s, n, T, L, 3, delays, None, D=400)
    for c in res:
        _report("delay steps", compare_call(s, c, M, S, n, T, delays, None))


def test_delay_model_segments_switch_mid_chunk():
    n, T, L = 512, 8, 1024 * 64
    s = streams(synth.SEED_BASE + 6, 1, 2 * L, 30.0)
    segs = [Seg(delay=10.0), Seg(delay=500.25, rate=-1e-5, phase=2.0, t_apply=1024 * 70, t_ref=1024 * 70),
            Seg(delay=3.5, t_apply=1024 * 100)]
    delays = default_delays(1, segs)
    res, M, S = run_gpu(s, n, T, L, 2, delays, None, D=600)
    for c in res:
        _report("segments", compare_call(s, c, M, S, n, T, delays, None))


def test_identity_weights_give_the_plain_dft_of_the_window():
    n, T, L = 1024, 1, 2048 * 16
    s = streams(synth.SEED_BASE + 7, 1, L, 40.0)
    w = np.ones(2 * n, np.float32)
    delays = default_delays(1, [Seg(delay=2.0)])
    res, M, S = run_gpu(s, n, T, L, 1, delays, None, D=4, weights=w)
    c = res[0]
    X = np.fft.fft(c["tap"][0, 0].astype(np.float64), axis=1)[:, :n]
    err = np.sqrt(np.sum(np.abs(c["pre"][0, 0] - X) ** 2) / np.sum(np.abs(X) ** 2))
    assert err < 1e-6
    _report("identity weights", compare_call(s, c, M, S, n, T, delays, None, weights=w))


@pytest.mark.parametrize("precision,spectra,heap", [(fengine.TC_FP16, 40, 16), (fengine.TC_BF16, 40, 16),
                                                    (fengine.TC_FP16, 37, 12), (fengine.TC_BF16, 37, 12)])
def test_reduced_precision_forms(precision, spectra, heap):
    """Tensor-core FIR + first DFT stage (FP16 / BF16 operands, FP32
    accumulation): pre-quantisation relative RMS <= 2e-3 against the FP64
    oracle, 8-bit output within 1 LSB; 8192 channels, 16 taps, random delays
    and gains. 37 spectra per call leave a ragged last tile, and heaps of 12
    spectra split the second stage's 4-spectrum items across heap rows."""
    from tests.fe_harness import REL_RMS_REDUCED
    n, T, L = 8192, 16, 16384 * spectra
    g = np.random.default_rng(15)
    tones = [(f, a, 0.3) for f, a in zip(g.uniform(0.01, 0.49, 3), g.uniform(20, 100, 3))]
    s = streams(synth.SEED_BASE + 12, 2, 2 * L, 40.0, tones=tones)
    delays = [[[Seg(delay=float(g.uniform(0, 2000)), rate=1e-9, phase=float(g.uniform(0, 6.28)))]
               for _ in range(2)] for _ in range(2)]
    gains = synth.random_gains(98, 4, n).reshape(2, 2, n)
    gains = [[gains[a, p] for p in range(2)] for a in range(2)]
    res, M, S = run_gpu(s, n, T, L, 2, delays, gains, S=heap, D=2100, precision=precision)
    for c in res:
        st = compare_call(s, c, M, S, n, T, delays, gains, rel_rms=REL_RMS_REDUCED)
        _report(f"tensor-core precision {precision}", st)


def test_reduced_precision_rejects_unsupported_shapes():
    with pytest.raises(fengine.FEngineError) as e:
        fengine.Plan(1, 16, 16, 32 * 8, precision=fengine.TC_FP16)
    assert e.value.status == 7


def test_chunking_invariance():
    """The same stream split into chunks of 1, 2 or 4 x 32 spectra gives
    bit-identical 8-bit output and pre-quantisation spectra."""
    n, T = 1024, 16
    total = 2048 * 128
    s = streams(synth.SEED_BASE + 8, 1, total, 32.0, tones=[(0.2, 80.0, 1.0)])
    delays = default_delays(1, [Seg(delay=11.7, rate=3e-6, phase=0.4)])
    outs = {}
    for per in (32, 64, 128):
        L = 2048 * per
        res, M, S = run_gpu(s, n, T, L, total // L, delays, None, S=32, D=32, taps=False)
        pre = np.concatenate([r["pre"][0] for r in res], axis=1)
        out = np.concatenate([r["out"] for r in res])
        outs[per] = (pre, out)
    for per in (64, 128):
        np.testing.assert_array_equal(outs[per][0], outs[32][0])
        np.testing.assert_array_equal(outs[per][1], outs[32][1])


def test_error_paths():
    import torch
    n, T, L = 256, 4, 512 * 8
    plan = fengine.Plan(1, n, T, L, max_delay_samples=10)
    d_in = torch.zeros(2 * L * 5 // 4, dtype=torch.uint8, device="cuda")
    d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
    assert plan.process(d_in, 0, d_out) == -(T - 1)
    with pytest.raises(fengine.FEngineError) as e:
        plan.process(d_in, 2 * L, d_out)          # gap
    assert e.value.status == 4
    with pytest.raises(fengine.FEngineError) as e:
        plan.process(d_in, L + 1, d_out)          # not a multiple of 2n
    assert e.value.status == 1
    plan.set_delay(0, 1, 10.6)                    # c = 11 > D = 10
    with pytest.raises(fengine.FEngineError) as e:
        plan.process(d_in, L, d_out)
    assert e.value.status == 8
    plan.set_delay(0, 1, -0.4)                    # c = 0: fine again
    plan.process(d_in, L, d_out)
    plan.reset()
    plan.process(d_in, 7 * L, d_out)              # any start after a reset
    torch.cuda.synchronize()
    plan.close()


@pytest.mark.parametrize("n,T,fft_n1", [(8192, 16, 16), (8192, 16, 32), (8192, 8, 64), (4096, 16, 8), (1024, 32, 8)])
def test_staged_input_equals_direct_decode_and_oracle(n, T, fft_n1):
    """Phase-1 tiles of 512 columns that hold one coarse delay and lie inside
    the chunk stage their packed rows in shared memory by 16-byte copies when
    the stream's bytes are 16-byte aligned (rows of 5N/4 bytes, N a multiple
    of 64), and decode each sample straight from global memory otherwise. The
    same chunks, once at a 16-byte-aligned address and once 4 bytes further
    on, give bit-identical spectra and 8-bit output, and both agree with the
    oracle. 128 spectra per call (tiles 1-3 away from the history), one
    stream with a delay rate that steps the coarse delay inside the chunk
    (tiles of several delay runs take the general path), no window tap."""
    N = 2 * n
    M = 128
    L = N * M
    g = np.random.default_rng(n + T)
    s = streams(synth.SEED_BASE + 40 + T, 2, 2 * L, 35.0, tones=[(0.21, 70.0, 0.4)])
    delays = [[[Seg(delay=float(g.uniform(0, 500)), rate=(3e-6 if (a, p) == (1, 0) else 1e-9),
                    phase=float(g.uniform(0, 6.28)))] for p in range(2)] for a in range(2)]
    gains = synth.random_gains(17, 4, n).reshape(2, 2, n)
    gains = [[gains[a, p] for p in range(2)] for a in range(2)]
    kw = dict(S=16, D=600, taps=False, fft_n1=fft_n1)
    res_a, M2, S = run_gpu(s, n, T, L, 2, delays, gains, **kw)
    res_b, _, _ = run_gpu(s, n, T, L, 2, delays, gains, in_offset=4, **kw)
    for ca, cb in zip(res_a, res_b):
        assert ca["m0"] == cb["m0"]
        np.testing.assert_array_equal(ca["pre"].view(np.uint32), cb["pre"].view(np.uint32))
        np.testing.assert_array_equal(ca["out"], cb["out"])
        _report(f"staged n={n} T={T} N1={fft_n1}", compare_call(s, ca, M2, S, n, T, delays, gains))


def test_staged_input_at_the_chunk_end_and_zero_delay():
    """Zero delay: the last window of a call ends on the chunk's last sample,
    so the 16-byte copies of the last tile's last segment would reach past
    the stream's bytes and that tile decodes directly while the others are
    staged. Aligned and offset input agree bit for bit and with the oracle."""
    n, T, M = 8192, 16, 64
    N = 2 * n
    L = N * M
    s = streams(synth.SEED_BASE + 77, 1, 2 * L, 30.0, tones=[(0.37, 60.0, 0.1)])
    delays = [[[Seg(delay=0.0)] for _ in range(2)]]
    kw = dict(S=16, D=0, taps=False)
    res_a, M2, S = run_gpu(s, n, T, L, 2, delays, None, **kw)
    res_b, _, _ = run_gpu(s, n, T, L, 2, delays, None, in_offset=4, **kw)
    for ca, cb in zip(res_a, res_b):
        np.testing.assert_array_equal(ca["pre"].view(np.uint32), cb["pre"].view(np.uint32))
        np.testing.assert_array_equal(ca["out"], cb["out"])
        _report("staged, zero delay", compare_call(s, ca, M2, S, n, T, delays, None))
