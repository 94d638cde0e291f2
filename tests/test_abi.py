"""Host-side checks of the C ABI (no GPU): the library builds and loads,
exports every symbol include/fengine.h declares, and its host-only entry
points agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_09886_gb300 import build, fengine

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fengine.load()


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "fengine.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fengine_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    declared = _declared_symbols()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(fengine.EXPORTS) == declared


def test_abi_version_and_strerror(lib):
    assert lib.fengine_abi_version() == 3 == fengine.ABI_VERSION
    for st in range(9):
        assert lib.fengine_strerror(st)
    assert b"unknown" in lib.fengine_strerror(99)


@pytest.mark.parametrize("n,T", [(16, 2), (1024, 16), (8192, 16), (32768, 4)])
def test_default_weights_match_oracle(lib, n, T):
    w32 = fengine.default_weights(n, T)
    w64 = O.pfb_weights(2 * n, T)
    assert np.max(np.abs(w32.astype(np.float64) - w64)) <= 2.0 ** -24 * np.max(np.abs(w64))


def test_quantiser_matches_oracle_on_every_tie_and_neighbour(lib):
    """The kernels' FP32 quantiser (same source, run on the host) against the
    oracle's round-half-away-and-saturate: every half-integer in [-130, 130],
    its float neighbours, and a dense random sample."""
    xs = []
    for k in range(-260, 261):
        h = np.float32(k / 2.0)
        v = h
        for _ in range(4):
            xs.append(v)
            v = np.nextafter(v, np.float32(np.inf), dtype=np.float32)
        v = h
        for _ in range(4):
            v = np.nextafter(v, np.float32(-np.inf), dtype=np.float32)
            xs.append(v)
    xs += list(np.random.default_rng(1).uniform(-140, 140, 20000).astype(np.float32))
    xs += [np.float32(v) for v in (0.0, -0.0, 1e-30, -1e-30, 0.49999997, -0.49999997, 1e30, -1e30)]
    for x in xs:
        assert fengine.quantise(float(x)) == O.quantise(float(x)), x


@pytest.mark.parametrize("kw,status", [
    (dict(n_pols=3), 1), (dict(n_channels=1000), 1), (dict(n_taps=3), 1),
    (dict(chunk_samples=1000), 1), (dict(spectra_per_heap=10 ** 6), 1),
    (dict(max_delay_samples=-1), 1), (dict(n_antennas=0), 1),
    (dict(fft_n1=12), 1), (dict(fft_n1=128), 1), (dict(fft_n1=2), 1), (dict(slab_spectra=33), 1),
    (dict(slab_spectra=-32), 1), (dict(min_delay_samples=1), 1), (dict(min_delay_samples=-(2 ** 31)), 1),
    (dict(precision=1, n_channels=16, chunk_samples=32 * 8), 7),
    (dict(precision=2, n_channels=16, chunk_samples=32 * 8), 7),
    (dict(precision=1, n_channels=8192, fft_n1=32, chunk_samples=16384 * 4), 1)])
def test_plan_config_validation_before_any_device_call(lib, kw, status):
    cfg = dict(n_antennas=1, n_pols=2, n_channels=1024, n_taps=16, chunk_samples=2048 * 8,
               spectra_per_heap=0, precision=0, max_delay_samples=0, weights=None, fft_n1=0, slab_spectra=0,
               min_delay_samples=0)
    cfg.update(kw)
    c = fengine.Config(**cfg)
    h = ctypes.c_void_p()
    assert lib.fengine_plan_create(ctypes.byref(c), ctypes.byref(h)) == status
    assert not h.value
    assert lib.fengine_last_error()


def test_binding_refuses_without_library(tmp_path):
    with pytest.raises(fengine.FEngineError):
        fengine._lib, saved = None, fengine._lib
        try:
            fengine.load(str(tmp_path / "missing.so"))
        finally:
            fengine._lib = saved


def test_autotune_rejects_bad_arguments_before_any_device_call(lib):
    c = fengine.Config(n_antennas=1, n_pols=2, n_channels=1024, n_taps=16, chunk_samples=2048 * 8,
                       spectra_per_heap=0, precision=0, max_delay_samples=0, weights=None, fft_n1=0,
                       slab_spectra=0, min_delay_samples=0)
    tuned = fengine.Config()
    n = ctypes.c_int32(-1)
    assert lib.fengine_autotune(ctypes.byref(c), None, 0, ctypes.byref(tuned), None, 0, ctypes.byref(n)) == 1
    assert lib.fengine_autotune(None, None, 3, ctypes.byref(tuned), None, 0, ctypes.byref(n)) == 1


def test_batch_and_service_refuse_bad_arguments_before_any_device_call(lib):
    EINVAL = 1
    vp = ctypes.c_void_p
    h = vp()
    # batch: pool size 1..64, an out pointer, a live handle, non-negative counts
    for n_pool in (0, -1, 65):
        assert lib.fengine_batch_create(n_pool, ctypes.byref(h)) == EINVAL
    assert lib.fengine_batch_create(8, None) == EINVAL
    assert lib.fengine_batch_destroy(None) == EINVAL
    first = ctypes.c_int64()
    assert lib.fengine_batch_process(None, None, None, 0, ctypes.byref(first)) == EINVAL
    # service: 1..64 streams and a positive budget, live handles everywhere
    fengine._service_signatures(lib)
    for n_streams, budget in ((0, 1 << 30), (65, 1 << 30), (4, 0), (4, -1)):
        cfg = fengine.ServiceConfig(n_streams, budget)
        assert lib.fengine_service_create(ctypes.byref(cfg), ctypes.byref(h)) == EINVAL
    assert lib.fengine_service_create(None, ctypes.byref(h)) == EINVAL
    assert lib.fengine_service_create(ctypes.byref(fengine.ServiceConfig(4, 1 << 30)), None) == EINVAL
    ticket = ctypes.c_int64()
    assert lib.fengine_service_submit(None, None, None, 0, None, None, None, ctypes.byref(ticket)) == EINVAL
    assert lib.fengine_service_set_delay(None, None, 0, 0, 0, 0, 1.0, 0.0, 0.0, 0.0) == EINVAL
    assert lib.fengine_service_set_gains(None, None, 0, 0, None, 0) == EINVAL
    lat = ctypes.c_double()
    assert lib.fengine_service_wait(None, 0, 10, ctypes.byref(lat)) == EINVAL
    assert lib.fengine_service_get_stats(None, None) == EINVAL
    assert lib.fengine_service_destroy(None) == EINVAL


def test_ingest_and_tune_cache_refuse_bad_arguments_before_any_device_call(lib, tmp_path):
    EINVAL = 1
    vp = ctypes.c_void_p
    h = vp()
    fengine._ingest_signatures(lib)
    # no plan, bad ring size or reorder depth, no out pointer
    assert lib.fengine_ingest_create(None, 0, 64, 1, ctypes.byref(h)) == EINVAL
    for ring, reorder in ((0, 1), (64, -1), (64, 4)):
        assert lib.fengine_ingest_create(vp(1), 0, ring, reorder, ctypes.byref(h)) == EINVAL
    assert lib.fengine_ingest_destroy(None) == EINVAL
    acc = ctypes.c_int32()
    assert lib.fengine_ingest_push(None, None, 0, ctypes.byref(acc)) == EINVAL
    em, t0, m0 = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    assert lib.fengine_ingest_poll(None, None, 0, None, None, ctypes.byref(em), ctypes.byref(t0),
                                   ctypes.byref(m0)) == EINVAL
    assert lib.fengine_ingest_get_stats(None, None) == EINVAL
    # the autotune cache: a configuration, a path and an out pointer
    c = fengine.Config(n_antennas=1, n_pols=2, n_channels=1024, n_taps=16, chunk_samples=2048 * 8,
                       spectra_per_heap=0, precision=0, max_delay_samples=0, weights=None, fft_n1=0,
                       slab_spectra=0, min_delay_samples=0)
    tuned, hit = fengine.Config(), ctypes.c_int32()
    path = str(tmp_path / "tune.jsonl").encode()
    assert lib.fengine_autotune_cached(None, None, 3, path, ctypes.byref(tuned), ctypes.byref(hit)) == EINVAL
    assert lib.fengine_autotune_cached(ctypes.byref(c), None, 3, None, ctypes.byref(tuned),
                                       ctypes.byref(hit)) == EINVAL
    assert lib.fengine_autotune_cached(ctypes.byref(c), None, 3, b"", ctypes.byref(tuned),
                                       ctypes.byref(hit)) == EINVAL
    assert lib.fengine_autotune_cached(ctypes.byref(c), None, 0, path, ctypes.byref(tuned),
                                       ctypes.byref(hit)) == EINVAL
    assert not (tmp_path / "tune.jsonl").exists()


@pytest.mark.parametrize("D,Th", [(2, 16), (8, 16), (32, 4), (16, 128)])
def test_ddc_default_filter_matches_oracle(lib, D, Th):
    h = fengine.ddc_default_filter(D, Th)
    np.testing.assert_allclose(h, O.ddc_weights(D, Th), rtol=2e-7, atol=1e-9)


def test_ddc_refuses_bad_configuration_before_any_device_call(lib):
    EINVAL = 1
    fengine._ddc_signatures(lib)
    h = ctypes.c_void_p()
    ok = dict(n_antennas=1, decimation=8, taps_per_phase=16, reserved=0, chunk_samples=8 * 1024,
              center_frequency=0.2, gain=1.0, filter=None)
    for bad in (dict(n_antennas=0), dict(decimation=6), dict(decimation=64), dict(taps_per_phase=0),
                dict(taps_per_phase=300), dict(reserved=1), dict(chunk_samples=8 * 1024 + 8),
                dict(chunk_samples=64), dict(center_frequency=0.5), dict(center_frequency=-0.1),
                dict(center_frequency=float("nan")), dict(gain=float("inf"))):
        cfg = fengine.DdcConfig(**{**ok, **bad})
        assert lib.fengine_ddc_create(ctypes.byref(cfg), ctypes.byref(h)) == EINVAL, bad
    assert lib.fengine_ddc_create(None, ctypes.byref(h)) == EINVAL
    assert lib.fengine_ddc_destroy(None) == EINVAL
    assert lib.fengine_ddc_reset(None) == EINVAL
    assert lib.fengine_ddc_process(None, None, None, 0, None, None) == EINVAL
    out = (ctypes.c_float * 8)()
    assert lib.fengine_ddc_default_filter(6, 4, out) == EINVAL
    assert lib.fengine_ddc_default_filter(8, 0, out) == EINVAL
