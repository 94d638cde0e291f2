"""Thin Python binding of libfengine (include/fengine.h).

Argument marshalling only: every step of the channelizer runs in the CUDA
kernels behind the C ABI. PyTorch supplies device memory and streams; tensors
are passed to the library as raw device pointers. If the shared library is
missing or fails to load, every entry point raises -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfengine.so")

FP32, TC_FP16, TC_BF16 = 0, 1, 2
ABI_VERSION = 3
HEAP_SAMPLES = 4096        # samples per digitiser heap (lost-data flags)
FAR_PAST = -(2 ** 62)      # t_apply of a model or gain set that applies at once
STATUS = {0: "FENGINE_OK", 1: "FENGINE_EINVAL", 2: "FENGINE_ENOMEM", 3: "FENGINE_ECUDA",
          4: "FENGINE_ESEQ", 5: "FENGINE_EBUSY", 6: "FENGINE_ETIMEOUT",
          7: "FENGINE_EUNSUPPORTED", 8: "FENGINE_EDELAY", 9: "FENGINE_EIO"}

# every symbol include/fengine.h declares
EXPORTS = ("fengine_strerror", "fengine_last_error", "fengine_abi_version", "fengine_quantise",
           "fengine_default_weights", "fengine_plan_create", "fengine_plan_destroy",
           "fengine_get_info", "fengine_set_delay", "fengine_set_gains", "fengine_reset",
           "fengine_process_chunk", "fengine_set_profiling", "fengine_stage_times",
           "fengine_batch_create", "fengine_batch_destroy", "fengine_batch_process",
           "fengine_service_create", "fengine_service_submit", "fengine_service_set_delay",
           "fengine_service_set_gains", "fengine_service_wait", "fengine_service_get_stats",
           "fengine_service_destroy", "fengine_process_chunk_noalloc", "fengine_autotune",
           "fengine_autotune_cached", "fengine_device_status", "fengine_ingest_create",
           "fengine_ingest_destroy", "fengine_ingest_push", "fengine_ingest_poll", "fengine_ingest_get_stats",
           "fengine_ddc_default_filter", "fengine_ddc_create", "fengine_ddc_destroy", "fengine_ddc_reset",
           "fengine_ddc_process")


class FEngineError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("n_antennas", ctypes.c_int32), ("n_pols", ctypes.c_int32),
                ("n_channels", ctypes.c_int32), ("n_taps", ctypes.c_int32),
                ("chunk_samples", ctypes.c_int64), ("spectra_per_heap", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_delay_samples", ctypes.c_int64),
                ("weights", ctypes.POINTER(ctypes.c_float)),
                ("fft_n1", ctypes.c_int32), ("slab_spectra", ctypes.c_int32),
                ("min_delay_samples", ctypes.c_int64)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("fft_n1", ctypes.c_int32), ("slab_spectra", ctypes.c_int32), ("ms_per_call", ctypes.c_float)]


class Info(ctypes.Structure):
    _fields_ = [("n_channels", ctypes.c_int32), ("n_taps", ctypes.c_int32),
                ("n_antennas", ctypes.c_int32), ("spectra_per_heap", ctypes.c_int32),
                ("fft_n1", ctypes.c_int32), ("fft_n2", ctypes.c_int32),
                ("spectra_per_chunk", ctypes.c_int64), ("history_samples", ctypes.c_int64),
                ("latency_spectra", ctypes.c_int64), ("out_bytes", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t), ("scratch_bytes", ctypes.c_size_t),
                ("slab_spectra", ctypes.c_int32), ("slabs_per_chunk", ctypes.c_int32),
                ("heaps_per_chunk", ctypes.c_int32), ("lost_data", ctypes.c_int32)]


class ChunkDesc(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("d_packed", ctypes.c_void_p),
                ("first_sample", ctypes.c_int64), ("d_out", ctypes.c_void_p),
                ("d_valid", ctypes.c_void_p), ("d_heap_flags", ctypes.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libfengine.so (built by paper_2303_09886_gb300.build). Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FEngineError(-1, f"{path} is missing: run paper_2303_09886_gb300.build.build() "
                               "(the CUDA extension is required; there is no fallback)")
    lib = ctypes.CDLL(path)
    lib.fengine_abi_version.restype = ctypes.c_int32
    if lib.fengine_abi_version() != ABI_VERSION:
        raise FEngineError(-1, f"{path} has ABI version {lib.fengine_abi_version()}, this binding needs "
                               f"{ABI_VERSION}: rebuild the library")
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.fengine_strerror.argtypes = [ctypes.c_int]
    lib.fengine_strerror.restype = ctypes.c_char_p
    lib.fengine_last_error.argtypes = []
    lib.fengine_last_error.restype = ctypes.c_char_p
    lib.fengine_abi_version.argtypes = []
    lib.fengine_abi_version.restype = i32
    lib.fengine_quantise.argtypes = [ctypes.c_float]
    lib.fengine_quantise.restype = i32
    lib.fengine_default_weights.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_float)]
    lib.fengine_plan_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
    lib.fengine_plan_destroy.argtypes = [vp]
    lib.fengine_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    lib.fengine_set_delay.argtypes = [vp, i32, i32, i64, i64, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double]
    lib.fengine_set_gains.argtypes = [vp, i32, i32, ctypes.POINTER(ctypes.c_float), i64]
    lib.fengine_reset.argtypes = [vp]
    lib.fengine_process_chunk.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp, ctypes.POINTER(i64)]
    lib.fengine_device_status.argtypes = [vp]
    lib.fengine_set_profiling.argtypes = [vp, i32]
    lib.fengine_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32)]
    lib.fengine_batch_create.argtypes = [i32, ctypes.POINTER(vp)]
    lib.fengine_batch_destroy.argtypes = [vp]
    lib.fengine_batch_process.argtypes = [vp, vp, ctypes.POINTER(ChunkDesc), i32, ctypes.POINTER(i64)]
    lib.fengine_autotune.argtypes = [ctypes.POINTER(Config), vp, i32, ctypes.POINTER(Config),
                                     ctypes.POINTER(TuneEntry), i32, ctypes.POINTER(i32)]
    lib.fengine_autotune_cached.argtypes = [ctypes.POINTER(Config), vp, i32, ctypes.c_char_p,
                                            ctypes.POINTER(Config), ctypes.POINTER(i32)]
    for name in ("fengine_autotune", "fengine_autotune_cached", "fengine_default_weights", "fengine_plan_create", "fengine_plan_destroy",
                 "fengine_get_info", "fengine_set_delay", "fengine_set_gains", "fengine_reset",
                 "fengine_process_chunk", "fengine_set_profiling", "fengine_stage_times",
                 "fengine_batch_create", "fengine_batch_destroy", "fengine_batch_process",
                 "fengine_device_status"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        lib = load()
        raise FEngineError(status, lib.fengine_last_error().decode(errors="replace"))


def _ptr(t):
    """Device pointer of a CUDA tensor (or None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def quantise(x: float) -> int:
    """The kernels' requantiser evaluated on the host (same source)."""
    return int(load().fengine_quantise(float(x)))


def default_weights(n_channels: int, n_taps: int) -> np.ndarray:
    out = np.empty(2 * n_channels * n_taps, np.float32)
    _check(load().fengine_default_weights(n_channels, n_taps,
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


class Plan:
    """One F-engine plan: n_antennas dual-pol streams on the current CUDA device."""

    def __init__(self, n_antennas: int, n_channels: int, n_taps: int, chunk_samples: int,
                 spectra_per_heap: int = 0, max_delay_samples: int = 0, weights=None,
                 precision: int = FP32, fft_n1: int = 0, slab_spectra: int = 0, min_delay_samples: int = 0):
        lib = load()
        self._w = None
        if weights is not None:
            self._w = np.ascontiguousarray(weights, dtype=np.float32)
            if self._w.size != 2 * n_channels * n_taps:
                raise ValueError("weights must have 2 * n_channels * n_taps entries")
        cfg = Config(n_antennas, 2, n_channels, n_taps, chunk_samples, spectra_per_heap, precision,
                     max_delay_samples,
                     self._w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if self._w is not None else None,
                     fft_n1, slab_spectra, min_delay_samples)
        h = ctypes.c_void_p()
        _check(lib.fengine_plan_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.info = Info()
        _check(lib.fengine_get_info(self._h, ctypes.byref(self.info)))
        self.n_antennas, self.n_channels, self.n_taps = n_antennas, n_channels, n_taps
        self.chunk_samples = chunk_samples
        self.N = 2 * n_channels
        self.M = int(self.info.spectra_per_chunk)
        self.S = int(self.info.spectra_per_heap)
        self.heaps = int(self.info.heaps_per_chunk)

    def close(self):
        if getattr(self, "_h", None):
            _check(load().fengine_plan_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_delay(self, ant: int, pol: int, delay: float, rate: float = 0.0, phase: float = 0.0,
                  phase_rate: float = 0.0, t_apply: int = -(2 ** 62), t_ref: int = 0):
        _check(load().fengine_set_delay(self._h, ant, pol, t_apply, t_ref, delay, rate, phase,
                                        phase_rate))

    def set_gains(self, ant: int, pol: int, gains, t_apply: int = FAR_PAST):
        g = np.ascontiguousarray(np.broadcast_to(np.asarray(gains, np.complex64), (self.n_channels,)))
        gi = g.view(np.float32)
        _check(load().fengine_set_gains(self._h, ant, pol, gi.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        t_apply))

    def device_status(self):
        """fengine_device_status: synchronise and raise if a kernel recorded a fault."""
        _check(load().fengine_device_status(self._h))

    def reset(self):
        _check(load().fengine_reset(self._h))

    STAGES = ("delay_table", "phase1", "phase2", "tail", "unpack")

    def set_profiling(self, enable: bool = True):
        _check(load().fengine_set_profiling(self._h, 1 if enable else 0))

    def stage_times(self):
        """Summed device milliseconds per stage since the last call, and the call count."""
        ms = (ctypes.c_float * 5)()
        calls = ctypes.c_int32()
        _check(load().fengine_stage_times(self._h, ms, ctypes.byref(calls)))
        return dict(zip(self.STAGES, list(ms))), calls.value

    def process(self, packed, first_sample: int, out, prequant=None, window_tap=None, stream=None,
                valid=None, heap_flags=None):
        """Enqueue one chunk. packed: uint8 CUDA tensor [ant, pol, 5L/4]; out: int8
        CUDA tensor of info.out_bytes; valid: optional uint8 CUDA tensor
        [ant, pol, L/4096] of received-heap flags; heap_flags: optional uint8 CUDA
        tensor [ant, heaps_per_chunk] out. Returns the first spectrum index."""
        import torch
        if packed.dtype != torch.uint8 or out.dtype != torch.int8:
            raise TypeError("packed must be uint8 and out int8")
        if packed.numel() != self.n_antennas * 2 * self.chunk_samples * 5 // 4:
            raise ValueError("packed has the wrong size")
        if out.numel() != self.info.out_bytes:
            raise ValueError("out has the wrong size")
        if prequant is not None and prequant.numel() != self.n_antennas * 2 * self.M * self.n_channels * 2:
            raise ValueError("prequant has the wrong size")
        if window_tap is not None and window_tap.numel() != self.n_antennas * 2 * self.M * self.N:
            raise ValueError("window_tap has the wrong size")
        if valid is not None and (valid.dtype != torch.uint8 or
                                  valid.numel() != self.n_antennas * 2 * (self.chunk_samples // HEAP_SAMPLES)):
            raise ValueError("valid must be uint8 [ant, pol, L/4096]")
        if heap_flags is not None and (heap_flags.dtype != torch.uint8 or
                                       heap_flags.numel() != self.n_antennas * self.heaps):
            raise ValueError("heap_flags must be uint8 [ant, heaps_per_chunk]")
        s = stream if stream is not None else torch.cuda.current_stream()
        fs = ctypes.c_int64()
        _check(load().fengine_process_chunk(self._h, ctypes.c_void_p(s.cuda_stream), _ptr(packed),
                                            first_sample, _ptr(valid), _ptr(out), _ptr(heap_flags),
                                            _ptr(prequant), _ptr(window_tap), ctypes.byref(fs)))
        return fs.value


def autotune(n_antennas: int, n_channels: int, n_taps: int, chunk_samples: int, spectra_per_heap: int = 0,
             max_delay_samples: int = 0, precision: int = FP32, calls: int = 5, stream=None):
    """fengine_autotune: time every valid work split and return
    ({"fft_n1": .., "slab_spectra": ..} of the fastest, [(fft_n1, slab_spectra, ms_per_call), ...])."""
    import torch
    cfg = Config(n_antennas, 2, n_channels, n_taps, chunk_samples, spectra_per_heap, precision,
                 max_delay_samples, None, 0, 0, 0)
    tuned = Config()
    entries = (TuneEntry * 32)()
    n = ctypes.c_int32()
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(load().fengine_autotune(ctypes.byref(cfg), ctypes.c_void_p(s.cuda_stream), calls, ctypes.byref(tuned),
                                   entries, 32, ctypes.byref(n)))
    table = [(entries[i].fft_n1, entries[i].slab_spectra, float(entries[i].ms_per_call)) for i in range(n.value)]
    return {"fft_n1": tuned.fft_n1, "slab_spectra": tuned.slab_spectra}, table


def autotune_cached(cache_path: str, n_antennas: int, n_channels: int, n_taps: int, chunk_samples: int,
                    spectra_per_heap: int = 0, max_delay_samples: int = 0, precision: int = FP32,
                    calls: int = 5, stream=None):
    """fengine_autotune_cached: the split stored in the JSON Lines file
    `cache_path` for this configuration and device, else a fresh tuning that
    is then stored. Returns ({"fft_n1": .., "slab_spectra": ..}, from_cache)."""
    import torch
    cfg = Config(n_antennas, 2, n_channels, n_taps, chunk_samples, spectra_per_heap, precision,
                 max_delay_samples, None, 0, 0, 0)
    tuned = Config()
    hit = ctypes.c_int32()
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(load().fengine_autotune_cached(ctypes.byref(cfg), ctypes.c_void_p(s.cuda_stream), calls,
                                          os.fsencode(cache_path), ctypes.byref(tuned), ctypes.byref(hit)))
    return {"fft_n1": tuned.fft_n1, "slab_spectra": tuned.slab_spectra}, bool(hit.value)


class Batch:
    """Many independent plans processed in one call (fengine_batch_process)."""

    def __init__(self, n_pool: int = 8):
        h = ctypes.c_void_p()
        _check(load().fengine_batch_create(n_pool, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _check(load().fengine_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def process(self, members, stream=None):
        """members: list of (Plan, packed uint8 CUDA tensor, first_sample, out int8 CUDA tensor
        [, valid, heap_flags]). Returns the first spectrum index of every member."""
        import torch
        n = len(members)
        descs = (ChunkDesc * max(n, 1))()
        for i, m in enumerate(members):
            plan, packed, first, out = m[:4]
            valid = m[4] if len(m) > 4 else None
            flags = m[5] if len(m) > 5 else None
            if packed.numel() != plan.n_antennas * 2 * plan.chunk_samples * 5 // 4:
                raise ValueError(f"member {i}: packed has the wrong size")
            if out.numel() != plan.info.out_bytes:
                raise ValueError(f"member {i}: out has the wrong size")
            descs[i] = ChunkDesc(plan._h.value, _ptr(packed).value, first, _ptr(out).value,
                                 _ptr(valid).value if valid is not None else None,
                                 _ptr(flags).value if flags is not None else None)
        fs = (ctypes.c_int64 * max(n, 1))()
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(load().fengine_batch_process(self._h, ctypes.c_void_p(s.cuda_stream), descs, n, fs))
        return [fs[i] for i in range(n)]


class ServiceConfig(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64)]


class ServiceStats(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("deferred", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("queued", ctypes.c_int64), ("bytes_in_use", ctypes.c_int64),
                ("peak_bytes", ctypes.c_int64), ("latency_p50_us", ctypes.c_double),
                ("latency_p99_us", ctypes.c_double), ("latency_max_us", ctypes.c_double)]


def _service_signatures(lib):
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.fengine_service_create.argtypes = [ctypes.POINTER(ServiceConfig), ctypes.POINTER(vp)]
    lib.fengine_service_submit.argtypes = [vp, vp, vp, i64, vp, vp, vp, ctypes.POINTER(i64)]
    lib.fengine_service_set_delay.argtypes = [vp, vp, i32, i32, i64, i64, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double]
    lib.fengine_service_set_gains.argtypes = [vp, vp, i32, i32, ctypes.POINTER(ctypes.c_float), i64]
    lib.fengine_service_wait.argtypes = [vp, i64, i32, ctypes.POINTER(ctypes.c_double)]
    lib.fengine_service_get_stats.argtypes = [vp, ctypes.POINTER(ServiceStats)]
    lib.fengine_service_destroy.argtypes = [vp]
    for name in ("fengine_service_create", "fengine_service_submit", "fengine_service_set_delay",
                 "fengine_service_set_gains", "fengine_service_wait", "fengine_service_get_stats",
                 "fengine_service_destroy"):
        getattr(lib, name).restype = ctypes.c_int


class Service:
    """Continuous-batching service over host-memory chunks (fengine_service_*).

    Host buffers passed to submit() must stay alive until wait() returns for
    the ticket; this wrapper keeps references to them."""

    def __init__(self, n_streams: int = 4, hbm_budget_bytes: int = 8 << 30):
        lib = load()
        _service_signatures(lib)
        h = ctypes.c_void_p()
        _check(lib.fengine_service_create(ctypes.byref(ServiceConfig(n_streams, hbm_budget_bytes)),
                                          ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, plan: Plan, h_packed: np.ndarray, first_sample: int, h_out: np.ndarray,
               h_valid: np.ndarray = None, h_heap_flags: np.ndarray = None) -> int:
        if not (h_packed.flags["C_CONTIGUOUS"] and h_out.flags["C_CONTIGUOUS"]):
            raise ValueError("host buffers must be contiguous")
        if h_packed.nbytes != plan.n_antennas * 2 * plan.chunk_samples * 5 // 4 or h_out.nbytes != plan.info.out_bytes:
            raise ValueError("host buffer size mismatch")
        if h_valid is not None and h_valid.nbytes != plan.n_antennas * 2 * (plan.chunk_samples // HEAP_SAMPLES):
            raise ValueError("h_valid size mismatch")
        if h_heap_flags is not None and h_heap_flags.nbytes != plan.n_antennas * plan.heaps:
            raise ValueError("h_heap_flags size mismatch")
        t = ctypes.c_int64()
        _check(load().fengine_service_submit(self._h, plan._h, h_packed.ctypes.data, first_sample,
                                             h_valid.ctypes.data if h_valid is not None else None,
                                             h_out.ctypes.data,
                                             h_heap_flags.ctypes.data if h_heap_flags is not None else None,
                                             ctypes.byref(t)))
        self._keep[t.value] = (h_packed, h_out, h_valid, h_heap_flags)
        return t.value

    def set_delay(self, plan: Plan, ant: int, pol: int, delay: float, rate: float = 0.0, phase: float = 0.0,
                  phase_rate: float = 0.0, t_apply: int = -(2 ** 62), t_ref: int = 0):
        _check(load().fengine_service_set_delay(self._h, plan._h, ant, pol, t_apply, t_ref, delay, rate, phase,
                                                phase_rate))

    def set_gains(self, plan: Plan, ant: int, pol: int, gains, t_apply: int = FAR_PAST):
        g = np.ascontiguousarray(np.broadcast_to(np.asarray(gains, np.complex64), (plan.n_channels,)))
        gi = g.view(np.float32)
        _check(load().fengine_service_set_gains(self._h, plan._h, ant, pol,
                                                gi.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), t_apply))

    def wait(self, ticket: int, timeout_ms: int = -1) -> float:
        """Block until the chunk is done; returns its latency in microseconds."""
        lat = ctypes.c_double()
        st = load().fengine_service_wait(self._h, ticket, timeout_ms, ctypes.byref(lat))
        if st != 6:   # keep buffers alive while a timed-out request still runs
            self._keep.pop(ticket, None)
        _check(st)
        return lat.value

    def stats(self) -> dict:
        s = ServiceStats()
        _check(load().fengine_service_get_stats(self._h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in ServiceStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _check(load().fengine_service_destroy(self._h))
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


HEAP_BYTES = HEAP_SAMPLES * 10 // 8


class Heap(ctypes.Structure):
    _fields_ = [("antenna", ctypes.c_int32), ("pol", ctypes.c_int32), ("timestamp", ctypes.c_int64),
                ("payload", ctypes.c_void_p)]


class IngestStats(ctypes.Structure):
    _fields_ = [("heaps_accepted", ctypes.c_int64), ("heaps_late", ctypes.c_int64),
                ("heaps_duplicate", ctypes.c_int64), ("heaps_outside", ctypes.c_int64),
                ("heaps_missing", ctypes.c_int64), ("chunks_emitted", ctypes.c_int64),
                ("bytes_to_device", ctypes.c_int64)]


def _ingest_signatures(lib):
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.fengine_ingest_create.argtypes = [vp, i64, i32, i32, ctypes.POINTER(vp)]
    lib.fengine_ingest_destroy.argtypes = [vp]
    lib.fengine_ingest_push.argtypes = [vp, ctypes.POINTER(Heap), i32, ctypes.POINTER(i32)]
    lib.fengine_ingest_poll.argtypes = [vp, vp, i32, vp, vp, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                        ctypes.POINTER(i64)]
    lib.fengine_ingest_get_stats.argtypes = [vp, ctypes.POINTER(IngestStats)]
    for name in ("fengine_ingest_create", "fengine_ingest_destroy", "fengine_ingest_push", "fengine_ingest_poll",
                 "fengine_ingest_get_stats"):
        getattr(lib, name).restype = ctypes.c_int


class Ingest:
    """Digitiser heaps in arrival order -> chunks on the device (fengine_ingest_*)."""

    def __init__(self, plan: Plan, first_sample: int = 0, ring_heaps: int = 4096, reorder_chunks: int = 1):
        lib = load()
        _ingest_signatures(lib)
        h = ctypes.c_void_p()
        _check(lib.fengine_ingest_create(plan._h, first_sample, ring_heaps, reorder_chunks, ctypes.byref(h)))
        self._h = h
        self.plan = plan

    def push(self, heaps) -> int:
        """heaps: sequence of (antenna, pol, timestamp, payload uint8 array of HEAP_BYTES).
        Returns how many were consumed; fewer than given means the ring or the
        reorder window is full (poll, then push the rest)."""
        arr = (Heap * max(len(heaps), 1))()
        for i, (a, p, ts, payload) in enumerate(heaps):
            if payload.dtype != np.uint8 or payload.nbytes != HEAP_BYTES or not payload.flags["C_CONTIGUOUS"]:
                raise ValueError("payload must be a contiguous uint8 array of HEAP_BYTES")
            arr[i] = Heap(a, p, ts, payload.ctypes.data)
        acc = ctypes.c_int32()
        st = load().fengine_ingest_push(self._h, arr, len(heaps), ctypes.byref(acc))
        if st not in (0, 5):          # FENGINE_EBUSY: stopped early, not an error here
            _check(st)
        return acc.value

    def poll(self, out, heap_flags=None, stream=None, flush: bool = False):
        """Send pushed heaps to the device; emit the oldest chunk if due.
        Returns (emitted, first_sample, first_spectrum)."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        em, t0, m0 = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().fengine_ingest_poll(self._h, ctypes.c_void_p(s.cuda_stream), int(flush), out.data_ptr(),
                                          heap_flags.data_ptr() if heap_flags is not None else None,
                                          ctypes.byref(em), ctypes.byref(t0), ctypes.byref(m0)))
        return bool(em.value), t0.value, m0.value

    def stats(self) -> dict:
        s = IngestStats()
        _check(load().fengine_ingest_get_stats(self._h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in IngestStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _check(load().fengine_ingest_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DdcConfig(ctypes.Structure):
    _fields_ = [("n_antennas", ctypes.c_int32), ("decimation", ctypes.c_int32),
                ("taps_per_phase", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("chunk_samples", ctypes.c_int64), ("center_frequency", ctypes.c_double),
                ("gain", ctypes.c_float), ("filter", ctypes.POINTER(ctypes.c_float))]


def _ddc_signatures(lib):
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.fengine_ddc_default_filter.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_float)]
    lib.fengine_ddc_create.argtypes = [ctypes.POINTER(DdcConfig), ctypes.POINTER(vp)]
    lib.fengine_ddc_destroy.argtypes = [vp]
    lib.fengine_ddc_reset.argtypes = [vp]
    lib.fengine_ddc_process.argtypes = [vp, vp, vp, i64, vp, vp]
    for name in ("fengine_ddc_default_filter", "fengine_ddc_create", "fengine_ddc_destroy", "fengine_ddc_reset",
                 "fengine_ddc_process"):
        getattr(lib, name).restype = ctypes.c_int


def ddc_default_filter(decimation: int, taps_per_phase: int) -> np.ndarray:
    """fengine_ddc_default_filter: the narrow-band mode's built-in low-pass."""
    lib = load()
    _ddc_signatures(lib)
    out = np.empty(decimation * taps_per_phase, np.float32)
    _check(lib.fengine_ddc_default_filter(decimation, taps_per_phase,
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


class DDC:
    """Narrow-band front end (fengine_ddc_*): the wide-band stream down-converted
    to a real 10-bit stream at 2/D of its rate holding the band around fc."""

    def __init__(self, n_antennas: int, decimation: int, taps_per_phase: int, chunk_samples: int,
                 center_frequency: float, gain: float = 1.0, filter=None):
        lib = load()
        _ddc_signatures(lib)
        self._filt = None if filter is None else np.ascontiguousarray(filter, np.float32)
        cfg = DdcConfig(n_antennas, decimation, taps_per_phase, 0, chunk_samples, center_frequency, gain,
                        None if self._filt is None else self._filt.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        h = ctypes.c_void_p()
        _check(lib.fengine_ddc_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.n_antennas, self.decimation, self.chunk_samples = n_antennas, decimation, chunk_samples
        self.out_samples = 2 * chunk_samples // decimation

    def process(self, packed, first_sample: int, out, out_float=None, stream=None):
        """packed: uint8 CUDA tensor [ant, pol, 5L/4]; out: uint8 CUDA tensor
        [ant, pol, 5L'/4], L' = 2L/D; out_float: optional float32 CUDA tensor [ant, pol, L']."""
        import torch
        if packed.numel() != self.n_antennas * 2 * self.chunk_samples * 5 // 4:
            raise ValueError("packed size mismatch")
        if out.numel() != self.n_antennas * 2 * self.out_samples * 5 // 4:
            raise ValueError("out size mismatch")
        if out_float is not None and out_float.numel() != self.n_antennas * 2 * self.out_samples:
            raise ValueError("out_float size mismatch")
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(load().fengine_ddc_process(self._h, ctypes.c_void_p(s.cuda_stream), packed.data_ptr(), first_sample,
                                          out.data_ptr(),
                                          out_float.data_ptr() if out_float is not None else None))

    def reset(self):
        _check(load().fengine_ddc_reset(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _check(load().fengine_ddc_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
