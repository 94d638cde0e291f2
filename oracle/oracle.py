"""Python face of the FP64 CPU oracle (``fengine_oracle.c``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
module. The product library never does, and this module imports nothing from
the product package.

The C file holds the arithmetic (plain FP64 definitions of the paper's steps,
Sec. 2.1 and Eq. 1); this module only builds it with gcc, marshals numpy
arrays and composes per-stream results into the heap layout.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fengine_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_I64P = ctypes.POINTER(ctypes.c_int64)
_F64P = ctypes.POINTER(ctypes.c_double)
_I32P = ctypes.POINTER(ctypes.c_int32)
_U8P = ctypes.POINTER(ctypes.c_uint8)
_I8P = ctypes.POINTER(ctypes.c_int8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP on)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_unpack10.argtypes = [_U8P, ctypes.c_int64, _I32P]
            lib.orc_unpack10.restype = None
            lib.orc_pfb_weights.argtypes = [ctypes.c_int, ctypes.c_int, _F64P]
            lib.orc_pfb_weights.restype = None
            lib.orc_delay_eval.argtypes = [ctypes.c_int32, _I64P, _I64P, _F64P, _F64P,
                                           _F64P, _F64P, ctypes.c_int64, _I64P, _F64P, _F64P]
            lib.orc_delay_eval.restype = None
            lib.orc_fir.argtypes = [_I32P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                    ctypes.c_int, _F64P, ctypes.c_int64, ctypes.c_int64, _F64P]
            lib.orc_fir.restype = None
            lib.orc_dft_naive.argtypes = [ctypes.c_int, _F64P, _F64P]
            lib.orc_dft_naive.restype = None
            lib.orc_fft.argtypes = [ctypes.c_int, _F64P]
            lib.orc_fft.restype = ctypes.c_int
            lib.orc_quantise.argtypes = [ctypes.c_double]
            lib.orc_quantise.restype = ctypes.c_int32
            lib.orc_channelize.argtypes = [
                _I32P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _F64P,
                ctypes.c_int32, _I64P, _I64P, _F64P, _F64P, _F64P, _F64P, _F64P,
                ctypes.c_int64, ctypes.c_int64, _F64P, _I8P, _I64P]
            lib.orc_channelize.restype = ctypes.c_int
            lib.orc_corner_turn.argtypes = [_I8P, _I8P, ctypes.c_int64, ctypes.c_int,
                                            ctypes.c_int, _I8P]
            lib.orc_corner_turn.restype = None
            lib.orc_window_usable.argtypes = [_U8P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_int64, ctypes.c_int64]
            lib.orc_window_usable.restype = ctypes.c_int
            lib.orc_spectrum_flags.argtypes = [_U8P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_int32, _I64P, _I64P,
                                               _F64P, _F64P, _F64P, _F64P, ctypes.c_int64, ctypes.c_int64,
                                               _U8P]
            lib.orc_spectrum_flags.restype = None
            lib.orc_heap_flags.argtypes = [_U8P, _U8P, ctypes.c_int64, ctypes.c_int, _U8P]
            lib.orc_heap_flags.restype = None
            lib.orc_segment_select.argtypes = [ctypes.c_int32, _I64P, ctypes.c_int64]
            lib.orc_segment_select.restype = ctypes.c_int32
            lib.orc_ddc_weights.argtypes = [ctypes.c_int, ctypes.c_int, _F64P]
            lib.orc_ddc_weights.restype = None
            lib.orc_quantise10.argtypes = [ctypes.c_double]
            lib.orc_quantise10.restype = ctypes.c_int32
            lib.orc_ddc.argtypes = [_I32P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _F64P,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int64, _F64P,
                                    _I32P]
            lib.orc_ddc.restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


# ----------------------------------------------------------------- steps

def unpack10(packed: np.ndarray, n_samples: int) -> np.ndarray:
    """10-bit MSB-first two's-complement fields -> int32 (Sec. 2.1 step 1)."""
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    if packed.size * 8 < 10 * n_samples:
        raise ValueError("packed buffer too short")
    out = np.empty(n_samples, dtype=np.int32)
    _load().orc_unpack10(_p(packed, _U8P), n_samples, _p(out, _I32P))
    return out


def pfb_weights(N: int, T: int) -> np.ndarray:
    """Default Hann-windowed-sinc prototype of length N*T, sum w^2 = 1."""
    w = np.empty(N * T, dtype=np.float64)
    _load().orc_pfb_weights(N, T, _p(w, _F64P))
    return w


def dft_naive(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.complex128)
    xi = x.view(np.float64).copy()
    X = np.empty_like(xi)
    _load().orc_dft_naive(x.size, _p(xi, _F64P), _p(X, _F64P))
    return X.view(np.complex128)


def fft(x: np.ndarray) -> np.ndarray:
    xi = np.ascontiguousarray(x, dtype=np.complex128).view(np.float64).copy()
    if _load().orc_fft(xi.size // 2, _p(xi, _F64P)) != 0:
        raise MemoryError("oracle fft")
    return xi.view(np.complex128)


def quantise(x: float) -> int:
    return int(_load().orc_quantise(float(x)))


class DelayModel:
    """Piecewise linear delay/phase model (one (antenna, pol) stream).

    Segments are (t_apply, t_ref, d0, rate, phi0, phi_rate): delay in samples
    d = d0 + rate (t - t_ref), phase in radians phi = phi0 + phi_rate (t - t_ref),
    used for spectra with timestamp >= t_apply.
    """

    def __init__(self, segments=None):
        self.segments = list(segments) if segments else [(-(2 ** 62), 0, 0.0, 0.0, 0.0, 0.0)]
        self.segments.sort(key=lambda s: s[0])

    @classmethod
    def constant(cls, delay=0.0, phase=0.0, rate=0.0, phase_rate=0.0, t_ref=0):
        return cls([(-(2 ** 62), t_ref, delay, rate, phase, phase_rate)])

    def arrays(self):
        seg = self.segments
        return (np.array([s[0] for s in seg], np.int64), np.array([s[1] for s in seg], np.int64),
                np.array([s[2] for s in seg], np.float64), np.array([s[3] for s in seg], np.float64),
                np.array([s[4] for s in seg], np.float64), np.array([s[5] for s in seg], np.float64))

    def eval(self, t0: int):
        ta, tr, d0, r, p0, pr = self.arrays()
        c = np.zeros(1, np.int64)
        dl = np.zeros(1, np.float64)
        ph = np.zeros(1, np.float64)
        _load().orc_delay_eval(len(self.segments), _p(ta, _I64P), _p(tr, _I64P), _p(d0, _F64P),
                               _p(r, _F64P), _p(p0, _F64P), _p(pr, _F64P), int(t0),
                               _p(c, _I64P), _p(dl, _F64P), _p(ph, _F64P))
        return int(c[0]), float(dl[0]), float(ph[0])


def fir(samples: np.ndarray, first: int, N: int, T: int, w: np.ndarray, t0: int, c: int):
    s = np.ascontiguousarray(samples, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    g = np.empty(N, np.float64)
    _load().orc_fir(_p(s, _I32P), int(first), s.size, N, T, _p(w, _F64P), int(t0), int(c),
                    _p(g, _F64P))
    return g


def segment_select(t_applies, t0: int) -> int:
    """Index of the gain (or delay) set that spectrum timestamp t0 uses: the
    last set whose t_apply <= t0, set 0 before every set (reading R12)."""
    ta = np.ascontiguousarray(t_applies, dtype=np.int64)
    return int(_load().orc_segment_select(ta.size, _p(ta, _I64P), int(t0)))


def channelize(samples: np.ndarray, first: int, N: int, T: int, w: np.ndarray,
               delay: DelayModel, gains, m_first: int, m_count: int,
               want_q: bool = True):
    """Whole hot path for one (antenna, pol) stream.

    gains: n complex values, or a list of (t_apply, n complex values) gain
    sets sorted by t_apply (spectrum t0 uses the set segment_select picks).
    Returns (prequant complex128 [m_count, n], q int8 [m_count, n, 2] or None,
    coarse int64 [m_count]).
    """
    if isinstance(gains, (list, tuple)) and gains and isinstance(gains[0], tuple):
        # runs of consecutive spectra with one gain set, each a plain call
        t_app = [g[0] for g in gains]
        sel = [segment_select(t_app, N * (m_first + i)) for i in range(m_count)]
        parts = []
        i = 0
        while i < m_count:
            j = i
            while j < m_count and sel[j] == sel[i]:
                j += 1
            parts.append(channelize(samples, first, N, T, w, delay, gains[sel[i]][1], m_first + i, j - i,
                                    want_q))
            i = j
        return (np.concatenate([p[0] for p in parts]),
                np.concatenate([p[1] for p in parts]) if want_q else None,
                np.concatenate([p[2] for p in parts]))
    n = N // 2
    s = np.ascontiguousarray(samples, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    if w.size != N * T:
        raise ValueError("weights must have N*T entries")
    g = np.ascontiguousarray(np.broadcast_to(np.asarray(gains, np.complex128), (n,)))
    gi = g.view(np.float64)
    ta, tr, d0, r, p0, pr = delay.arrays()
    pre = np.empty((m_count, n), np.complex128)
    q = np.empty((m_count, n, 2), np.int8) if want_q else None
    co = np.empty(m_count, np.int64)
    rc = _load().orc_channelize(
        _p(s, _I32P), int(first), s.size, N, T, _p(w, _F64P), len(delay.segments),
        _p(ta, _I64P), _p(tr, _I64P), _p(d0, _F64P), _p(r, _F64P), _p(p0, _F64P), _p(pr, _F64P),
        _p(gi, _F64P), int(m_first), int(m_count), _p(pre.view(np.float64), _F64P),
        _p(q, _I8P) if q is not None else ctypes.cast(None, _I8P), _p(co, _I64P))
    if rc != 0:
        raise MemoryError("oracle channelize")
    return pre, q, co


def corner_turn(q_pol0: np.ndarray, q_pol1: np.ndarray, S: int) -> np.ndarray:
    """Per-antenna heap layout [h][k][s][pol][re,im] (Sec. 2.2, Sec. 3.6)."""
    q0 = np.ascontiguousarray(q_pol0, np.int8)
    q1 = np.ascontiguousarray(q_pol1, np.int8)
    M, n = q0.shape[0], q0.shape[1]
    out = np.empty(M * n * 4, np.int8)
    _load().orc_corner_turn(_p(q0, _I8P), _p(q1, _I8P), M, n, S, _p(out, _I8P))
    return out


# ------------------------------------------------------------- lost data

HEAP_SAMPLES = 4096   # samples per digitiser heap (Sec. 2.2)


def window_usable(received: np.ndarray, heap_first: int, start: int, length: int,
                  heap_len: int = HEAP_SAMPLES) -> bool:
    """Sec. 3.7: True iff every heap that [start, start + length) touches was
    received (heaps outside received's range are missing)."""
    r = np.ascontiguousarray(received, dtype=np.uint8)
    return bool(_load().orc_window_usable(_p(r, _U8P), int(heap_first), r.size, int(heap_len),
                                          int(start), int(length)))


def spectrum_flags(received: np.ndarray, heap_first: int, N: int, T: int, delay: DelayModel,
                   m_first: int, m_count: int, heap_len: int = HEAP_SAMPLES) -> np.ndarray:
    """Sec. 3.7: uint8 [m_count], 1 where spectrum m's PFB window has no
    missing sample, 0 where it is flagged unusable."""
    r = np.ascontiguousarray(received, dtype=np.uint8)
    ta, tr, d0, rt, p0, pr = delay.arrays()
    out = np.empty(m_count, np.uint8)
    _load().orc_spectrum_flags(_p(r, _U8P), int(heap_first), r.size, int(heap_len), N, T,
                               len(delay.segments), _p(ta, _I64P), _p(tr, _I64P), _p(d0, _F64P),
                               _p(rt, _F64P), _p(p0, _F64P), _p(pr, _F64P), int(m_first), int(m_count),
                               _p(out, _U8P))
    return out


def heap_flags(usable_pol0: np.ndarray, usable_pol1: np.ndarray, S: int) -> np.ndarray:
    """Sec. 3.7: uint8 per output heap of S spectra (both polarisations),
    1 = transmitted, 0 = holds an unusable spectrum and is not transmitted."""
    u0 = np.ascontiguousarray(usable_pol0, np.uint8)
    u1 = np.ascontiguousarray(usable_pol1, np.uint8)
    M = u0.size
    out = np.empty((M + S - 1) // S, np.uint8)
    _load().orc_heap_flags(_p(u0, _U8P), _p(u1, _U8P), M, S, _p(out, _U8P))
    return out


# ------------------------------------------------------- narrow-band mode

def ddc_weights(D: int, Th: int) -> np.ndarray:
    """R15: default low-pass of the narrow-band front end, D Th taps, unit DC gain."""
    h = np.empty(D * Th, np.float64)
    _load().orc_ddc_weights(D, Th, _p(h, _F64P))
    return h


def quantise10(x: float) -> int:
    """R15: round half away from zero, saturate to [-511, 511]."""
    return int(_load().orc_quantise10(float(x)))


def ddc(samples: np.ndarray, first: int, D: int, h: np.ndarray, fc: float, g: float, j0: int, n_out: int):
    """R15 down-converter: outputs j0 .. j0 + n_out - 1 of one stream as
    (y FP64 before requantisation, q 10-bit int32)."""
    s = np.ascontiguousarray(samples, np.int32)
    hh = np.ascontiguousarray(h, np.float64)
    y = np.empty(n_out, np.float64)
    q = np.empty(n_out, np.int32)
    _load().orc_ddc(_p(s, _I32P), int(first), s.size, int(D), hh.size, _p(hh, _F64P), float(fc), float(g),
                    int(j0), int(n_out), _p(y, _F64P), _p(q, _I32P))
    return y, q
