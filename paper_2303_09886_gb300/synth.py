"""Seeded synthetic digitiser streams shaped like the paper's workloads.

This module is the one input generator that both the CUDA path and the FP64
oracle are fed from. It holds none of the channelizer's arithmetic: it makes
10-bit signed voltage samples (Gaussian noise plus tones, rounded and clipped
to the digitiser range, Sec. 2.1 step 1) and packs them the way a digitiser
sends them (10 bits per sample, no padding, most significant bit first,
4 samples per 5 bytes; Sec. 2.2).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20230317
SAMPLE_MIN, SAMPLE_MAX = -512, 511


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def digitiser_samples(seed: int, n: int, sigma: float, tones=(), chirp=None, start: int = 0,
                      block: int = 1 << 22) -> np.ndarray:
    """int16 samples for absolute indices [start, start + n).

    tones: iterable of (frequency in cycles/sample, amplitude, phase in rad).
    chirp: optional (f_begin, f_end, amplitude, phase, span) -- a linear chirp
           whose frequency moves from f_begin to f_end over `span` samples
           counted from absolute index 0.
    Noise is drawn in order from one PCG64 stream seeded with `seed`, so the
    result is a function of (seed, n, start, sigma, tones, chirp).
    """
    g = rng(seed)
    out = np.empty(n, np.int16)
    for b0 in range(0, n, block):
        b1 = min(n, b0 + block)
        i = np.arange(start + b0, start + b1, dtype=np.float64)
        x = g.standard_normal(b1 - b0) * sigma
        for f, a, ph in tones:
            x += a * np.cos(2.0 * np.pi * np.mod(f * i, 1.0) + ph)
        if chirp is not None:
            f0, f1, a, ph, span = chirp
            k = (f1 - f0) / span
            cyc = np.mod(f0 * i + 0.5 * k * i * i, 1.0)
            x += a * np.cos(2.0 * np.pi * cyc + ph)
        out[b0:b1] = np.clip(np.rint(x), SAMPLE_MIN, SAMPLE_MAX).astype(np.int16)
    return out


def dithered_tone(seed: int, n: int, freq: float, amplitude: float, phase: float = 0.0,
                  start: int = 0) -> np.ndarray:
    """int16 samples [start, start + n) of one tone quantised to 10 bits with
    a uniform dither of one LSB (round(x + u), u ~ U(-1/2, 1/2)): the
    quantisation error then has zero mean whatever the tone, as in the
    paper's FFT-precision experiment (Sec. 3.5) and its channel-response
    measurement (Sec. 5.2)."""
    g = rng(seed)
    i = np.arange(start, start + n, dtype=np.float64)
    x = amplitude * np.cos(2.0 * np.pi * np.mod(freq * i, 1.0) + phase) + g.uniform(-0.5, 0.5, n)
    return np.clip(np.rint(x), SAMPLE_MIN, SAMPLE_MAX).astype(np.int16)


def pack10(samples: np.ndarray) -> np.ndarray:
    """Pack int samples in [-512, 511] into the 10-bit MSB-first byte stream.

    Four samples u0..u3 (10-bit two's complement fields) become five bytes
    u0[9:2] | u0[1:0] u1[9:4] | u1[3:0] u2[9:6] | u2[5:0] u3[9:8] | u3[7:0].
    """
    s = np.asarray(samples)
    if s.size % 4:
        raise ValueError("sample count must be a multiple of 4")
    if s.size and (s.min() < SAMPLE_MIN or s.max() > SAMPLE_MAX):
        raise ValueError("samples outside the 10-bit range")
    u = (s.astype(np.int32) & 0x3FF).reshape(-1, 4)
    out = np.empty((u.shape[0], 5), np.uint8)
    out[:, 0] = u[:, 0] >> 2
    out[:, 1] = ((u[:, 0] & 0x3) << 6) | (u[:, 1] >> 4)
    out[:, 2] = ((u[:, 1] & 0xF) << 4) | (u[:, 2] >> 6)
    out[:, 3] = ((u[:, 2] & 0x3F) << 2) | (u[:, 3] >> 8)
    out[:, 4] = u[:, 3] & 0xFF
    return out.reshape(-1)


def random_gains(seed: int, n_streams: int, n: int, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """complex64 [n_streams, n] with |g| ~ U(lo, hi), arg ~ U(0, 2 pi)."""
    g = rng(seed)
    mag = g.uniform(lo, hi, size=(n_streams, n))
    ph = g.uniform(0.0, 2.0 * np.pi, size=(n_streams, n))
    return (mag * np.exp(1j * ph)).astype(np.complex64)
