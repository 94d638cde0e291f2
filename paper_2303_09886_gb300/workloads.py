"""Synthetic workloads shaped like the paper's F-engine configurations.

Each workload fixes the plan shape (antennas, channels, taps, chunk length),
the seeded signal recipe (Gaussian noise plus tones or a chirp, rounded and
clipped to 10 bits, Sec. 2.1 step 1), and the delay and gain models. They
stand in for the live digitiser streams the paper measures on (Sec. 5); no
dataset exists. Inputs are generated on the host with numpy PCG64 streams
seeded from 20230317 + workload index.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import synth


@dataclasses.dataclass
class Workload:
    name: str
    index: int
    n_antennas: int
    n_channels: int
    n_taps: int
    chunk_samples: int
    sigma: float
    max_delay: int
    spectra_per_heap: int = 256
    description: str = ""

    @property
    def seed(self) -> int:
        return synth.SEED_BASE + self.index

    @property
    def N(self) -> int:
        return 2 * self.n_channels

    @property
    def samples_per_step(self) -> int:
        return self.n_antennas * 2 * self.chunk_samples

    def _rng(self):
        return synth.rng(self.seed)

    def tones(self, ant: int, pol: int):
        if self.index == 1:
            return [(192.0 / self.N, 100.0, 0.7 + 0.1 * pol)]
        g = synth.rng(self.seed * 1000 + 10 * ant + pol)
        return [(float(f), float(a), float(p)) for f, a, p in
                zip(g.uniform(0.01, 0.49, 3), g.uniform(20, 100, 3), g.uniform(0, 2 * np.pi, 3))]

    def chirp(self):
        if self.index == 3:
            return (0.05, 0.45, 60.0, 0.0, float(self.chunk_samples))
        return None

    def delays(self):
        """[(ant, pol, delay, rate, phase, phase_rate)] (samples, samples/sample, rad, rad/sample)."""
        out = []
        if self.index == 1:
            for p in range(2):
                out.append((0, p, 7.3, 0.0, 0.1, 0.0))
            return out
        g = self._rng()
        rate = 5e-9 if self.index == 3 else 1e-9
        for a in range(self.n_antennas):
            d0 = float(g.uniform(0, 2000))
            ph = float(g.uniform(0, 2 * np.pi))
            for p in range(2):
                out.append((a, p, d0, rate, ph, 0.0))
        return out

    def gains(self):
        """complex64 [ant, pol, n] or None (unit gains)."""
        if self.index == 1:
            return None
        return synth.random_gains(self.seed + 17, self.n_antennas * 2, self.n_channels).reshape(
            self.n_antennas, 2, self.n_channels)

    def samples(self, ant: int, pol: int, n: int | None = None, start: int = 0) -> np.ndarray:
        n = self.chunk_samples if n is None else n
        return synth.digitiser_samples(self.seed + 101 * ant + 7 * pol, n, self.sigma,
                                       self.tones(ant, pol), self.chirp(), start=start)

    def packed_chunk(self) -> np.ndarray:
        """uint8 [ant, pol, 5 L / 4]: one chunk of every stream."""
        out = np.empty((self.n_antennas, 2, self.chunk_samples * 5 // 4), np.uint8)
        for a in range(self.n_antennas):
            for p in range(2):
                out[a, p] = synth.pack10(self.samples(a, p))
        return out


WORKLOADS = {
    1: Workload("cfg1-1k", 1, 1, 1024, 16, 1 << 20, 32.0, 16,
                description="1 ant x 2 pol, 1024 ch, 16 taps, 2^20 samples/pol, sigma 32 + "
                            "bin-centred tone A=100 at ch 192, coarse 7 + fine 0.3, phase 0.1"),
    2: Workload("cfg2-8k", 2, 4, 8192, 16, 1 << 25, 40.0, 2100,
                description="4 ant x 2 pol, 8192 ch, 16 taps, 2^25 samples/pol per chunk, sigma 40 + "
                            "3 random tones, delays U(0,2000) rate 1e-9, random gains |g| in [0.5,2]"),
    3: Workload("cfg3-32k", 3, 1, 32768, 16, 1 << 28, 24.0, 2100,
                description="1 ant x 2 pol, 32768 ch, 16 taps, 2^28 samples/pol per chunk, sigma 24 + "
                            "linear chirp 0.05->0.45 A=60, delays U(0,2000) rate 5e-9"),
}
