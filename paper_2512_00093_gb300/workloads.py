"""Seeded synthetic workloads (inputs only; no generator arithmetic here).

The paper measures 10^9 outputs of one stream (Table 1) and jumps of
J = 2^64 - 1 and 2^120 - 1 (Table 2); it uses no dataset.  These recipes
restate those workloads for many streams at once.  Both the CUDA path and the
CPU oracle take their inputs from here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED = 12345


@dataclass(frozen=True)
class Tiny:
    """One stream, 10^6 outputs (u24 and f32), plus one jump of 10^6."""
    seed: int = SEED
    count: int = 10**6
    jump: int = 10**6


@dataclass(frozen=True)
class Partitioned:
    """65,536 streams at k*J, J = 2^40, 4,096 u24 outputs each, written as
    a row-per-stream [65,536 x 4,096] array."""
    seed: int = SEED
    n_streams: int = 65536
    J: int = 1 << 40
    count: int = 4096
    k0: int = 0
    n_verify: int = 256
    verify_seed: int = 2024

    def verify_rows(self) -> np.ndarray:
        rng = np.random.default_rng(self.verify_seed)
        return np.sort(rng.choice(self.n_streams, size=self.n_verify, replace=False))


@dataclass(frozen=True)
class BatchedUneven:
    """10^6 streams at k*J, J = 2^64, lengths floor(64 * 1024^u) with
    u ~ U[0, 1) from numpy default_rng(7), clipped to [64, 65536]; f32
    outputs packed back to back (offsets = exclusive prefix sum)."""
    seed: int = SEED
    n_streams: int = 10**6
    J: int = 1 << 64
    len_seed: int = 7
    lo: int = 64
    hi: int = 65536

    def lengths(self, n: int | None = None) -> np.ndarray:
        n = self.n_streams if n is None else n
        u = np.random.default_rng(self.len_seed).random(self.n_streams)[:n]
        return np.clip(np.floor(self.lo * np.power(1024.0, u)), self.lo, self.hi).astype(np.int64)


@dataclass(frozen=True)
class LargeJumps:
    """16,384 streams at k*J with J = 2^120 + 12,345, 1,024 u24 outputs."""
    seed: int = SEED
    n_streams: int = 16384
    J: int = (1 << 120) + 12345
    count: int = 1024


@dataclass(frozen=True)
class Serving:
    """Poisson request stream: mean 20k req/s for 60 s (seed 11); seed
    uniform in 1..10^4, stream index uniform in 0..2^20, J = 2^48, count
    floor(10^(3 + 4u)), dtype u24 or f32 with probability 1/2."""
    rate: float = 20000.0
    duration: float = 60.0
    rng_seed: int = 11
    J: int = 1 << 48

    def requests(self, duration: float | None = None):
        dur = self.duration if duration is None else duration
        rng = np.random.default_rng(self.rng_seed)
        n = rng.poisson(self.rate * dur)
        t = np.sort(rng.random(n) * dur)
        seeds = rng.integers(1, 10**4 + 1, n)
        ks = rng.integers(0, (1 << 20) + 1, n)
        counts = np.floor(10.0 ** (3.0 + 4.0 * rng.random(n))).astype(np.int64)
        f32 = rng.random(n) < 0.5
        return t, seeds, ks, counts, f32


@dataclass(frozen=True)
class ServingHot:
    """A labelled variant of the serving stream in which requests revisit a
    small set of streams (seeds 1..64, stream index 0..15: 1,024 streams), so
    that most requests resume a stream an earlier request left resident:
    Poisson 20k req/s for 10 s (seed 13), J = 2^48, count
    floor(10^(3 + 3u)), u24 or f32 with probability 1/2."""
    rate: float = 20000.0
    duration: float = 10.0
    rng_seed: int = 13
    J: int = 1 << 48
    seeds: int = 64
    ks: int = 16

    def requests(self, duration: float | None = None):
        dur = self.duration if duration is None else duration
        rng = np.random.default_rng(self.rng_seed)
        n = rng.poisson(self.rate * dur)
        t = np.sort(rng.random(n) * dur)
        seeds = rng.integers(1, self.seeds + 1, n)
        ks = rng.integers(0, self.ks, n)
        counts = np.floor(10.0 ** (3.0 + 3.0 * rng.random(n))).astype(np.int64)
        f32 = rng.random(n) < 0.5
        return t, seeds, ks, counts, f32


def random_exponents(n: int, max_bits: int, seed: int) -> list[int]:
    """n exponents with bit lengths spread over 0..max_bits (edge cases first)."""
    rng = np.random.default_rng(seed)
    fixed = [0, 1, 2, 5, 6, 7, 63, 64, 96, 97, 98, 193, 1000, 10**6, (1 << 40),
             (1 << 64) - 1, (1 << 120) - 1, (1 << 120) + 12345, (1 << max_bits) - 1]
    out = [e for e in fixed if e < (1 << max_bits)]
    while len(out) < n:
        bits = int(rng.integers(1, max_bits + 1))
        e = 0
        for w in range((bits + 31) // 32):
            e |= int(rng.integers(0, 1 << 32)) << (32 * w)
        out.append(e & ((1 << bits) - 1))
    return out[:n]
