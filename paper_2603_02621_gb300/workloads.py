"""Seeded synthetic inputs for the Goldbach verifier.

This module holds no arithmetic of the method (no sieving, no primality, no
cover): it only turns a seed into the integer ranges, sample indices and
request streams that both the CUDA path and the CPU oracle are given.  The
generator is splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), written out from its published definition.

Workload shapes (GoldbachGPU, arXiv 2603.02621, exhaustive verification of
every even n in a range, Sec. 2.3 and Table 4):

* ``batched_ranges``: many ranges of uneven length and offset, lengths
  log-uniform in [2^10, 2^26] even integers, starts uniform in
  [10^9, 10^15] rounded down to even;
* ``serving_stream``: Poisson arrivals mixing range queries (log-uniform
  2^16..2^30 evens, offsets uniform in [10^9, 4e18]) and single-n queries
  (uniform even n < 4e18);
* ``sample_indices``: seeded distinct indices, for sampled oracle checks of
  large configurations.
"""
from __future__ import annotations

import math

MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64: state += golden gamma; output = a two-round xor-shift-multiply
    finaliser of the state."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, n: int) -> int:
        """integer in [0, n) (n < 2^64), by rejection of the biased tail."""
        if n <= 0:
            raise ValueError("n must be positive")
        lim = (1 << 64) - ((1 << 64) % n)
        while True:
            x = self.next_u64()
            if x < lim:
                return x % n


def batched_ranges(count: int = 4096, seed: int = 1,
                   log2_min: int = 10, log2_max: int = 26,
                   start_min: int = 10**9, start_max: int = 10**15):
    """List of (lo, hi) half-open even-n ranges: length 2^(a + (b-a)u) even n,
    start uniform in [start_min, start_max] rounded down to even."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        u = rng.uniform()
        length = int(round(2.0 ** (log2_min + (log2_max - log2_min) * u)))
        length = max(1, length)
        start = start_min + rng.below(start_max - start_min + 1)
        start -= start & 1
        out.append((start, start + 2 * length))
    return out


def sample_indices(n: int, k: int, seed: int):
    """k distinct indices in [0, n), ascending."""
    rng = SplitMix64(seed)
    k = min(k, n)
    chosen = set()
    while len(chosen) < k:
        chosen.add(rng.below(n))
    return sorted(chosen)


def serving_stream(count: int, seed: int = 7, rate: float = 2000.0,
                   range_frac: float = 0.9, log2_min: int = 16, log2_max: int = 30,
                   off_min: int = 10**9, off_max: int = 4 * 10**18,
                   n_max: int = 4 * 10**18):
    """Request list [(t_arrival_s, kind, a, b)]: kind 'range' with even-n range
    [a, b), or kind 'query' with a = the even n and b = 0."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate
        if rng.uniform() < range_frac:
            u = rng.uniform()
            length = int(round(2.0 ** (log2_min + (log2_max - log2_min) * u)))
            start = off_min + rng.below(off_max - off_min + 1)
            start -= start & 1
            out.append((t, "range", start, start + 2 * length))
        else:
            n = 4 + rng.below(n_max - 4)
            n -= n & 1
            out.append((t, "query", n, 0))
    return out
