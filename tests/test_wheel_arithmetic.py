"""The sieve kernels' start and wheel arithmetic, checked on the CPU.

The tile sieve and the slices strike only the multiples m p with m coprime
to 15 for most primes (a mod-30 wheel), and find a prime's first multiple in
a slice from a residue table instead of a 64-bit reduction.  The constants
of the wheel are read from the kernel header and checked against their
definition; the kernels' integer formulas are replayed here in 32-bit
arithmetic and compared with the plain definition (first odd multiple,
cofactor coprime to 15) on random primes and windows.  The GPU tests then
check the kernels themselves against the oracle."""
import math
import os
import random
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TILE = os.path.join(ROOT, "paper_2603_02621_gb300", "csrc", "gb_sieve_tile.cuh")
M32 = (1 << 32) - 1
SLICE_BITS = 7 << 18                 # kMidSliceBits


def _const(name):
    src = open(TILE).read()
    m = re.search(r"constexpr\s+uint(?:32|64)_t\s+" + name + r"\s*=\s*(0x[0-9a-fA-F]+)", src)
    assert m, name
    return int(m.group(1), 16)


RES30 = [r for r in range(1, 30) if math.gcd(r, 30) == 1]          # the 8 coprime residues


def test_wheel_constants_follow_their_definition():
    half_gaps, next_pos, next_half = _const("kHalfGaps30"), _const("kNextPos30"), _const("kNextHalf30")
    for w in range(8):
        nxt = RES30[w + 1] if w < 7 else 31
        assert (half_gaps >> (4 * w)) & 15 == (nxt - RES30[w]) // 2
    for j in range(15):
        m = 2 * j + 1
        c = next(r for r in RES30 + [31] if r >= m)
        assert (next_pos >> (3 * j)) & 7 == RES30.index(c) % 8
        assert (next_half >> (2 * j)) & 3 == (c - m) // 2


def _first_odd_multiple(b, p):
    r = (-b) % p
    return (r + p) >> 1 if r & 1 else r >> 1


def _wheel_walk(b, p, i, nb):
    """The kernels' walk from the first multiple's index i (b + 2i = m p, m
    odd): the cofactor's residue mod 30 from (b + 2i) p^3, the first coprime
    residue from there, then the rotating register of half gaps."""
    half_gaps, next_pos, next_half = _const("kHalfGaps30"), _const("kNextPos30"), _const("kNextHalf30")
    pm = p % 30
    inv = pm * pm % 30 * pm % 30
    j = ((b % 30 + 2 * (i % 15)) % 30 * inv % 30) >> 1
    pos = (next_pos >> (3 * j)) & 7
    i += p * ((next_half >> (2 * j)) & 3)
    g = ((half_gaps >> (4 * pos)) | (half_gaps << (32 - 4 * pos))) & M32 if pos else half_gaps
    out = []
    while i < nb:
        out.append(i)
        i += p * (g & 15)
        g = ((g >> 4) | (g << 28)) & M32
    return out


def test_wheel_walk_strikes_the_cofactors_coprime_to_15():
    rng = random.Random(3)
    primes = [p for p in range(47, 1 << 16, 2) if all(p % d for d in range(3, int(p ** 0.5) + 1, 2))]
    for _ in range(3000):
        p = rng.choice(primes)
        nb = rng.choice([1 << 18, rng.randrange(64, 1 << 18, 64)])
        b = rng.randrange(-(1 << 20), 1 << 60) | 1
        i = _first_odd_multiple(b, p)
        if p * p > b:
            i = max(i, (p * p - b) >> 1)
        if i >= nb:
            continue
        want = [k for k in range(i, nb, p) if math.gcd((b + 2 * k) // p, 15) == 1]
        assert _wheel_walk(b, p, i, nb) == want


def test_residue_start_equals_the_first_odd_multiple():
    """The slices' start: (-b_s) mod p for slice s of a window at B from
    (-B) mod p and s (2S mod p), the product (< 2^33) reduced with
    floor(2^33 / p) in 32-bit arithmetic (quotient at most two short)."""
    rng = random.Random(5)
    for _ in range(20000):
        p = rng.randrange(3, 1 << 20) | 1
        B = rng.choice([rng.randrange(-(1 << 21), 1 << 21) | 1, rng.randrange(1, (1 << 63) - (1 << 40)) | 1])
        s = rng.choice([0, 1, 8191, rng.randrange(0, 8192)])
        rb, c, m2 = (-B) % p, (2 * SLICE_BITS) % p, (1 << 33) // p
        t = s * c
        assert t < 1 << 33
        qt = ((t >> 1) * m2) >> 32
        r = (t - qt * p) & M32
        assert r < 3 * p
        r = r - p if r >= p else r
        r = r - p if r >= p else r
        x = rb - r if rb >= r else rb + (p - r)
        start = (x + p) >> 1 if x & 1 else x >> 1
        assert start == _first_odd_multiple(B + 2 * s * SLICE_BITS, p)
