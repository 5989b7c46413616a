"""ctypes wrapper around the plain-C oracle (``oracle/gb_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` import this module.  The library under
``paper_2603_02621_gb300/`` never does, and the two share no code.

Every function restates a definition of GoldbachGPU (arXiv 2603.02621):

* ``sieve_window`` -- prime flags of consecutive integers by the sieve of
  Eratosthenes (Sec. 2.1, Sec. 2.3.1);
* ``pmin_range`` / ``verify_segments`` -- the minimal Goldbach prime
  p_min(n) = min{p prime : n - p prime} for each even n, by an ascending scan
  over p <= P (Sec. 2.1, Sec. 2.3.2), and the per-segment histogram, maximum
  and unresolved count built from it (Sec. 2.3.2-2.3.3);
* ``mr_isprime`` -- deterministic Miller-Rabin for 64-bit n (Sec. 2.4);
* ``td_isprime`` / ``td_pmin`` / ``td_partitions`` -- trial division brute
  force, used only to pin the rest;
* ``partitions`` -- the Goldbach partition count c(n) named as future work
  in Sec. 4.5.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liboracle.so``."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC",
                           "-o", tmp, _SRC, "-lpthread", "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u64, i64, u32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32
        vp = ctypes.c_void_p
        lib.or_isqrt.restype = u64
        lib.or_isqrt.argtypes = [u64]
        lib.or_sieve_window.restype = ctypes.c_int
        lib.or_sieve_window.argtypes = [i64, u64, vp]
        lib.or_primes_upto.restype = i64
        lib.or_primes_upto.argtypes = [u64, vp, u64]
        lib.or_pmin_range.restype = ctypes.c_int
        lib.or_pmin_range.argtypes = [u64, u64, u32, vp]
        lib.or_verify_segments.restype = ctypes.c_int
        lib.or_verify_segments.argtypes = [u64, u64, u64, u32, ctypes.c_int,
                                           vp, vp, u32]
        lib.or_td_isprime.restype = ctypes.c_int
        lib.or_td_isprime.argtypes = [u64]
        lib.or_mr_isprime.restype = ctypes.c_int
        lib.or_mr_isprime.argtypes = [u64]
        lib.or_pmin_single.restype = u32
        lib.or_pmin_single.argtypes = [u64, u32]
        lib.or_td_pmin.restype = u64
        lib.or_td_pmin.argtypes = [u64]
        lib.or_partitions.restype = u64
        lib.or_partitions.argtypes = [u64]
        lib.or_td_partitions.restype = u64
        lib.or_td_partitions.argtypes = [u64]
        lib.or_count_strikes.restype = u64
        lib.or_count_strikes.argtypes = [i64, u64, u64, u64]
        lib.or_count_strikes_coprime15.restype = u64
        lib.or_count_strikes_coprime15.argtypes = [i64, u64, u64, u64]
        lib.or_count_strikes_coprime105.restype = u64
        lib.or_count_strikes_coprime105.argtypes = [i64, u64, u64, u64]
        lib.or_prime_pi.restype = u64
        lib.or_prime_pi.argtypes = [u64, ctypes.c_int]
        _lib = lib
        return lib


def default_threads() -> int:
    return os.cpu_count() or 1


def isqrt(x: int) -> int:
    return int(_load().or_isqrt(x))


def sieve_window(a: int, length: int) -> np.ndarray:
    """uint8 flags: out[i] = 1 iff a + i is prime (integers, evens included)."""
    out = np.zeros(length, dtype=np.uint8)
    if length:
        rc = _load().or_sieve_window(a, length, out.ctypes.data)
        assert rc == 0
    return out


def odd_bits(a_odd: int, n_bits: int) -> np.ndarray:
    """uint8 flags of the odd numbers a_odd, a_odd + 2, ... (n_bits of them),
    taken from ``sieve_window``; a_odd may be negative."""
    assert a_odd % 2 == 1 or a_odd % 2 == -1
    f = sieve_window(a_odd, 2 * n_bits)
    return f[0::2].copy()


def primes_upto(x: int) -> np.ndarray:
    lib = _load()
    n = lib.or_primes_upto(x, None, 0)
    out = np.zeros(max(n, 1), dtype=np.uint32)
    lib.or_primes_upto(x, out.ctypes.data, n)
    return out[:n]


def pmin_range(lo: int, hi: int, P: int) -> np.ndarray:
    """uint32 p_min for every even n in [lo, hi) with p <= P (0 = none)."""
    out = np.zeros((hi - lo) // 2, dtype=np.uint32)
    rc = _load().or_pmin_range(lo, hi, P, out.ctypes.data)
    assert rc == 0
    return out


def verify_segments(lo: int, hi: int, S: int, P: int, hist_len: int,
                    threads: int | None = None):
    """Per-segment outputs for segments of S even n from lo.

    Returns (summary, hist): summary is uint64 [nseg, 4] with columns
    n_checked, unresolved, max_pmin, max_pmin_n (smallest n attaining the max),
    and hist is uint64 [nseg, hist_len] with hist[k, i] = #n in segment k whose
    p_min is the i-th prime (p_0 = 2)."""
    nseg = ((hi - lo) // 2 + S - 1) // S
    summ = np.zeros((nseg, 4), dtype=np.uint64)
    hist = np.zeros((nseg, hist_len), dtype=np.uint64)
    rc = _load().or_verify_segments(lo, hi, S, P, threads or default_threads(),
                                    summ.ctypes.data, hist.ctypes.data, hist_len)
    assert rc == 0
    return summ, hist


def td_isprime(n: int) -> bool:
    return bool(_load().or_td_isprime(n))


def mr_isprime(n: int) -> bool:
    return bool(_load().or_mr_isprime(n))


def pmin_single(n: int, P: int) -> int:
    return int(_load().or_pmin_single(n, P))


def td_pmin(n: int) -> int:
    return int(_load().or_td_pmin(n))


def partitions(n: int) -> int:
    return int(_load().or_partitions(n))


def td_partitions(n: int) -> int:
    return int(_load().or_td_partitions(n))


def prime_pi(x: int, threads: int | None = None) -> int:
    return int(_load().or_prime_pi(x, threads or default_threads()))


def count_strikes(a_odd: int, nbits: int, p_lo: int, p_hi: int) -> int:
    """Strikes of the primes in [p_lo, p_hi] (from p^2 on) in the window of
    nbits odd numbers from a_odd."""
    return int(_load().or_count_strikes(a_odd, nbits, p_lo, p_hi))


def count_strikes_coprime15(a_odd: int, nbits: int, p_lo: int, p_hi: int) -> int:
    """As count_strikes, only the multiples j p with j coprime to 15 (the
    strikes left when the multiples of 3 and 5 are cleared already)."""
    return int(_load().or_count_strikes_coprime15(a_odd, nbits, p_lo, p_hi))


def count_strikes_coprime105(a_odd: int, nbits: int, p_lo: int, p_hi: int) -> int:
    """As count_strikes, only the multiples j p with j coprime to 105 (the
    strikes left when the multiples of 3, 5 and 7 are cleared already)."""
    return int(_load().or_count_strikes_coprime105(a_odd, nbits, p_lo, p_hi))


def cover_iterations(lo: int, hi: int, P: int) -> int:
    """Work of a loop-inverted cover over [lo, hi) (Sec. 2.3.1, the cover's
    outer loop over primes): the sum over the 64-n words (word w holds
    n = lo + 2 (64 w .. 64 w + 63)) of the number of odd primes applied in
    ascending order until the word is full -- the largest position, among the
    odd primes 3, 5, 7, ..., of p_min(n) over the word's n; 0 for n = 4
    (p_min 2) and for n past hi; the count of odd primes <= P for an n with no
    p <= P."""
    pm = pmin_range(lo, hi, P).astype(np.int64)
    primes = primes_upto(P).astype(np.int64)
    K = len(primes) - 1
    pos = np.searchsorted(primes, pm)             # 2 -> 0, 3 -> 1, 5 -> 2, ...
    pos[pm == 0] = K
    pad = (-len(pos)) % 64
    pos = np.concatenate([pos, np.zeros(pad, dtype=np.int64)])
    return int(pos.reshape(-1, 64).max(axis=1).sum())
