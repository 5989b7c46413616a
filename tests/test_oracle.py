"""Pins for the CPU oracle, against facts that do not come from the oracle.

Each test checks the oracle against something fixed elsewhere: values printed
in GoldbachGPU (arXiv 2603.02621), standard prime counts, hand-worked cases,
factorizations checked by multiplication, trial-division brute force, and
invariants of the definition p_min(n) = min{p prime : n - p prime}.
"""
import math

import numpy as np
import pytest

from conftest import read_golden
from paper_2603_02621_gb300 import workloads


def facts():
    return {k: int(v) for k, v in read_golden("paper_facts.txt")}


# ---------------------------------------------------------------- sieve

@pytest.mark.parametrize("x,pi", [(int(a), int(b)) for a, b in read_golden("prime_counts.txt")
                                  if int(a) <= 10**9])
def test_prime_pi(oracle, x, pi):
    assert oracle.prime_pi(x) == pi


@pytest.mark.slow
def test_prime_pi_1e10(oracle):
    assert oracle.prime_pi(10**10) == 455052511


def test_pi_1e6_from_paper(oracle):
    # Sec. 3.3: P_SMALL = 10^6 gives 78,498 resident primes
    assert len(oracle.primes_upto(10**6)) == facts()["pi_1e6"]


def test_first_primes_textbook(oracle):
    first25 = [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59,
               61, 67, 71, 73, 79, 83, 89, 97]
    assert oracle.primes_upto(100).tolist() == first25


def test_sieve_window_low_and_negative(oracle):
    # numbers below 2 are not prime; 2 and 3 are
    f = oracle.sieve_window(-7, 20)
    vals = [x for x in range(-7, 13) if f[x + 7]]
    assert vals == [2, 3, 5, 7, 11]


@pytest.mark.parametrize("a", [10**6, 10**9 + 7, 10**12 - 1000, 999_999_999_937])
def test_sieve_window_vs_trial_division(oracle, a):
    f = oracle.sieve_window(a, 2000)
    td = np.array([oracle.td_isprime(a + i) for i in range(2000)], dtype=np.uint8)
    assert np.array_equal(f, td)


@pytest.mark.parametrize("a", [10**15 + 1, 4 * 10**18 - 10**11, 4 * 10**18 - 4001])
def test_sieve_window_high_vs_mr(oracle, a):
    # at these offsets trial division is too slow: compare with Miller-Rabin,
    # itself pinned against trial division below
    f = oracle.sieve_window(a, 3000)
    mr = np.array([oracle.mr_isprime(a + i) for i in range(3000)], dtype=np.uint8)
    assert np.array_equal(f, mr)
    assert f.sum() > 0


def test_odd_bits_layout(oracle):
    # bit i of an odd-only window at base 1 stands for 2i + 1 (Sec. 2.2 layout
    # with the base moved from 3 to 1)
    b = oracle.odd_bits(1, 50)
    assert [2 * i + 1 for i in range(50) if b[i]] == [p for p in oracle.primes_upto(99).tolist() if p != 2]


# ---------------------------------------------------------------- primality

def test_mr_vs_trial_division_small(oracle):
    for n in range(0, 20000):
        assert oracle.mr_isprime(n) == oracle.td_isprime(n), n


def test_mr_vs_trial_division_random(oracle):
    rng = workloads.SplitMix64(12345)
    for _ in range(300):
        n = rng.below(10**12)
        assert oracle.mr_isprime(n) == oracle.td_isprime(n), n


@pytest.mark.parametrize("n,factors", [
    (2047, [23, 89]),
    (3215031751, [151, 751, 28351]),
    (3825123056546413051, [149491, 747451, 34233211]),
])
def test_mr_rejects_strong_pseudoprimes(oracle, n, factors):
    # composites that fool Miller-Rabin with the smallest bases; the
    # factorization (checked here by multiplication) proves them composite
    assert math.prod(factors) == n
    assert not oracle.mr_isprime(n)


def test_mr_known_large_primes(oracle):
    # 2^61 - 1 is a Mersenne prime; 2^64 - 59 is the largest prime below 2^64
    assert oracle.mr_isprime(2**61 - 1)
    assert oracle.mr_isprime(2**64 - 59)
    # 2^64 - 1 = 3 * 5 * 17 * 257 * 641 * 65537 * 6700417
    assert math.prod([3, 5, 17, 257, 641, 65537, 6700417]) == 2**64 - 1
    assert not oracle.mr_isprime(2**64 - 1)


# ---------------------------------------------------------------- p_min

def test_small_pmin_golden(oracle):
    for n, p, q in read_golden("small_pmin.txt"):
        n, p, q = int(n), int(p), int(q)
        assert p + q == n
        pm = oracle.pmin_range(n, n + 2, 1 << 16)
        assert int(pm[0]) == p, n


def test_pmin_bruteforce_to_1e4(oracle):
    pm = oracle.pmin_range(4, 10002, 1 << 16)
    for j, n in enumerate(range(4, 10002, 2)):
        assert int(pm[j]) == oracle.td_pmin(n), n


def test_pmin_bound_P_inclusive_and_unresolved(oracle):
    # p <= P is inclusive; with P below p_min(n) the n is unresolved (0)
    pm = oracle.pmin_range(98, 100, 19)
    assert int(pm[0]) == 19
    pm = oracle.pmin_range(98, 100, 18)
    assert int(pm[0]) == 0


def test_pmin_invariants_high_offsets(oracle):
    # p_min and n - p_min prime; no smaller prime works (Miller-Rabin, pinned above)
    rng = workloads.SplitMix64(99)
    primes = oracle.primes_upto(1 << 15).tolist()
    for base in (10**12, 10**15, 4 * 10**18 - 10**11):
        lo = base + 2 * rng.below(10**6)
        lo -= lo & 1
        pm = oracle.pmin_range(lo, lo + 400, 1 << 15)
        for j in range(0, 200, 7):
            n = lo + 2 * j
            p = int(pm[j])
            assert p > 0
            assert oracle.mr_isprime(p) and oracle.mr_isprime(n - p)
            for r in primes:
                if r >= p:
                    break
                assert not oracle.mr_isprime(n - r)
            assert oracle.pmin_single(n, 1 << 15) == p


def test_pmin_bruteforce_sample_1e12(oracle):
    # at 10^12 trial division of n - p is still affordable for a few n
    lo = 10**12 - 200
    pm = oracle.pmin_range(lo, lo + 40, 1 << 15)
    for j in range(0, 20, 3):
        n = lo + 2 * j
        p = int(pm[j])
        assert oracle.td_isprime(p) and oracle.td_isprime(n - p)
        for r in range(3, p, 2):
            if oracle.td_isprime(r):
                assert not oracle.td_isprime(n - r)


# ---------------------------------------------------------------- segments

def test_verify_segments_consistency(oracle):
    lo, hi, S, P = 4, 2 * 10**6 + 2, 1 << 16, 1 << 12
    primes = oracle.primes_upto(P).tolist()
    H = len(primes)
    summ, hist = oracle.verify_segments(lo, hi, S, P, H)
    pm = oracle.pmin_range(lo, hi, P)
    nseg = summ.shape[0]
    assert nseg == ((hi - lo) // 2 + S - 1) // S
    idx = {p: i for i, p in enumerate(primes)}
    for k in range(nseg):
        seg = pm[k * S:(k + 1) * S]
        assert summ[k, 0] == len(seg)
        assert summ[k, 1] == int((seg == 0).sum())
        assert int(hist[k].sum()) + int(summ[k, 1]) == len(seg)
        mx = int(seg.max())
        assert summ[k, 2] == mx
        first = int(np.argmax(seg == mx))
        assert summ[k, 3] == lo + 2 * (k * S + first)   # smallest n attaining the max
        ref = np.zeros(H, dtype=np.uint64)
        for p in seg[seg > 0].tolist():
            ref[idx[p]] += 1
        assert np.array_equal(hist[k], ref)


def test_segmentation_invariance(oracle):
    lo, hi, P = 10**9, 10**9 + 3 * 10**6, 1 << 15
    H = len(oracle.primes_upto(P))
    a, ha = oracle.verify_segments(lo, hi, 1 << 18, P, H)
    b, hb = oracle.verify_segments(lo, hi, 1 << 20, P, H)
    assert np.array_equal(ha.sum(axis=0), hb.sum(axis=0))
    assert a[:, 1].sum() == b[:, 1].sum() == 0
    ia, ib = int(np.argmax(a[:, 2])), int(np.argmax(b[:, 2]))
    assert (a[ia, 2], a[ia, 3]) == (b[ib, 2], b[ib, 3])


def test_even_counts_from_paper(oracle):
    # Tables 1 and 4: [4, N] holds N/2 - 1 even n; half-open [4, N + 2)
    f = facts()
    for N, key in [(10**7, "even_checked_1e7"), (10**8, "even_checked_1e8")]:
        summ, _ = oracle.verify_segments(4, N + 2, 1 << 24, 1 << 10, 1)
        assert int(summ[:, 0].sum()) == f[key]


def test_no_unresolved_with_psmall_1e6_to_1e8(oracle):
    # Sec. 3.3 / Table 4: with P_SMALL = 10^6 no n up to 10^12 needs Phase 2;
    # checked here to 10^8 (P = 2^20 > 10^6 covers the same claim)
    summ, _ = oracle.verify_segments(4, 10**8 + 2, 1 << 24, 10**6, 1)
    assert int(summ[:, 1].sum()) == facts()["unresolved_psmall_1e6"]


# ---------------------------------------------------------------- partitions

def test_partitions_hand_values(oracle):
    # c(n) = #{p <= n/2 : p, n - p prime}; 100 = 3+97 = 11+89 = 17+83 = 29+71 = 41+59 = 47+53
    assert [oracle.partitions(n) for n in (4, 6, 8, 10, 100)] == [1, 1, 1, 2, 6]


def test_partitions_bruteforce(oracle):
    for n in range(4, 3000, 2):
        assert oracle.partitions(n) == oracle.td_partitions(n), n


@pytest.mark.parametrize("a,nbits,plo,phi", [
    (1, 5000, 3, 10**6),
    (10**6 + 1, 3001, 47, 10**6),
    (10**9 + 7, 999, 5, 31),
    (-41, 300, 3, 100),
])
def test_strike_count_brute_force(oracle, a, nbits, plo, phi):
    # every odd number of the window, every prime in range: multiples >= p^2
    last = a + 2 * (nbits - 1)
    primes = [p for p in oracle.primes_upto(min(phi, math.isqrt(max(last, 0)))).tolist() if p >= plo and p > 2]
    want = 0
    for i in range(nbits):
        m = a + 2 * i
        if m < 4:
            continue
        want += sum(1 for p in primes if m % p == 0 and m >= p * p)
    assert oracle.count_strikes(a, nbits, plo, phi) == want


@pytest.mark.parametrize("a,nbits,plo,phi", [
    (1, 5000, 3, 10**6),
    (10**6 + 1, 3001, 47, 10**6),
    (10**9 + 7, 999, 5, 31),
    (-41, 300, 3, 100),
    (10**12 + 1, 4001, 7, 10**6),
])
def test_strike_count_coprime15_brute_force(oracle, a, nbits, plo, phi):
    # every odd number m = j p of the window, p in range, m >= p^2, with the
    # cofactor j coprime to 15
    last = a + 2 * (nbits - 1)
    primes = [p for p in oracle.primes_upto(min(phi, math.isqrt(max(last, 0)))).tolist() if p >= plo and p > 2]
    want = 0
    for i in range(nbits):
        m = a + 2 * i
        if m < 4:
            continue
        want += sum(1 for p in primes if m % p == 0 and m >= p * p and math.gcd(m // p, 15) == 1)
    got = oracle.count_strikes_coprime15(a, nbits, plo, phi)
    assert got == want
    # the cofactors divisible by 3 or 5 are exactly the rest
    if plo > 5:
        assert got < oracle.count_strikes(a, nbits, plo, phi) or want == 0


@pytest.mark.parametrize("a,nbits,plo,phi", [
    (1, 5000, 3, 1000),
    (10**6 + 1, 3001, 47, 10**6),
    (10**9 + 7, 999, 5, 31),
    (-41, 300, 3, 100),
    (10**12 + 1, 4001, 7, 10**6),
    (4 * 10**18 - 10**11 + 1, 2001, 1 << 20, 1 << 22),
])
def test_strike_count_coprime105_brute_force(oracle, a, nbits, plo, phi):
    # every odd number m = j p of the window, p in range, m >= p^2, with the
    # cofactor j coprime to 105
    last = a + 2 * (nbits - 1)
    r = min(phi, math.isqrt(max(last, 0)))
    if a > 10**15:
        # too far for a prime list to sqrt: test each candidate factor p of m
        # directly, with p prime by trial division (p < 2^22)
        cands = [p for p in range(plo | 1, r + 1, 2) if oracle.mr_isprime(p)]
    else:
        cands = [p for p in oracle.primes_upto(r).tolist() if p >= plo and p > 2]
    want = 0
    for p in cands:
        j0 = max(-(-max(a, 4) // p), p)
        j0 += (j0 + 1) % 2                       # odd cofactor (m odd)
        for j in range(j0, last // p + 1, 2):
            if math.gcd(j, 105) == 1:
                want += 1
    got = oracle.count_strikes_coprime105(a, nbits, plo, phi)
    assert got == want
    # the cofactors coprime to 15 but divisible by 7 are the difference
    extra = sum(1 for p in cands for j in range(max(-(-max(a, 4) // p), p), last // p + 1)
                if j % 2 and math.gcd(j, 15) == 1 and j % 7 == 0)
    assert oracle.count_strikes_coprime15(a, nbits, plo, phi) - got == extra


def test_cover_iterations_worked_by_hand(oracle):
    # one 64-n word, n = 4 .. 130: the largest p_min there is 19 (at n = 98
    # and n = 128: n - 3, ..., n - 17 are all composite, n - 19 is prime),
    # the 7th odd prime; with P = 13 those n stay open and the word costs all
    # 5 odd primes <= 13
    assert oracle.pmin_single(98, 100) == 19 and oracle.pmin_single(128, 100) == 19
    assert oracle.cover_iterations(4, 132, 1 << 10) == 7
    assert oracle.cover_iterations(4, 132, 13) == 5
    # words are independent: two words cost the sum of each alone
    assert oracle.cover_iterations(4, 260, 1 << 10) == 7 + oracle.cover_iterations(132, 260, 1 << 10)
    # a range of one n = 4 costs nothing
    assert oracle.cover_iterations(4, 6, 1 << 10) == 0
