"""Bucket sieve of the primes above the tile split (per-tile hit lists applied
in shared memory) against the global-atomic strikes (GB_LARGE=atomic) and the
CPU oracle, bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gbm():
    from paper_2603_02621_gb300 import gb
    gb.load()
    assert torch.cuda.is_available()
    return gb


def _ctx(gbm, monkeypatch, mode, **kw):
    monkeypatch.setenv("GB_LARGE", mode)
    cfg = dict(device=0, base_limit=1 << 31, p1=1 << 15, p2=1 << 20)
    cfg.update(kw)
    return gbm.Context(**cfg)


def _tile_strikes(oracle, A, nbits, p_end):
    """The oracle's count of the strikes the tile sieve and the slices make
    for the primes 47 .. p_end - 1, with the default tile (2^18 bits): every
    odd multiple (>= p^2) for the warp-struck primes (below 512) and for the
    slices' primes from 2^16 on, only those with the cofactor coprime to 15
    for the primes between (the mod-30 wheel of the tile's one-thread primes
    and of the slices' primes below 2^16).  The split between tile and slices
    is 2^13 once the window's sieving primes reach 2^18, else the tile."""
    import math
    last = A + 2 * (nbits - 1)
    split = 1 << 13 if math.isqrt(last) >= 1 << 18 else 1 << 18
    wheel_end = min(max(split, 1 << 16), p_end)
    n = oracle.count_strikes(A, nbits, 47, 511) + oracle.count_strikes_coprime15(A, nbits, 512, wheel_end - 1)
    if p_end > wheel_end:
        n += oracle.count_strikes(A, nbits, wheel_end, p_end - 1)
    return n


def _sieve(g, A, nbits):
    words = (nbits + 63) // 64
    q = torch.full((words,), -1, dtype=torch.int64, device="cuda")
    pc = g.sieve_segment(A, nbits, q)
    return q.cpu().numpy(), pc


@pytest.mark.parametrize("A,nbits,kw", [
    (4 * 10**18 - 10**11 + 1, (1 << 30) + 12345, {}),                 # two chunks, ragged tail
    (10**15 + 1, (1 << 22) + 77, dict(bucket_split=1 << 12)),           # small primes in the lists
    (2 * 10**18 + 1, (1 << 21) + 64, dict(tile_bits=1 << 16, bucket_split=1 << 16)),
])
def test_bucket_equals_atomic(gbm, monkeypatch, oracle, A, nbits, kw):
    with _ctx(gbm, monkeypatch, "bucket", **kw) as g:
        qb, pb = _sieve(g, A, nbits)
    with _ctx(gbm, monkeypatch, "atomic", **kw) as g:
        qa, pa = _sieve(g, A, nbits)
    np.testing.assert_array_equal(qb, qa)
    assert pb == pa
    # sampled bits against the oracle's Miller-Rabin
    from paper_2603_02621_gb300.workloads import sample_indices
    bits = np.unpackbits(qb.view(np.uint8), bitorder="little")
    for i in sample_indices(nbits, 3000, seed=5):
        assert bool(bits[i]) == oracle.mr_isprime(A + 2 * i), i
    # every bit of a short stretch against the oracle's window sieve
    ref = oracle.odd_bits(A, 1 << 16)
    np.testing.assert_array_equal(bits[:1 << 16], ref)


def test_bucket_window_vs_oracle_full(gbm, monkeypatch, oracle):
    A, nbits = 10**12 + 1, (1 << 22) + 3
    with _ctx(gbm, monkeypatch, "bucket", bucket_split=1 << 10) as g:
        qb, pc = _sieve(g, A, nbits)
    bits = np.unpackbits(qb.view(np.uint8), bitorder="little")
    ref = oracle.odd_bits(A, nbits)
    np.testing.assert_array_equal(bits[:nbits], ref)
    assert not bits[nbits:].any()
    assert pc == int(ref.sum())


@pytest.mark.parametrize("A,nbits,mode", [
    (10**9 + 1, 3 * (1 << 18) + 128, "atomic"),          # tile primes only
    (10**12 - 999, (1 << 22) + 64, "atomic"),            # tile + slice primes (below 2^20)
    (4 * 10**18 - 10**11 + 1, (1 << 26) + 64, "atomic"),  # tile + slice + atomic large primes
    (4 * 10**18 - 10**11 + 1, (1 << 26) + 64, "bucket"),  # ... with the bucket lists
])
def test_strike_counters_equal_the_oracle(gbm, monkeypatch, oracle, A, nbits, mode):
    """The work the roofline divides by: the kernels' strike counters equal the
    oracle's count of (prime, multiple >= p^2) pairs, primes 47..sqrt (the
    one-thread primes of the tile: cofactors coprime to 15)."""
    import math
    with _ctx(gbm, monkeypatch, mode) as g:
        q = torch.zeros(((nbits + 63) // 64,), dtype=torch.int64, device="cuda")
        gbm.gb_profile_enable(g.handle, True)
        g.sieve_segment(A, nbits, q)
        w = gbm.gb_profile_work(g.handle)
        gbm.gb_profile_enable(g.handle, False)
    last = A + 2 * (nbits - 1)
    assert w["sieve_strikes"] + w["large_strikes"] == _tile_strikes(oracle, A, nbits, math.isqrt(last) + 1)


@pytest.mark.parametrize("A,nbits", [
    (4 * 10**18 - 10**11 + 1, (1 << 30) + 12345),    # dense and bucketed primes, four chunks and a ragged tail
    (10**15 + 1, (1 << 29) + 777),                    # every carried prime below half a chunk
    (10**14 + 1, (1 << 31) + 64),                     # the top primes have p^2 inside the window
    ((1 << 62) - (1 << 30) + 1, (1 << 29) + 5),       # primes up to 2^31: the widest bucket ring
])
def test_carry_equals_atomic(gbm, monkeypatch, oracle, A, nbits):
    """The large primes started once per window and carried from chunk to
    chunk (default; multiples m p with m coprime to 210) give the same bits as
    the per-chunk restart with every odd multiple (GB_LARGE=atomic), and
    sampled bits agree with the oracle's Miller-Rabin."""
    monkeypatch.delenv("GB_LARGE", raising=False)
    with gbm.Context(device=0, base_limit=1 << 31, p1=1 << 15, p2=1 << 20) as g:
        qc, pc = _sieve(g, A, nbits)
    with _ctx(gbm, monkeypatch, "atomic") as g:
        qa, pa = _sieve(g, A, nbits)
    np.testing.assert_array_equal(qc, qa)
    assert pc == pa
    from paper_2603_02621_gb300.workloads import sample_indices
    bits = np.unpackbits(qc.view(np.uint8), bitorder="little")
    for i in sample_indices(nbits, 2000, seed=7):
        assert bool(bits[i]) == oracle.mr_isprime(A + 2 * i), i


@pytest.mark.parametrize("A,nbits", [
    (4 * 10**18 - 10**11 + 1, (1 << 29) + 64),
    (10**14 + 1, (1 << 30) + 64),
])
def test_carry_strike_counter_equals_the_oracle(gbm, monkeypatch, oracle, A, nbits):
    """The work counted by the carried large primes: strikes of m p with m
    coprime to 105 for the primes from 2^20 to sqrt(A); below 2^20 the tile's
    and the slices' strikes (_tile_strikes), above sqrt(A) (p^2 inside the
    window) every odd multiple."""
    import math
    monkeypatch.delenv("GB_LARGE", raising=False)
    with gbm.Context(device=0, base_limit=1 << 31, p1=1 << 15, p2=1 << 20) as g:
        q = torch.zeros(((nbits + 63) // 64,), dtype=torch.int64, device="cuda")
        gbm.gb_profile_enable(g.handle, True)
        g.sieve_segment(A, nbits, q)
        w = gbm.gb_profile_work(g.handle)
        gbm.gb_profile_enable(g.handle, False)
    last = A + 2 * (nbits - 1)
    r0, r1 = math.isqrt(A), math.isqrt(last)
    want = (_tile_strikes(oracle, A, nbits, 1 << 20) + oracle.count_strikes_coprime105(A, nbits, 1 << 20, r0)
            + oracle.count_strikes(A, nbits, r0 + 1, r1))
    assert w["sieve_strikes"] + w["large_strikes"] == want


@pytest.mark.parametrize("cap", [1, 64])
def test_carry_full_columns_strike_through(gbm, monkeypatch, cap):
    """Bucket columns far too small (GB_CARRY_CAP): most carried primes find
    their column full and strike the rest of the window at once; the bits
    are the same as the per-chunk restart's."""
    A, nbits = 4 * 10**18 - 10**11 + 1, (1 << 29) + 12345
    monkeypatch.setenv("GB_CARRY_CAP", str(cap))
    monkeypatch.delenv("GB_LARGE", raising=False)
    with gbm.Context(device=0, base_limit=1 << 31, p1=1 << 15, p2=1 << 20) as g:
        qc, pc = _sieve(g, A, nbits)
    monkeypatch.delenv("GB_CARRY_CAP")
    with _ctx(gbm, monkeypatch, "atomic") as g:
        qa, pa = _sieve(g, A, nbits)
    np.testing.assert_array_equal(qc, qa)
    assert pc == pa


def test_carry_stops_below_2_31(gbm, monkeypatch, oracle):
    """Above 2^62 the sieving primes pass 2^31; a bucket entry holds p / 2 in
    30 bits, so the carried primes stop at 2^31 and the larger ones restart
    in every chunk.  A range near 8e18 whose q window spans two chunks: every
    segment's record and histogram row equal the per-chunk restart's
    (GB_LARGE=atomic), and one seeded segment equals the oracle's."""
    lo, hi, S = 8 * 10**18, 8 * 10**18 + 2 * (1 << 29), 1 << 24
    kw = dict(hist_cap=3512, segs=True, seg_hist_stride=3512)
    monkeypatch.delenv("GB_LARGE", raising=False)
    with gbm.Context(device=0, base_limit=1 << 32, seg_len=S, p1=1 << 15, p2=1 << 20) as g:
        rc = g.verify_range(lo, hi, **kw)
    with _ctx(gbm, monkeypatch, "atomic", base_limit=1 << 32, seg_len=S) as g:
        ra = g.verify_range(lo, hi, **kw)
    rec = lambda r: [(s["n_checked"], s["unresolved"], s["max_pmin"], s["max_pmin_n"]) for s in r["segs"]]
    assert rec(rc) == rec(ra) and len(rc["segs"]) == 32
    np.testing.assert_array_equal(rc["seg_hist"], ra["seg_hist"])
    from paper_2603_02621_gb300.workloads import sample_indices
    k = int(sample_indices(32, 1, seed=5)[0])
    s = rc["segs"][k]
    summ, hist = oracle.verify_segments(s["lo"], s["hi"], S, 1 << 20, 3512)
    assert [s["n_checked"], s["unresolved"], s["max_pmin"], s["max_pmin_n"]] == summ[0].tolist()
    np.testing.assert_array_equal(rc["seg_hist"][k], hist[0])
