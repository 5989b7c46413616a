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
    oracle's count of (prime, multiple >= p^2) pairs, primes 47..sqrt."""
    import math
    with _ctx(gbm, monkeypatch, mode) as g:
        q = torch.zeros(((nbits + 63) // 64,), dtype=torch.int64, device="cuda")
        gbm.gb_profile_enable(g.handle, True)
        g.sieve_segment(A, nbits, q)
        w = gbm.gb_profile_work(g.handle)
        gbm.gb_profile_enable(g.handle, False)
    last = A + 2 * (nbits - 1)
    assert w["sieve_strikes"] + w["large_strikes"] == oracle.count_strikes(A, nbits, 47, math.isqrt(last))
