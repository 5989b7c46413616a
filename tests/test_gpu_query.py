"""Single-n queries (gb_query / gb_query_batch): p_min(n) of arbitrary even
n < 2^63 on the GPU (window pre-sieve of the partners, deterministic
Miller-Rabin), against the CPU oracle's trial division and Miller-Rabin."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

P2 = 1 << 20
SPSP = 3825123056546413051      # strong pseudoprime to the bases 2..31 (composite: 149491 * 747451 * 34233211)


@pytest.fixture(scope="module")
def gbm():
    from paper_2603_02621_gb300 import gb
    gb.load()
    assert torch.cuda.is_available()
    return gb


@pytest.fixture(scope="module")
def qctx(gbm):
    with gbm.Context(device=0, base_limit=1 << 20, p1=1 << 15, p2=P2) as g:
        yield g


def test_query_small_n_trial_division(qctx, oracle):
    ns = np.arange(4, 10**4 + 1, 2, dtype=np.uint64)
    got = qctx.query_batch(ns)
    want = np.array([oracle.td_pmin(int(n)) for n in ns], dtype=np.uint32)
    np.testing.assert_array_equal(got, want)
    assert qctx.query(4) == 2 and qctx.query(6) == 3 and qctx.query(8) == 3


def test_query_random_large_n(qctx, oracle):
    from paper_2603_02621_gb300.workloads import SplitMix64
    rng = SplitMix64(77)
    ns = [2 * rng.below(2 * 10**18 - 2) + 4 for _ in range(1500)]          # uniform even n < 4e18
    ns += [2 * rng.below(1 << 61) + (1 << 62) for _ in range(300)]        # up to 2^63
    ns += [(1 << 63) - 2, (1 << 63) - 4, 4 * 10**18 - 2, 10**12, 2**32, 2**32 + 2]
    got = qctx.query_batch(ns)
    want = np.array([oracle.pmin_single(n, P2) for n in ns], dtype=np.uint32)
    np.testing.assert_array_equal(got, want)
    for n, p in zip(ns[:200], got[:200]):
        assert oracle.mr_isprime(int(p)) and oracle.mr_isprime(n - int(p))


def test_query_rejects_strong_pseudoprime_partner(qctx, oracle):
    # q = n - 3 passes Miller-Rabin to every base up to 31; only base 37
    # shows it composite, so an incomplete test would answer 3
    for p0 in (3, 5, 7, 11):
        n = SPSP + p0
        got = qctx.query(n)
        assert got != p0
        assert got == oracle.pmin_single(n, P2)


def test_query_bound_and_against_range_path(qctx, oracle):
    # with a small P some n have no partner: p_min 0, as the oracle says
    lo = 10**11                      # within the context's base_limit^2 = 2^40
    ns = np.arange(lo, lo + 2 * 5000, 2, dtype=np.uint64)
    got = qctx.query_batch(ns, 97)
    want = np.array([oracle.pmin_single(int(n), 97) for n in ns], dtype=np.uint32)
    np.testing.assert_array_equal(got, want)
    assert (got == 0).any()
    # the per-n p_min array of the range path agrees with the queries
    pm = torch.zeros(5000, dtype=torch.int32, device="cuda")
    qctx.verify_range(lo, lo + 2 * 5000, pmin=pm)
    np.testing.assert_array_equal(pm.cpu().numpy().view(np.uint32), qctx.query_batch(ns))


def test_query_device_buffers_and_errors(qctx, gbm, oracle):
    ns = torch.tensor([4, 100, 10**18, 3 * 10**18 + 2], dtype=torch.int64, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    qctx.query_batch(ns, out=out)
    assert out.cpu().tolist() == [oracle.pmin_single(int(n), P2) for n in ns.cpu().tolist()]
    with pytest.raises(RuntimeError):
        qctx.query(7)
    with pytest.raises(RuntimeError):
        qctx.query(2)
    bad = torch.tensor([10, 11, 12], dtype=torch.int64, device="cuda")
    out = torch.full((3,), 99, dtype=torch.int32, device="cuda")
    qctx.query_batch(bad, out=out, allow_einval=True)
    assert out.cpu().tolist() == [3, 0, 5]
    assert len(qctx.query_batch([])) == 0
