"""The work the cover's roofline divides by: the generic cover kernel counts,
per 64-n word, the odd primes it applies until the word is full; the total
must equal the oracle's count from the p_min values."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gbm():
    from paper_2603_02621_gb300 import gb
    gb.load()
    assert torch.cuda.is_available()
    return gb


@pytest.mark.parametrize("lo,hi,P1,S", [
    (4, 4 + 2 * (1 << 21), 1 << 15, 1 << 20),
    (10**12, 10**12 + 2 * ((1 << 21) + 777), 1 << 15, 1 << 18),
    (10**9, 10**9 + 2 * 300000, 97, 1 << 16),            # many words left open after P1
])
def test_generic_cover_iterations_equal_the_oracle(gbm, oracle, lo, hi, P1, S):
    with gbm.Context(device=0, base_limit=1 << 21, seg_len=S, p1=P1, p2=0, cover_prefix=1) as g:
        gbm.gb_profile_enable(g.handle, True)
        r = g.verify_range(lo, hi)
        w = gbm.gb_profile_work(g.handle)
        gbm.gb_profile_enable(g.handle, False)
    assert r["n_checked"] == (hi - lo) // 2
    assert w["cover_iterations"] == oracle.cover_iterations(lo, hi, P1)


def test_event_only_profiling_counts_no_work(gbm):
    """GB_PROFILE_EVENTS times the kernels with the work counters off (the
    timed kernels are the unprofiled ones); mode 1 counts the same call's work;
    the outputs do not depend on the mode."""
    lo, hi = 10**12, 10**12 + 2 * (1 << 22)
    with gbm.Context(device=0, base_limit=1 << 21, seg_len=1 << 20, p1=1 << 15, p2=1 << 20) as g:
        gbm.gb_profile_enable(g.handle, gbm.GB_PROFILE_EVENTS)
        r0 = g.verify_range(lo, hi, hist_cap=3512)
        w0 = gbm.gb_profile_work(g.handle)
        t0 = gbm.gb_profile_read(g.handle)
        gbm.gb_profile_enable(g.handle, True)
        r1 = g.verify_range(lo, hi, hist_cap=3512)
        w1 = gbm.gb_profile_work(g.handle)
        gbm.gb_profile_enable(g.handle, False)
    assert w0 == dict(sieve_strikes=0, cover_iterations=0, large_strikes=0)
    assert t0["sieve"]["launches"] >= 1 and t0["sieve"]["ms"] > 0 and t0["cover"]["ms"] > 0
    assert w1["sieve_strikes"] > 0 and w1["cover_iterations"] > 0 and w1["large_strikes"] > 0
    assert (r0["max_pmin"], r0["max_pmin_n"], r0["unresolved"]) == (r1["max_pmin"], r1["max_pmin_n"], r1["unresolved"])
    assert (r0["hist"] == r1["hist"]).all()
