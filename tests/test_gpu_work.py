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
