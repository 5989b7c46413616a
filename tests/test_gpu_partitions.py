"""Goldbach partition counts r(n) on the GPU (popcount of the prime bitset AND
its reversal) against the CPU oracle, bit for bit."""
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


@pytest.fixture(scope="module")
def pctx(gbm):
    with gbm.Context(device=0, base_limit=1 << 17) as g:
        yield g


def test_partitions_all_small_n(pctx, oracle):
    lo, hi = 4, 20002
    got = pctx.partitions(lo, hi)
    want = np.array([oracle.partitions(n) for n in range(lo, hi, 2)], dtype=np.uint32)
    np.testing.assert_array_equal(got, want)
    assert got[(100 - 4) // 2] == 6 and got[0] == 1 and got[1] == 1


def test_partitions_ragged_blocks_and_offsets(pctx, oracle):
    # a range starting mid-block, 77 n (not a multiple of 32), near 1e6
    lo = 10**6 + 34
    got = pctx.partitions(lo, lo + 2 * 77)
    want = [oracle.partitions(lo + 2 * j) for j in range(77)]
    assert got.tolist() == want


def test_partitions_large_n_sampled(pctx, oracle):
    lo = (1 << 28) - 40
    got = pctx.partitions(lo, lo + 2 * 64)
    for j in (0, 13, 31, 32, 63):
        assert int(got[j]) == oracle.partitions(lo + 2 * j), j
    # device output equals host output
    out = torch.zeros(64, dtype=torch.int32, device="cuda")
    pctx.partitions(lo, lo + 2 * 64, out=out)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), got)


def test_partitions_near_2_32_consistent(pctx):
    lo = 1 << 32
    a = pctx.partitions(lo, lo + 2 * 40)
    b = pctx.partitions(lo + 2 * 8, lo + 2 * 24)            # a sub-range gives the same counts
    np.testing.assert_array_equal(a[8:24], b)
    assert (a > 0).all()


def test_partitions_rejects_bad_ranges(pctx):
    with pytest.raises(RuntimeError):
        pctx.partitions(5, 11)
    with pytest.raises(RuntimeError):
        pctx.partitions(2, 10)
    with pytest.raises(RuntimeError):
        pctx.partitions(1 << 35, (1 << 35) + 2)
    assert len(pctx.partitions(100, 100)) == 0
