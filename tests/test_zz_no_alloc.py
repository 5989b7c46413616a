"""gb_verify_range_noalloc: the entry point for callers that must not allocate
device memory during a call (a request loop sharing the GPU, where cudaMalloc
could synchronize the device, or a caller living inside a fixed memory budget).

Its results must equal the oracle's and gb_verify_range's on the same inputs,
exactly (all outputs are integers), call after call: the scratch array it
shares between calls keeps the previous call's contents, so two different
calls in a row check that nothing leaks from one into the next.  The library's
allocation counter must not move across any of its calls, and the free device
memory must not move across a call once the array's module is loaded.

Collected last (file name), so that a run stopping at the first failure has
run every other test before this one."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

H = 3512   # pi(2^15): histogram entries up to the first-pass bound
P2 = 1 << 20


def _same(a, b):
    for key in ("n_checked", "unresolved", "max_pmin", "max_pmin_n", "hist_len", "n_segments", "p_final"):
        assert a[key] == b[key], key
    assert np.array_equal(a["hist"], b["hist"])
    assert a["segs"] == b["segs"]
    assert np.array_equal(a["seg_hist"], b["seg_hist"])


def _vs_oracle(oracle, got, lo, hi):
    n = (hi - lo) // 2
    summ, hist = oracle.verify_segments(lo, hi, n, P2, H, threads=oracle.default_threads())
    assert got["n_checked"] == n
    assert [got["unresolved"], got["max_pmin"], got["max_pmin_n"]] == [int(x) for x in summ[0, 1:]]
    np.testing.assert_array_equal(got["hist"], hist[0])
    np.testing.assert_array_equal(got["seg_hist"][0], hist[0])


def _noalloc(gb, g, lo, hi, **kw):
    before = gb.gb_alloc_stats()
    out = g.verify_range_noalloc(lo, hi, **kw)
    assert gb.gb_alloc_stats() == before, "gb_verify_range_noalloc allocated"
    return out


@pytest.mark.parametrize("large", ["atomic", "bucket"])
def test_noalloc_first_call_on_fresh_context(oracle, monkeypatch, large):
    """A fresh context whose first call is the no-allocation one, on windows
    near 1.2e13 whose sieving primes pass 2^20 (the large-prime bands, where
    GB_LARGE=bucket would otherwise size its lists), against the oracle."""
    from paper_2603_02621_gb300 import gb
    assert torch.cuda.is_available()
    if large == "bucket":
        monkeypatch.setenv("GB_LARGE", "bucket")
    else:
        monkeypatch.delenv("GB_LARGE", raising=False)
    lo1 = 12 * 10**12
    lo2 = 12 * 10**12 + 2 * 10**8 + 6
    kw = dict(hist_cap=H, seg_hist_stride=H)
    with gb.Context(device=0, base_limit=1 << 22, seg_len=1 << 22, p1=1 << 15, p2=P2) as g:
        a = _noalloc(gb, g, lo1, lo1 + 2 * (1 << 22), **kw)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        b = _noalloc(gb, g, lo2, lo2 + 2 * 3_000_001, **kw)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        _vs_oracle(oracle, a, lo1, lo1 + 2 * (1 << 22))
        _vs_oracle(oracle, b, lo2, lo2 + 2 * 3_000_001)
        # the same inputs through gb_verify_range (which may grow its arenas)
        _same(a, g.verify_range(lo1, lo1 + 2 * (1 << 22), **kw))
        _same(b, g.verify_range(lo2, lo2 + 2 * 3_000_001, **kw))


def test_noalloc_matches_verify_range_twice():
    from paper_2603_02621_gb300 import gb
    assert torch.cuda.is_available()
    with gb.Context(device=0, base_limit=1 << 20, seg_len=1 << 22, p1=1 << 15, p2=P2) as g:
        for lo, hi in [(10**9, 10**9 + 2 * 3 * 10**6), (4, 2 * 10**6 + 2)]:
            kw = dict(hist_cap=H, seg_hist_stride=H)
            ref = g.verify_range(lo, hi, **kw)
            got = _noalloc(gb, g, lo, hi, **kw)
            _same(got, ref)
            # the p_min array path (generic cover kernel), into device memory
            n = (hi - lo) // 2
            pa = torch.zeros(n, dtype=torch.int32, device="cuda")
            pb = torch.zeros(n, dtype=torch.int32, device="cuda")
            ra = g.verify_range(lo, hi, pmin=pa, **kw)
            rb = _noalloc(gb, g, lo, hi, pmin=pb, **kw)
            torch.cuda.synchronize()
            _same(rb, ra)
            assert torch.equal(pa, pb)


def test_noalloc_rejects_oversized_requests():
    from paper_2603_02621_gb300 import gb
    with gb.Context(device=0, base_limit=1 << 20, seg_len=1 << 24, p1=1 << 15, p2=P2) as g:
        with pytest.raises(gb.GbError) as e:
            g.verify_range_noalloc(10**9, 10**9 + 2 * ((1 << 22) + 2))     # more than GB_NOALLOC_MAX_N
        assert e.value.code == gb.GB_ERANGE
        with pytest.raises(gb.GbError) as e:
            g.verify_range_noalloc(10**9, 10**9 + 200, pmin=np.zeros(100, dtype=np.uint32))   # host pmin
        assert e.value.code == gb.GB_EINVAL
