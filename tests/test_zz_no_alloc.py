"""gb_verify_range_noalloc: the entry point for callers that must not allocate
device memory during a call (a request loop sharing the GPU, where cudaMalloc
could synchronize the device, or a caller living inside a fixed memory budget).
Its results must equal gb_verify_range's on the same inputs, exactly (all
outputs are integers), call after call: the scratch array it shares between
calls keeps the previous call's contents, so two different calls in a row
check that nothing leaks from one into the next.

Collected last (file name), so that a run stopping at the first failure has
run every other test before this one."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

H = 3512   # pi(2^15): histogram entries up to the first-pass bound


def _same(a, b):
    for key in ("n_checked", "unresolved", "max_pmin", "max_pmin_n", "hist_len", "n_segments", "p_final"):
        assert a[key] == b[key], key
    assert np.array_equal(a["hist"], b["hist"])
    assert a["segs"] == b["segs"]
    assert np.array_equal(a["seg_hist"], b["seg_hist"])


def test_noalloc_matches_verify_range_twice():
    from paper_2603_02621_gb300 import gb
    assert torch.cuda.is_available()
    with gb.Context(device=0, base_limit=1 << 20, seg_len=1 << 22, p1=1 << 15, p2=1 << 20) as g:
        for lo, hi in [(10**9, 10**9 + 2 * 3 * 10**6), (4, 2 * 10**6 + 2)]:
            kw = dict(hist_cap=H, seg_hist_stride=H)
            ref = g.verify_range(lo, hi, **kw)
            got = g.verify_range_noalloc(lo, hi, **kw)
            _same(got, ref)
            # the p_min array path (generic cover kernel), into device memory
            n = (hi - lo) // 2
            pa = torch.zeros(n, dtype=torch.int32, device="cuda")
            pb = torch.zeros(n, dtype=torch.int32, device="cuda")
            ra = g.verify_range(lo, hi, pmin=pa, **kw)
            rb = g.verify_range_noalloc(lo, hi, pmin=pb, **kw)
            torch.cuda.synchronize()
            _same(rb, ra)
            assert torch.equal(pa, pb)


def test_noalloc_rejects_oversized_requests():
    from paper_2603_02621_gb300 import gb
    with gb.Context(device=0, base_limit=1 << 20, seg_len=1 << 24, p1=1 << 15, p2=1 << 20) as g:
        with pytest.raises(gb.GbError) as e:
            g.verify_range_noalloc(10**9, 10**9 + 2 * ((1 << 22) + 2))     # more than GB_NOALLOC_MAX_N
        assert e.value.code == gb.GB_ERANGE
        with pytest.raises(gb.GbError) as e:
            g.verify_range_noalloc(10**9, 10**9 + 200, pmin=np.zeros(100, dtype=np.uint32))   # host pmin
        assert e.value.code == gb.GB_EINVAL
