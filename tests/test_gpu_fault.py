"""Error paths under host-side fault injection on the GPU machine: an allocation
the library is told has failed returns GB_ENOMEM and leaves the context
usable; the server refuses a submit at admission and cancels queued requests.
Every fault is made on the host; no kernel faults, traps or hangs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture()
def gbm():
    from paper_2603_02621_gb300 import gb
    gb.load()
    assert torch.cuda.is_available()
    yield gb
    gb.gb_fault_set(None)


def test_injected_allocation_failure_returns_enomem(gbm, oracle):
    lo, hi = 10**9, 10**9 + 2 * 200001
    with gbm.Context(device=0, base_limit=1 << 16, seg_len=1 << 18, p1=1 << 15, p2=1 << 20) as g:
        before = gbm.gb_alloc_stats()
        gbm.gb_fault_set("alloc@1")
        with pytest.raises(gbm.GbError) as e:
            g.verify_range(lo, hi, hist_cap=4096)          # the first call sizes the context's arenas
        assert e.value.code == gbm.GB_ENOMEM and "injected" in str(e.value)
        assert gbm.gb_alloc_stats()["count"] == before["count"]
        gbm.gb_fault_set(None)
        r = g.verify_range(lo, hi, hist_cap=4096)          # the same context, usable
        summ, hist = oracle.verify_segments(lo, hi, (hi - lo) // 2, 1 << 20, 4096)
        assert [r["n_checked"], r["unresolved"], r["max_pmin"], r["max_pmin_n"]] == summ[0].tolist()
        np.testing.assert_array_equal(r["hist"], hist[0])


def test_server_refuses_and_cancels(gbm):
    with gbm.Context(device=0, base_limit=1 << 26, p1=1 << 15, p2=1 << 20) as g:
        alone = g.verify_batch([(10**12, 10**12 + 2 * 4099)])["records"][0]
        with gbm.Server(g, lanes=1) as srv:
            gbm.gb_fault_set("submit@2,cancel@2")   # the refused submit counts no cancel event
            t1 = srv.submit("range", 10**12, 10**12 + 2 * 4099)
            with pytest.raises(gbm.GbError) as e:
                srv.submit("range", 10**12, 10**12 + 2 * 4099)      # refused at admission
            assert e.value.code == gbm.GB_EBUSY
            t3 = srv.submit("range", 10**12, 10**12 + 2 * 4099)     # queued, then cancelled
            gbm.gb_fault_set(None)
            r1, r3 = srv.wait(t1), srv.wait(t3)
            assert r1["status"] == gbm.GB_OK and r1["range"]["max_pmin"] == alone["max_pmin"]
            assert r3["status"] == gbm.GB_ECANCELED and r3["range"]["lo"] == 10**12
            # an explicit cancel of a request queued behind a long one on the single lane
            big = srv.submit("range", 10**15, 10**15 + 2 * (1 << 30))
            small = srv.submit("range", 10**12, 10**12 + 2 * 4099)
            assert srv.cancel(small) == gbm.GB_OK
            assert srv.wait(small)["status"] == gbm.GB_ECANCELED
            rb = srv.wait(big)
            assert rb["status"] == gbm.GB_OK and rb["range"]["unresolved"] == 0
            assert srv.cancel(big) == gbm.GB_EBUSY                   # finished: too late
            with pytest.raises(gbm.GbError):
                srv.cancel(10**9)                                     # never issued
