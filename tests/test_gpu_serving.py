"""Serving (gb_server_*): a Poisson request stream of range verifications and
single-n queries at offsets up to 4e18, served with continuous batching over
several lanes.  Each result must be identical served in the mix, served
alone, and computed by the plain entry points; a sample is checked against
the CPU oracle."""
import threading
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

P2 = 1 << 20


@pytest.fixture(scope="module")
def gbm():
    from paper_2603_02621_gb300 import gb
    gb.load()
    assert torch.cuda.is_available()
    return gb


@pytest.fixture(scope="module")
def sctx(gbm):
    # base primes to 2^31: every range below 4.6e18
    with gbm.Context(device=0, base_limit=1 << 31, p1=1 << 15, p2=P2) as g:
        yield g


def _requests(count, seed=7):
    from paper_2603_02621_gb300.workloads import serving_stream
    # the serving mix with shorter ranges (2^10..2^20 even n) to keep the test short
    return serving_stream(count=count, seed=seed, log2_min=10, log2_max=20)


def _serve(gbm, ctx, reqs, lanes, budget, max_batch, paced=False):
    out = [None] * len(reqs)
    with gbm.Server(ctx, lanes=lanes, hbm_budget=budget, max_batch=max_batch) as srv:
        tickets = []
        t0 = time.perf_counter()
        for t, kind, a, b in reqs:
            if paced:
                dt = t - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            tickets.append(srv.submit(kind, a, b))
        for i, tk in enumerate(tickets):
            out[i] = srv.wait(tk)
        stats = srv.stats()
    return out, stats


def test_serving_mix_equals_alone(gbm, sctx, oracle):
    reqs = _requests(160)
    mixed, st = _serve(gbm, sctx, reqs, lanes=3, budget=1 << 30, max_batch=24, paced=True)
    assert st["submitted"] == st["completed"] == len(reqs)
    alone, st1 = _serve(gbm, sctx, reqs, lanes=1, budget=1 << 30, max_batch=1)
    assert st1["batches"] == len(reqs)
    for (t, kind, a, b), m, s in zip(reqs, mixed, alone):
        assert m["status"] == 0 and s["status"] == 0
        if kind == "range":
            assert m["range"] == s["range"], (a, b)
            assert m["range"]["n_checked"] == (b - a) // 2 and m["range"]["unresolved"] == 0
        else:
            assert m["p_min"] == s["p_min"], a
    # the plain entry points, with the server closed
    ranges = [(a, b) for t, kind, a, b in reqs if kind == "range"]
    plain = sctx.verify_batch(ranges)["records"]
    got = [m["range"] for (t, kind, a, b), m in zip(reqs, mixed) if kind == "range"]
    assert got == plain
    qs = [(a, m["p_min"]) for (t, kind, a, b), m in zip(reqs, mixed) if kind == "query"]
    assert len(qs) > 0
    np.testing.assert_array_equal(sctx.query_batch([n for n, _ in qs]), [p for _, p in qs])
    # the oracle on every query and on the shortest ranges
    for n, p in qs:
        assert p == oracle.pmin_single(n, P2)
    short = sorted(ranges, key=lambda r: r[1] - r[0])[:6]
    for a, b in short:
        summ, _ = oracle.verify_segments(a, b, (b - a) // 2, P2, 8, threads=4)
        rec = next(m["range"] for (t, kind, x, y), m in zip(reqs, mixed) if (x, y) == (a, b))
        assert [rec["n_checked"], rec["unresolved"], rec["max_pmin"], rec["max_pmin_n"]] == [int(v) for v in summ[0]]


def test_serving_admission_by_memory(gbm, sctx):
    # ranges of 2^20 even n hold ~0.16 MB each: a 1 MB budget admits a few at a time
    reqs = [(0.0, "range", 10**15 + 2**22 * i, 10**15 + 2**22 * i + 2**21) for i in range(24)]
    budget = 1 << 20
    res, st = _serve(gbm, sctx, reqs, lanes=4, budget=budget, max_batch=64)
    assert st["in_flight_max_bytes"] <= budget
    assert st["batches"] >= 4
    assert all(r["status"] == 0 and r["range"]["unresolved"] == 0 for r in res)


def test_serving_rejects_bad_requests(gbm, sctx):
    with gbm.Server(sctx, lanes=1) as srv:
        with pytest.raises(RuntimeError):
            srv.submit("range", 11, 21)
        with pytest.raises(RuntimeError):
            srv.submit("query", 7)
        with pytest.raises(RuntimeError):
            srv.submit("range", 10**6, 10**6 + 2 * (2**32 + 1))
        with pytest.raises(RuntimeError):
            srv.wait(12345)
        t = srv.submit("query", 10**18)
        assert srv.wait(t)["p_min"] > 0


def test_serving_concurrent_submitters(gbm, sctx):
    reqs = _requests(90, seed=8)
    res = {}
    with gbm.Server(sctx, lanes=2, hbm_budget=1 << 30, max_batch=16) as srv:
        def client(part):
            for i in part:
                t, kind, a, b = reqs[i]
                res[i] = srv.wait(srv.submit(kind, a, b))
        th = [threading.Thread(target=client, args=(range(k, len(reqs), 3),)) for k in range(3)]
        for x in th:
            x.start()
        for x in th:
            x.join()
    assert len(res) == len(reqs) and all(r["status"] == 0 for r in res.values())


def test_serving_queries_do_not_wait_for_ranges(gbm, sctx, oracle):
    """Queries have a lane of their own: queued behind long ranges, they are
    still answered before those ranges finish."""
    with gbm.Server(sctx, lanes=1, hbm_budget=8 << 30, max_batch=64) as srv:
        big = [srv.submit("range", 10**15 + 2**34 * i, 10**15 + 2**34 * i + 2**33) for i in range(4)]
        qn = [10**18 + 2 * k for k in range(1, 33)]
        qt = [srv.submit("query", n) for n in qn]
        qr = [srv.wait(t) for t in qt]
        rr = [srv.wait(t) for t in big]
    assert all(r["status"] == 0 for r in qr + rr)
    assert all(r["range"]["unresolved"] == 0 for r in rr)
    assert max(r["t_done_us"] for r in qr) < max(r["t_done_us"] for r in rr)
    for n, r in zip(qn, qr):
        assert r["p_min"] == oracle.pmin_single(n, P2)


def test_shared_context_lifetime(gbm, oracle):
    """Contexts made by gb_init_shared use the parent's base primes; the
    primes stay valid until the last context holding them is destroyed,
    whichever order they are destroyed in."""
    lo, hi = 10**12, 10**12 + 2 * 20000
    summ, _ = oracle.verify_segments(lo, hi, 20000, P2, 8, threads=4)
    want = [int(v) for v in summ[0]]

    def check(g):
        r = g.verify_range(lo, hi)
        assert [r["n_checked"], r["unresolved"], r["max_pmin"], r["max_pmin_n"]] == want

    parent = gbm.Context(device=0, base_limit=1 << 21, p1=1 << 15, p2=P2)
    child = parent.share()
    check(child)
    child.close()
    check(parent)                      # the parent's primes survive the child
    child2 = parent.share(torch.cuda.Stream().cuda_stream)
    parent.close()
    check(child2)                      # and the child's survive the parent
    child2.close()
