"""Exhaustive verification at scale (uint64 n): [4, 10^12] (the range of the
paper's Table 4) and the 10^11-wide window below 4e18, segments of 2^27 even
n, base primes to 2^31, P1 = 2^15 then the retry pass to P2 = 2^20.

Every segment's record and histogram row is checked against invariants and
the merged totals; a seeded sample of 256 segments per range
(GB_SAMPLED_SEGMENTS to change it) is recomputed by the CPU oracle and must
match bit for bit."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

S = 1 << 27
P1, P2 = 1 << 15, 1 << 20
HL = 3512                      # pi(2^15)
SAMPLES = int(os.environ.get("GB_SAMPLED_SEGMENTS", "256"))


@pytest.fixture(scope="module")
def gbm():
    from paper_2603_02621_gb300 import gb
    gb.load()
    assert torch.cuda.is_available()
    return gb


@pytest.fixture(scope="module")
def ctx31(gbm):
    with gbm.Context(device=0, base_limit=1 << 31, seg_len=S, p1=P1, p2=P2) as g:
        yield g


def _run_and_check(ctx, oracle, lo, hi, seed):
    out = ctx.verify_range(lo, hi, hist_cap=HL, segs=True, seg_hist_stride=HL)
    n = (hi - lo) // 2
    nseg = (n + S - 1) // S
    segs, rows = out["segs"], out["seg_hist"]
    assert out["n_checked"] == n and out["n_segments"] == nseg and len(segs) == nseg
    assert out["unresolved"] == 0
    # per-segment invariants and the merge
    assert sum(s["n_checked"] for s in segs) == n
    np.testing.assert_array_equal(rows.sum(axis=0, dtype=np.uint64), out["hist"])
    assert int(out["hist"].sum()) == n
    best = max(segs, key=lambda s: (s["max_pmin"], -s["max_pmin_n"]))
    assert (out["max_pmin"], out["max_pmin_n"]) == (best["max_pmin"], best["max_pmin_n"])
    for k, s in enumerate(segs):
        assert s["lo"] == lo + 2 * k * S and s["hi"] == min(lo + 2 * (k + 1) * S, hi)
        assert int(rows[k].sum()) == s["n_checked"] and s["unresolved"] == 0
    p, m = out["max_pmin"], out["max_pmin_n"]
    assert oracle.mr_isprime(p) and oracle.mr_isprime(m - p) and oracle.pmin_single(m, P2) == p

    # seeded sample of segments, each recomputed by the oracle in one thread
    from paper_2603_02621_gb300.workloads import sample_indices
    pick = sample_indices(nseg, SAMPLES, seed=seed)
    oracle.verify_segments(hi - 4, hi, 2, P2, 8, threads=1)    # build the oracle's prime cache once

    def one(k):
        a, b = segs[k]["lo"], segs[k]["hi"]
        summ, hist = oracle.verify_segments(a, b, S, P2, HL, threads=1)
        return k, summ[0], hist[0]

    with cf.ThreadPoolExecutor(max_workers=oracle.default_threads()) as ex:
        for k, summ, hist in ex.map(one, pick):
            s = segs[k]
            assert [s["n_checked"], s["unresolved"], s["max_pmin"], s["max_pmin_n"]] == [int(x) for x in summ], k
            np.testing.assert_array_equal(rows[k], hist, err_msg=f"segment {k}")
    return out


def test_exhaustive_4_to_1e12(ctx31, oracle):
    out = _run_and_check(ctx31, oracle, 4, 10**12 + 2, seed=12)
    assert out["n_checked"] == 10**12 // 2 - 1          # N/2 - 1 even n in [4, N]


def test_window_below_4e18(ctx31, oracle):
    lo, hi = 4 * 10**18 - 10**11, 4 * 10**18
    out = _run_and_check(ctx31, oracle, lo, hi, seed=18)
    assert out["n_checked"] == 10**11 // 2
