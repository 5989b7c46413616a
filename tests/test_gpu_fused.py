"""Sieve and cover fused per CTA (GB_FUSED=1): Q stays in shared memory.
Every per-segment output must equal the unfused path's and the oracle's."""
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


def _run(gbm, monkeypatch, fused, lo, hi, P=0, **cfg):
    monkeypatch.setenv("GB_FUSED", "1" if fused else "0")
    base = dict(device=0, base_limit=1 << 20, seg_len=1 << 24, p1=1 << 15, p2=1 << 20)
    base.update(cfg)
    with gbm.Context(**base) as g:
        S = g.config()["seg_len"]
        nseg = ((hi - lo) // 2 + S - 1) // S
        return g.verify_range(lo, hi, P, hist_cap=4096, segs=True, seg_hist_stride=4096)


def _same(a, b):
    for k in ("n_checked", "unresolved", "max_pmin", "max_pmin_n", "hist_len"):
        assert a[k] == b[k], k
    assert a["segs"] == b["segs"]
    np.testing.assert_array_equal(a["seg_hist"], b["seg_hist"])
    np.testing.assert_array_equal(a["hist"], b["hist"])


@pytest.mark.parametrize("lo,hi,P,cfg", [
    (4, 2**31 + 2, 0, {}),                                   # 128 segments from n = 4
    (10**10, 10**10 + 2 * (3 * 2**24 + 12345), 0, {}),       # ragged last segment
    (10**9, 10**9 + 2 * 10**6, 0, dict(seg_len=1 << 18)),   # chunks cut by segment ends
    (10**11, 10**11 + 2 * 2**20, 313, {}),                  # small P1: the retry pass sieves to HBM
    (10**13, 10**13 + 2 * 2**20, 0, dict(base_limit=1 << 22)),  # primes above the split: unfused fallback
])
def test_fused_equals_unfused(gbm, monkeypatch, lo, hi, P, cfg):
    _same(_run(gbm, monkeypatch, True, lo, hi, P, **cfg), _run(gbm, monkeypatch, False, lo, hi, P, **cfg))


def test_fused_vs_oracle(gbm, monkeypatch, oracle):
    lo, hi, S = 4, 4 + 2 * (2 * 2**20 + 777), 1 << 20
    got = _run(gbm, monkeypatch, True, lo, hi, seg_len=S)
    summ, hist = oracle.verify_segments(lo, hi, S, 1 << 20, 4096)
    for k, s in enumerate(got["segs"]):
        assert [s["n_checked"], s["unresolved"], s["max_pmin"], s["max_pmin_n"]] == [int(v) for v in summ[k]]
    np.testing.assert_array_equal(got["seg_hist"], hist)
