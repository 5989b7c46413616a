"""Batched mode (gb_verify_batch): many ranges of uneven length and offset in
one pass, compared range by range with the CPU oracle and with the plain
gb_verify_range path.  Integer outputs, bit-exact."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

P1 = 1 << 15
P2 = 1 << 20


@pytest.fixture(scope="module")
def gbm():
    from paper_2603_02621_gb300 import gb
    gb.load()
    assert torch.cuda.is_available()
    return gb


@pytest.fixture(scope="module")
def ctx(gbm):
    # base primes to 2^31: windows up to 4.6e18
    with gbm.Context(device=0, base_limit=1 << 31, seg_len=1 << 20, p1=P1, p2=P2) as g:
        yield g


def _check_vs_oracle(oracle, ranges, out, stride):
    for i, (lo, hi) in enumerate(ranges):
        n = (hi - lo) // 2
        summ, hist = oracle.verify_segments(lo, hi, n, P2, stride)
        r = out["records"][i]
        assert (r["lo"], r["hi"], r["n_checked"]) == (lo, hi, n), (lo, hi)
        assert r["unresolved"] == int(summ[0, 1]), (lo, hi)
        assert (r["max_pmin"], r["max_pmin_n"]) == (int(summ[0, 2]), int(summ[0, 3])), (lo, hi)
        if stride:
            np.testing.assert_array_equal(out["hist"][i], hist[0], err_msg=f"{lo} {hi}")
            nz = np.nonzero(hist[0])[0]
            assert r["hist_len"] == (int(nz[-1]) + 1 if len(nz) else 0)


def _mixed_ranges():
    from paper_2603_02621_gb300.workloads import batched_ranges
    fixed = [
        (4, 6),                           # n = 4 alone (p_min 2)
        (4, 4 + 2 * 5003),                # from the start, ragged
        (6, 8),
        (10**6, 10**6 + 2),               # one n
        (10**9, 10**9 + 2 * 70001),       # several block-cover chunks
        (2 * 10**10, 2 * 10**10 + 2 * 7680 * 32),   # exactly one chunk of words
        (3 * 10**11 + 2, 3 * 10**11 + 2 + 2 * 300007),  # primes above a tile (bucket path)
    ]
    rnd = batched_ranges(count=40, seed=11, log2_min=3, log2_max=17, start_min=10**6, start_max=10**12)
    return fixed + rnd


def test_batch_vs_oracle(ctx, oracle):
    ranges = _mixed_ranges()
    stride = len(oracle.primes_upto(P1))
    out = ctx.verify_batch(ranges, hist_stride=stride)
    _check_vs_oracle(oracle, ranges, out, stride)


def test_batch_matches_verify_range(ctx):
    from paper_2603_02621_gb300.workloads import batched_ranges
    ranges = batched_ranges(count=24, seed=5, log2_min=10, log2_max=22, start_min=10**9, start_max=10**15)
    ranges += [(10**15, 10**15 + 2 * (1 << 22)), (4 * 10**18, 4 * 10**18 + 2 * 100003)]
    stride = 4096
    out = ctx.verify_batch(ranges, hist_stride=stride)
    for i, (lo, hi) in enumerate(ranges):
        ref = ctx.verify_range(lo, hi, hist_cap=stride)
        r = out["records"][i]
        for k in ("n_checked", "unresolved", "max_pmin", "max_pmin_n", "hist_len"):
            assert r[k] == ref[k], (lo, hi, k)
        np.testing.assert_array_equal(out["hist"][i], ref["hist"], err_msg=f"{lo} {hi}")


def test_batch_device_outputs(ctx, oracle):
    ranges = _mixed_ranges()[:20]
    stride = 512
    host = ctx.verify_batch(ranges, hist_stride=stride)
    res = torch.zeros((len(ranges), 48), dtype=torch.uint8, device="cuda")
    rows = torch.zeros((len(ranges), stride), dtype=torch.int64, device="cuda")
    ctx.verify_batch(ranges, hist_stride=stride, results=res, hist=rows)
    raw = res.cpu().numpy()
    u64 = raw[:, :40].copy().view(np.uint64)
    u32 = raw[:, 40:].copy().view(np.uint32)
    for i, r in enumerate(host["records"]):
        assert [int(x) for x in u64[i]] == [r["lo"], r["hi"], r["n_checked"], r["unresolved"], r["max_pmin_n"]]
        assert [int(x) for x in u32[i]] == [r["max_pmin"], r["hist_len"]]
    np.testing.assert_array_equal(rows.cpu().numpy().view(np.uint64), host["hist"])


def test_batch_small_P_redo(ctx, oracle):
    # P = 313 (64 odd primes): many n stay open after the batched pass and are
    # redone by the plain path with its retry bound
    ranges = [(10**11, 10**11 + 2 * 40001), (10**12 + 2, 10**12 + 2 + 2 * 20011), (10**6, 10**6 + 2 * 999)]
    out = ctx.verify_batch(ranges, 313, hist_stride=256)
    _check_vs_oracle(oracle, ranges, out, 256)
    for i, (lo, hi) in enumerate(ranges):
        ref = ctx.verify_range(lo, hi, 313, hist_cap=256)
        assert out["records"][i]["max_pmin"] == ref["max_pmin"]


def test_batch_rejects_bad_input(ctx, gbm):
    assert ctx.verify_batch([])["rc"] == gbm.GB_OK
    with pytest.raises(RuntimeError):
        ctx.verify_batch([(10**6 + 1, 10**6 + 11)])
    with pytest.raises(RuntimeError):
        ctx.verify_batch([(10**6, 10**6)])
    with pytest.raises(RuntimeError):
        ctx.verify_batch([(10**6, 10**6 + 100)], 17)     # fewer than 48 odd primes
    out = ctx.verify_batch([(10**9, 10**9 + 2 * 5000)], hist_stride=3, allow_erange=True)
    assert out["rc"] == gbm.GB_ERANGE and out["records"][0]["hist_len"] > 3


def test_batch_4096_ranges_sampled(ctx, oracle):
    """The 4096-range workload (lengths log-uniform 2^10..2^26 even n, starts
    uniform in [1e9, 1e15]): invariants on every range; 64 seeded ranges,
    drawn from the whole batch (so from the whole length span), recomputed by
    the oracle: records and p_min histogram rows element by element."""
    from paper_2603_02621_gb300.workloads import batched_ranges, sample_indices
    ranges = batched_ranges(count=4096, seed=1)
    stride = len(oracle.primes_upto(P1))
    out = ctx.verify_batch(ranges, hist_stride=stride)
    for (lo, hi), r in zip(ranges, out["records"]):
        assert (r["lo"], r["hi"], r["n_checked"], r["unresolved"]) == (lo, hi, (hi - lo) // 2, 0)
        assert lo <= r["max_pmin_n"] < hi
        assert oracle.mr_isprime(r["max_pmin"]) and oracle.mr_isprime(r["max_pmin_n"] - r["max_pmin"])
    np.testing.assert_array_equal(out["hist"].sum(axis=1, dtype=np.uint64),
                                  np.array([(hi - lo) // 2 for lo, hi in ranges], dtype=np.uint64))
    pick = sample_indices(len(ranges), 64, seed=3)
    lens = sorted((ranges[i][1] - ranges[i][0]) // 2 for i in pick)
    assert lens[0] < (1 << 12) and lens[-1] > (1 << 24)          # the sample spans the length range
    _check_vs_oracle(oracle, [ranges[i] for i in pick],
                     {"records": [out["records"][i] for i in pick], "hist": out["hist"][pick]}, stride)


def test_set_config_and_autotune(gbm):
    from paper_2603_02621_gb300.workloads import batched_ranges
    ranges = batched_ranges(count=64, seed=2, log2_min=10, log2_max=18, start_min=10**9, start_max=10**13)
    with gbm.Context(device=0, base_limit=1 << 26, seg_len=1 << 20, p1=P1, p2=P2) as g:
        before = g.verify_batch(ranges, hist_stride=512)
        plain_before = [g.verify_range(lo, hi, hist_cap=512) for lo, hi in ranges[:3]]
        with pytest.raises(RuntimeError):
            g.set_config(base_limit=1 << 20)
        with pytest.raises(RuntimeError):
            g.set_config(cover_prefix=100)
        cfg = g.set_config(tile_bits=1 << 16, bucket_split=1 << 15, cover_prefix=64, p1=1 << 12)
        assert (cfg["tile_bits"], cfg["bucket_split"], cfg["cover_prefix"], cfg["p1"]) == (1 << 16, 1 << 15, 64, 1 << 12)
        cfg, ms = g.autotune(ranges, gbm.GB_TUNE_BATCH, reps=1)
        assert ms > 0 and g.config() == cfg
        after = g.verify_batch(ranges, hist_stride=512)
        assert after["records"] == before["records"]
        np.testing.assert_array_equal(after["hist"], before["hist"])
        cfg, ms = g.autotune(ranges[:3], gbm.GB_TUNE_PLAIN, reps=1)
        assert ms > 0
        for (lo, hi), ref in zip(ranges[:3], plain_before):
            got = g.verify_range(lo, hi, hist_cap=512)
            for k in ("n_checked", "unresolved", "max_pmin", "max_pmin_n", "hist_len"):
                assert got[k] == ref[k]
            np.testing.assert_array_equal(got["hist"], ref["hist"])


def test_batch_graph_and_plain_launches_agree(gbm, monkeypatch):
    """The batch kernels captured as a CUDA graph (default) and launched one
    by one (GB_BATCH_GRAPH=0) give the same outputs; repeated calls re-use
    the graph by update."""
    from paper_2603_02621_gb300.workloads import batched_ranges
    ranges = batched_ranges(count=200, seed=9, log2_min=4, log2_max=19, start_min=10**9, start_max=10**14)
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("GB_BATCH_GRAPH", flag)
        with gbm.Context(device=0, base_limit=1 << 24, seg_len=1 << 20, p1=P1, p2=P2) as g:
            a = g.verify_batch(ranges, hist_stride=600)
            b = g.verify_batch(ranges[::-1], hist_stride=600)
            c = g.verify_batch(ranges, hist_stride=600)
            assert a["records"] == c["records"] and a["records"] == b["records"][::-1]
            np.testing.assert_array_equal(a["hist"], c["hist"])
            np.testing.assert_array_equal(a["hist"], b["hist"][::-1])
            outs.append(a)
    assert outs[0]["records"] == outs[1]["records"]
    np.testing.assert_array_equal(outs[0]["hist"], outs[1]["hist"])


def test_autotune_cache_hit(gbm, monkeypatch, tmp_path):
    """With GB_TUNE_CACHE set, a second autotune of the same sample on the
    same GPU applies the stored setting without timing anything."""
    import time
    from paper_2603_02621_gb300.workloads import batched_ranges
    ranges = batched_ranges(count=32, seed=4, log2_min=10, log2_max=16, start_min=10**9, start_max=10**12)
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("GB_TUNE_CACHE", str(path))
    with gbm.Context(device=0, base_limit=1 << 20, seg_len=1 << 20, p1=P1, p2=P2) as g:
        before = g.verify_batch(ranges, hist_stride=512)
        cfg1, ms1 = g.autotune(ranges, gbm.GB_TUNE_BATCH, reps=1)
        t0 = time.perf_counter()
        cfg2, ms2 = g.autotune(ranges, gbm.GB_TUNE_BATCH, reps=1)
        assert time.perf_counter() - t0 < 0.5
        assert cfg2 == cfg1 and ms2 == pytest.approx(ms1, rel=1e-6)
        after = g.verify_batch(ranges, hist_stride=512)
        assert after["records"] == before["records"]
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith(torch.cuda.get_device_name(0) + "|")
