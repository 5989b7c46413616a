"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

All outputs are integers and must match bit for bit: sieve bitsets, p_min
arrays, per-segment histograms, maxima with their n, unresolved counts.
"""
import numpy as np
import pytest

from conftest import read_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _unpack(words_tensor, nbits):
    b = np.unpackbits(words_tensor.cpu().numpy().view(np.uint8), bitorder="little")
    return b[:nbits], b[nbits:]


@pytest.fixture(scope="module")
def gbm():
    from paper_2603_02621_gb300 import gb
    gb.load()
    assert torch.cuda.is_available()
    return gb


@pytest.fixture(scope="module")
def ctx16(gbm):
    with gbm.Context(device=0, base_limit=1 << 16, seg_len=1 << 16, p1=1 << 15, p2=1 << 20) as g:
        yield g


@pytest.fixture(scope="module")
def ctx_big(gbm):
    # base primes to 2^31: covers windows up to 4.6e18
    with gbm.Context(device=0, base_limit=1 << 31, seg_len=1 << 20, p1=1 << 15, p2=1 << 20) as g:
        yield g


def hist_len_for(oracle, P):
    return len(oracle.primes_upto(P))


_ORACLE_SEGMENTS = {}


def oracle_segments(oracle, lo, hi, S, P, HL):
    """The oracle's per-segment records and histograms of [lo, hi), computed
    once per module run and shared by the tests that compare with them."""
    key = (lo, hi, S, P, HL)
    if key not in _ORACLE_SEGMENTS:
        _ORACLE_SEGMENTS[key] = oracle.verify_segments(lo, hi, S, P, HL, threads=oracle.default_threads())
    return _ORACLE_SEGMENTS[key]


def assert_segments_equal_oracle(r, summ, hist):
    rec = [[s["n_checked"], s["unresolved"], s["max_pmin"], s["max_pmin_n"]] for s in r["segs"]]
    assert rec == summ.tolist()
    np.testing.assert_array_equal(r["seg_hist"], hist)


# ------------------------------------------------------------------ sieve

@pytest.mark.parametrize("A,nbits", [
    (1, 5 * 10**6 + 37),                 # base range, several tiles, ragged tail
    (-(1 << 20) + 1, (1 << 20) + 777),   # window reaching below 0 (first-segment halo)
    (-5, 100),                           # tiny, straddles 1 and the wheel primes
    (10**9 + 1, 3 * (1 << 18) + 101),
    (10**12 - 999, (1 << 19) + 5),
    (2**40 + 1, (1 << 18) + 64),
])
def test_sieve_segment_vs_oracle(ctx16, oracle, A, nbits):
    words = (nbits + 63) // 64
    q = torch.full((words,), -1, dtype=torch.int64, device="cuda")
    pc = ctx16.sieve_segment(A, nbits, q)
    bits, tail = _unpack(q, nbits)
    ref = oracle.odd_bits(A, nbits)
    assert np.array_equal(bits, ref)
    assert not tail.any()                 # bits past n_bits are zero
    assert pc == int(ref.sum())


@pytest.mark.parametrize("A,nbits", [
    (10**15 + 1, (1 << 18) + 63),
    (4 * 10**18 - 10**11 + 1, (1 << 18) + 1),
])
def test_sieve_segment_high_offsets(ctx_big, oracle, A, nbits):
    words = (nbits + 63) // 64
    q = torch.zeros(words, dtype=torch.int64, device="cuda")
    pc = ctx_big.sieve_segment(A, nbits, q)
    bits, _ = _unpack(q, nbits)
    ref = oracle.odd_bits(A, nbits)
    assert np.array_equal(bits, ref)
    assert pc == int(ref.sum())


def test_sieve_rejects_even_base(ctx16, gbm):
    q = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(gbm.GbError) as e:
        ctx16.sieve_segment(10, 64, q)
    assert e.value.code == gbm.GB_EINVAL


def test_sieve_rejects_beyond_base_limit(ctx16, gbm):
    q = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(gbm.GbError):
        ctx16.sieve_segment(2**41 + 1, 64, q)      # sqrt beyond the 2^20 prime list


@pytest.mark.parametrize("x,pi", [(int(a), int(b)) for a, b in read_golden("prime_counts.txt")])
def test_prime_pi(gbm, x, pi):
    with gbm.Context(device=0, base_limit=1 << 17) as g:
        assert g.prime_pi(x) == pi


# ------------------------------------------------------------------ cover

def test_pmin_array_4_to_1e7(gbm, oracle):
    """Every even n in [4, 10^7], one segment, P = 2^16: the full p_min array."""
    lo, hi, P = 4, 10**7 + 2, 1 << 16
    S = ((5 * 10**6 + 2047) // 2048) * 2048
    with gbm.Context(device=0, base_limit=1 << 16, seg_len=S, p1=P) as g:
        pm = np.zeros((hi - lo) // 2, dtype=np.uint32)
        H = hist_len_for(oracle, P)
        r = g.verify_range(lo, hi, pmin=pm, hist_cap=H, segs=True)
        assert g.prime_pi(10**7) == 664579
    ref = oracle.pmin_range(lo, hi, P)
    assert r["n_checked"] == 4999999 and r["n_segments"] == 1
    assert np.array_equal(pm, ref)
    summ, hist = oracle.verify_segments(lo, hi, S, P, H)
    assert r["unresolved"] == int(summ[0, 1]) == 0
    assert (r["max_pmin"], r["max_pmin_n"]) == (int(summ[0, 2]), int(summ[0, 3]))
    assert np.array_equal(r["hist"], hist[0])


def test_exhaustive_4_to_1e10_full(gbm, oracle):
    """Exhaustive [4, 10^10]: segments of 2^24, base primes to 10^5, P1 = 2^15
    with a GPU retry pass to 2^20; per-segment histogram, max, unresolved."""
    lo, hi = 4, 10**10 + 2
    S, P1, P2 = 1 << 24, 1 << 15, 1 << 20
    H = hist_len_for(oracle, P1)
    with gbm.Context(device=0, base_limit=10**5, seg_len=S, p1=P1, p2=P2) as g:
        r = g.verify_range(lo, hi, seg_hist_stride=H, hist_cap=H)
    assert r["n_checked"] == 4999999999 and r["p_final"] == P2
    summ, hist = oracle.verify_segments(lo, hi, S, P2, H)
    assert r["n_segments"] == summ.shape[0] == 299
    got = np.array([[s["n_checked"], s["unresolved"], s["max_pmin"], s["max_pmin_n"]]
                    for s in r["segs"]], dtype=np.uint64)
    assert np.array_equal(got, summ)
    assert np.array_equal(r["seg_hist"], hist)
    assert np.array_equal(r["hist"], hist.sum(axis=0))
    assert r["unresolved"] == 0
    k = int(np.argmax(summ[:, 2]))
    assert (r["max_pmin"], r["max_pmin_n"]) == (int(summ[k, 2]), int(summ[k, 3]))


@pytest.mark.parametrize("lo,hi", [
    (4, 6), (6, 8), (4, 130), (4, 4098), (10**9 + 2, 10**9 + 4),
    (10**9 + 2, 10**9 + 2 + 2 * 4095), (2**40, 2**40 + 2 * 3001),
    (4, 2 * (1 << 16) * 3 + 4 + 2 * 77),   # three full segments of 2^16 + ragged
])
def test_edge_ranges(ctx16, oracle, lo, hi):
    P2 = 1 << 20
    H = hist_len_for(oracle, 1 << 15)
    pm = np.zeros((hi - lo) // 2, dtype=np.uint32)
    r = ctx16.verify_range(lo, hi, pmin=pm, seg_hist_stride=H, hist_cap=H)
    assert np.array_equal(pm, oracle.pmin_range(lo, hi, P2))
    summ, hist = oracle.verify_segments(lo, hi, 1 << 16, P2, H)
    got = np.array([[s["n_checked"], s["unresolved"], s["max_pmin"], s["max_pmin_n"]]
                    for s in r["segs"]], dtype=np.uint64)
    assert np.array_equal(got, summ)
    assert np.array_equal(r["seg_hist"], hist)


@pytest.mark.parametrize("lo,hi", [
    (4, 6), (6, 8), (4, 130), (4, 4098), (10**9 + 2, 10**9 + 4),
    (10**9 + 2, 10**9 + 2 + 2 * 4095), (2**40, 2**40 + 2 * 3001),
    (4, 2 * (1 << 16) * 3 + 4 + 2 * 77),
    (10**12 + 10, 10**12 + 10 + 2 * 300007),
])
def test_edge_ranges_two_phase(ctx16, oracle, lo, hi):
    """Without a p_min array the two-phase cover kernel runs; same outputs."""
    P2 = 1 << 20
    H = hist_len_for(oracle, 1 << 15)
    r = ctx16.verify_range(lo, hi, seg_hist_stride=H, hist_cap=H)
    summ, hist = oracle.verify_segments(lo, hi, 1 << 16, P2, H)
    got = np.array([[s["n_checked"], s["unresolved"], s["max_pmin"], s["max_pmin_n"]]
                    for s in r["segs"]], dtype=np.uint64)
    assert np.array_equal(got, summ)
    assert np.array_equal(r["seg_hist"], hist)
    assert np.array_equal(r["hist"], hist.sum(axis=0))


def test_two_phase_into_retry(gbm, oracle):
    """P1 = 2^8 (53 odd primes: first phase of 32, second phase to 256), retry
    to 2^16: n with p_min > 256 travel through all three stages."""
    lo, hi = 10**9, 10**9 + 2 * 2 * 10**6
    H = hist_len_for(oracle, 1 << 16)
    with gbm.Context(device=0, base_limit=1 << 16, seg_len=1 << 18, p1=1 << 8, p2=1 << 16) as g:
        r = g.verify_range(lo, hi, seg_hist_stride=H, hist_cap=H)
    summ, hist = oracle.verify_segments(lo, hi, 1 << 18, 1 << 16, H)
    assert hist[:, 55:].sum() > 0                       # some p_min above 2^8 exist
    got = np.array([[s["n_checked"], s["unresolved"], s["max_pmin"], s["max_pmin_n"]]
                    for s in r["segs"]], dtype=np.uint64)
    assert np.array_equal(got, summ)
    assert np.array_equal(r["seg_hist"], hist)


def test_two_phase_without_retry_counts_unresolved(gbm, oracle):
    lo, hi = 10**9, 10**9 + 2 * 10**6
    with gbm.Context(device=0, base_limit=1 << 16, seg_len=1 << 18, p1=1 << 8) as g:
        r = g.verify_range(lo, hi, segs=True)
    ref = oracle.pmin_range(lo, hi, 1 << 8)
    assert r["unresolved"] == int((ref == 0).sum()) > 0
    assert r["max_pmin"] == int(ref.max())


@pytest.mark.parametrize("ka", ["48", "64", "80", "144", "192", "256"])
@pytest.mark.parametrize("lo", [10**6, 3 * 10**11, 4 * 10**18 - 10**7])
def test_two_phase_matches_generic(gbm, oracle, monkeypatch, ka, lo):
    """The block cover (a first block of 48 or 64 primes and 0 to 6 blocks of
    32, so the segment maximum comes from the probing or from a re-run of the
    last block that set a bit, with its input list kept or overwritten), the
    generic cover kernel and the oracle give identical per-segment records
    and histograms."""
    hi = lo + 2 * 5 * 10**6
    base = dict(device=0, base_limit=1 << 31, seg_len=1 << 20, p1=1 << 15, p2=1 << 20)
    monkeypatch.setenv("GB_KA", ka)
    with gbm.Context(**base) as g:
        a = g.verify_range(lo, hi, seg_hist_stride=3512, hist_cap=3512)
    monkeypatch.delenv("GB_KA")
    monkeypatch.setenv("GB_COVER", "generic")
    with gbm.Context(**base) as g:
        b = g.verify_range(lo, hi, seg_hist_stride=3512, hist_cap=3512)
    assert a["segs"] == b["segs"]
    assert np.array_equal(a["seg_hist"], b["seg_hist"])
    summ, hist = oracle_segments(oracle, lo, hi, 1 << 20, 1 << 20, 3512)
    assert_segments_equal_oracle(a, summ, hist)


@pytest.mark.parametrize("p2", [0, 1 << 20])
def test_block_cover_48_schedule_chosen_by_magnitude(gbm, oracle, monkeypatch, p2):
    """P1 = 293 holds 61 odd primes: near 1e12 the block cover is chosen
    without an override and takes its 48-prime schedule (K in [48, 63]);
    identical to the generic cover and to the oracle, with and without the
    retry pass."""
    monkeypatch.delenv("GB_KA", raising=False)
    monkeypatch.delenv("GB_COVER", raising=False)
    lo, hi = 10**12, 10**12 + 2 * 3 * 10**6
    HL = 62                                        # primes <= 293
    stride = HL if p2 == 0 else hist_len_for(oracle, p2)
    base = dict(device=0, base_limit=1 << 20, seg_len=1 << 20, p1=293, p2=p2)
    with gbm.Context(**base) as g:
        a = g.verify_range(lo, hi, seg_hist_stride=stride, hist_cap=stride)
    monkeypatch.setenv("GB_COVER", "generic")
    with gbm.Context(**base) as g:
        b = g.verify_range(lo, hi, seg_hist_stride=stride, hist_cap=stride)
    assert a["segs"] == b["segs"]
    assert np.array_equal(a["seg_hist"], b["seg_hist"])
    summ, hist = oracle.verify_segments(lo, hi, 1 << 20, p2 or 293, stride, threads=oracle.default_threads())
    assert_segments_equal_oracle(a, summ, hist)
    if p2 == 0:
        assert a["unresolved"] > 0
    else:
        assert a["unresolved"] == 0


@pytest.mark.parametrize("p1,ka", [(420, "80"), (227, "48"), (313, "64"), (617, "112")])
def test_block_cover_maximum_without_probing(gbm, monkeypatch, p1, ka):
    """P1 holds exactly as many odd primes as the blocks (K = KA: 80 up to
    420, 48 up to 227, 64 up to 313, 112 up to 617), so no n is settled by
    probing and every
    warp takes its maximum from a re-run: near 4e18 block 0 leaves most words
    open, so the later block writes over its input and the re-run goes
    through every block; without a retry pass the open n count as
    unresolved.  Identical to the generic cover."""
    lo, hi = 4 * 10**18 - 2 * 3 * 10**6, 4 * 10**18
    base = dict(device=0, base_limit=1 << 31, seg_len=1 << 20, p1=p1, p2=0)
    monkeypatch.setenv("GB_KA", ka)
    with gbm.Context(**base) as g:
        a = g.verify_range(lo, hi, seg_hist_stride=128, hist_cap=128)
    monkeypatch.delenv("GB_KA")
    monkeypatch.setenv("GB_COVER", "generic")
    with gbm.Context(**base) as g:
        b = g.verify_range(lo, hi, seg_hist_stride=128, hist_cap=128)
    assert a["unresolved"] > 0
    assert a["segs"] == b["segs"]
    assert np.array_equal(a["seg_hist"], b["seg_hist"])


def test_n4_histogram_entry(ctx16):
    r = ctx16.verify_range(4, 6, hist_cap=4)
    assert r["max_pmin"] == 2 and r["max_pmin_n"] == 4
    assert r["hist"].tolist() == [1, 0, 0, 0]


def test_retry_pass_matches_single_pass(gbm, oracle):
    """Force almost every n into the retry pass (P1 = 31): the two-pass result
    equals a single pass to P2 and the oracle."""
    lo, hi = 4, 2 * 10**6 + 2
    H = hist_len_for(oracle, 1 << 16)
    with gbm.Context(device=0, base_limit=1 << 16, seg_len=1 << 18, p1=31, p2=1 << 16) as g:
        pa = np.zeros((hi - lo) // 2, dtype=np.uint32)
        ra = g.verify_range(lo, hi, pmin=pa, seg_hist_stride=H, hist_cap=H)
    with gbm.Context(device=0, base_limit=1 << 16, seg_len=1 << 18, p1=1 << 16) as g:
        pb = np.zeros((hi - lo) // 2, dtype=np.uint32)
        rb = g.verify_range(lo, hi, pmin=pb, seg_hist_stride=H, hist_cap=H)
    assert np.array_equal(pa, pb)
    assert np.array_equal(pa, oracle.pmin_range(lo, hi, 1 << 16))
    assert np.array_equal(ra["seg_hist"], rb["seg_hist"])
    assert ra["segs"] == rb["segs"]


def test_unresolved_counted_when_P_small(gbm, oracle):
    """With P1 = 7 and no retry, every n whose p_min exceeds 7 is unresolved."""
    lo, hi = 4, 20002
    with gbm.Context(device=0, base_limit=1 << 16, seg_len=2048, p1=7) as g:
        pm = np.zeros((hi - lo) // 2, dtype=np.uint32)
        r = g.verify_range(lo, hi, pmin=pm, segs=True)
    ref = oracle.pmin_range(lo, hi, 7)
    assert np.array_equal(pm, ref)
    assert r["unresolved"] == int((ref == 0).sum()) > 0


def test_pmin_device_buffer(ctx16, oracle):
    lo, hi = 10**9, 10**9 + 2 * 300001
    pm = torch.zeros((hi - lo) // 2, dtype=torch.int32, device="cuda")
    ctx16.verify_range(lo, hi, pmin=pm)
    torch.cuda.synchronize()
    assert np.array_equal(pm.cpu().numpy().view(np.uint32), oracle.pmin_range(lo, hi, 1 << 20))


@pytest.mark.parametrize("cfg", [
    dict(tile_bits=1 << 16, cta_threads=128),
    dict(tile_bits=1 << 20, cta_threads=512),
    dict(seg_len=1 << 12, slab_bits=1 << 14),        # many slabs
    dict(seg_len=1 << 22),
])
def test_tuning_invariance(gbm, cfg):
    """Merged outputs do not depend on tile, CTA, segment or slab sizes."""
    lo, hi = 10**11, 10**11 + 2 * 3 * 10**6
    base = dict(device=0, base_limit=1 << 19, seg_len=1 << 16, p1=1 << 15, p2=1 << 20)
    with gbm.Context(**base) as g:
        a = g.verify_range(lo, hi, hist_cap=3600)
    with gbm.Context(**{**base, **cfg}) as g:
        b = g.verify_range(lo, hi, hist_cap=3600)
    for key in ("n_checked", "unresolved", "max_pmin", "max_pmin_n", "hist_len"):
        assert a[key] == b[key], key
    assert np.array_equal(a["hist"], b["hist"])


def test_high_offset_window_sampled(ctx_big, oracle):
    """Segments of the window [4e18 - 1e11, 4e18) at seeded positions."""
    from paper_2603_02621_gb300 import workloads
    lo0, S = 4 * 10**18 - 10**11, 1 << 20
    nseg = (10**11 // 2 + S - 1) // S
    H = hist_len_for(oracle, 1 << 15)
    for k in workloads.sample_indices(nseg, 4, seed=3):
        lo = lo0 + 2 * k * S
        hi = min(lo + 2 * S, 4 * 10**18)
        r = ctx_big.verify_range(lo, hi, seg_hist_stride=H)
        summ, hist = oracle.verify_segments(lo, hi, S, 1 << 20, H)
        s = r["segs"][0]
        assert [s["n_checked"], s["unresolved"], s["max_pmin"], s["max_pmin_n"]] == summ[0].tolist()
        assert np.array_equal(r["seg_hist"], hist)


def test_invalid_ranges(ctx16, gbm):
    for lo, hi in [(3, 10), (4, 9), (10, 10), (12, 10), (2, 10)]:
        with pytest.raises(gbm.GbError) as e:
            ctx16.verify_range(lo, hi)
        assert e.value.code == gbm.GB_EINVAL
    with pytest.raises(gbm.GbError):
        ctx16.verify_range(2**41, 2**41 + 10)     # sqrt beyond the 2^20 prime list


def test_ranges_next_to_the_upper_limit(gbm, oracle):
    """The last ranges the API takes (hi up to 2^63 - 2^26): records against
    the oracle; one past the limit is refused."""
    with gbm.Context(device=0, base_limit=1 << 32, seg_len=1 << 20, p1=1 << 15, p2=1 << 20) as g:
        hi = gbm.GB_MAX_HI
        lo = hi - 2 * 20000
        r = g.verify_range(lo, hi)
        # the oracle's Miller-Rabin p_min of every n (no window sieve to 3e9 needed)
        pm = [oracle.pmin_single(n, 1 << 20) for n in range(lo, hi, 2)]
        best = max(pm)
        assert min(pm) > 0
        assert [r["n_checked"], r["unresolved"], r["max_pmin"], r["max_pmin_n"]] == \
            [len(pm), 0, best, lo + 2 * pm.index(best)]
        b = g.verify_batch([(lo, hi)])["records"][0]
        assert [b["max_pmin"], b["max_pmin_n"], b["unresolved"]] == [r["max_pmin"], r["max_pmin_n"], 0]
        with pytest.raises(RuntimeError):
            g.verify_range(hi, hi + 2)
        with pytest.raises(RuntimeError):
            g.verify_batch([(hi, hi + 2)])


def test_retry_list_overflow_is_redone(gbm):
    """P1 = 31 leaves nearly every 64-n word of a 2^28-n slab open, more than
    the retry list holds (2^21 words): the call is redone as one pass to P2
    and must give the same totals as the ordinary P1 = 2^15 run."""
    with gbm.Context(device=0, base_limit=1 << 20, seg_len=1 << 24, p1=1 << 15, p2=1 << 20) as g:
        lo, hi = 10**9, 10**9 + 2 * (1 << 28)
        ref = g.verify_range(lo, hi, hist_cap=4096)
        got = g.verify_range(lo, hi, 31, hist_cap=4096)
    for k in ("n_checked", "unresolved", "max_pmin", "max_pmin_n", "hist_len"):
        assert got[k] == ref[k], k
    np.testing.assert_array_equal(got["hist"], ref["hist"])
    assert got["p_final"] == 1 << 20 and ref["unresolved"] == 0


def test_histogram_capacity_too_small(ctx16, gbm, oracle):
    lo, hi = 10**9, 10**9 + 2 * 40000
    full = ctx16.verify_range(lo, hi, hist_cap=1024)
    short = ctx16.verify_range(lo, hi, hist_cap=5, allow_erange=True)
    assert short["rc"] == gbm.GB_ERANGE and full["rc"] == gbm.GB_OK
    np.testing.assert_array_equal(short["hist"], full["hist"][:5])
    assert short["max_pmin"] == full["max_pmin"] and short["hist_len"] == full["hist_len"] > 5
