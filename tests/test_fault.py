"""Host-side fault injection (GB_FAULT, gb_fault_set): the spec parser and
the event counting the library checks at each allocation and submit.  No GPU:
the library loads and these calls touch no device."""
import pytest


@pytest.fixture(scope="module")
def gbm():
    from paper_2603_02621_gb300 import gb
    gb.load()
    yield gb
    gb.gb_fault_set(None)


def test_fault_spec_parsing(gbm):
    for good in ("alloc@1", "submit@3,cancel@2", "alloc@7,", "", None):
        gbm.gb_fault_set(good)
    for bad in ("alloc", "alloc@0", "alloc@x", "free@1", "alloc@-1", "@3", "alloc@99999999999999999999"):
        with pytest.raises(gbm.GbError) as e:
            gbm.gb_fault_set(bad)
        assert e.value.code == gbm.GB_EINVAL
    gbm.gb_fault_set(None)


def test_fault_fires_on_the_nth_event_only(gbm):
    gbm.gb_fault_set("alloc@3")
    assert [gbm.gb_fault_tick(gbm.GB_FAULT_ALLOC) for _ in range(6)] == [False, False, True, False, False, False]
    assert not any(gbm.gb_fault_tick(gbm.GB_FAULT_SUBMIT) for _ in range(5))
    gbm.gb_fault_set("submit@1,cancel@2")
    assert gbm.gb_fault_tick(gbm.GB_FAULT_SUBMIT) and not gbm.gb_fault_tick(gbm.GB_FAULT_SUBMIT)
    assert [gbm.gb_fault_tick(gbm.GB_FAULT_CANCEL) for _ in range(3)] == [False, True, False]
    # a new spec restarts the counts; a malformed one leaves the spec in force
    gbm.gb_fault_set("alloc@2")
    with pytest.raises(gbm.GbError):
        gbm.gb_fault_set("alloc@")
    assert [gbm.gb_fault_tick(gbm.GB_FAULT_ALLOC) for _ in range(3)] == [False, True, False]
    gbm.gb_fault_set("")
    assert not any(gbm.gb_fault_tick(k) for k in range(3) for _ in range(4))
    assert not gbm.gb_fault_tick(17)


def test_autotune_cache_file_format(gbm, tmp_path):
    """The autotune cache (GB_TUNE_CACHE): entries keyed by GPU, mode and
    sample; the last entry of a key wins, other keys and damaged lines are
    ignored, a missing file or key is a miss."""
    path = str(tmp_path / "tune.txt")
    key = "NVIDIA GB300|152|1|4096|00000000deadbeef|32000000|1048576|8589934592"
    assert gbm.gb_tune_cache_lookup(path, key) is None
    a = dict(tile_bits=1 << 18, bucket_split=1 << 16, p1=1 << 14, cover_prefix=144, seg_len=1 << 24, cta_threads=256)
    b = dict(a, tile_bits=1 << 17, cta_threads=512)
    gbm.gb_tune_cache_store(path, key, a, 61.5)
    gbm.gb_tune_cache_store(path, key.replace("GB300", "B200"), b, 80.0)
    with open(path, "a") as f:
        f.write(key + "\t262144 65536 garbage\n")
    assert gbm.gb_tune_cache_lookup(path, key) == (a, 61.5)
    gbm.gb_tune_cache_store(path, key, b, 60.25)
    assert gbm.gb_tune_cache_lookup(path, key) == (b, 60.25)
    assert gbm.gb_tune_cache_lookup(path, key + "x") is None
    with pytest.raises(gbm.GbError):
        gbm.gb_tune_cache_store(path, "bad\tkey", a, 1.0)
