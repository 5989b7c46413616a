"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/gb.h declares, and its host-only helpers follow the
paper's bitset layout."""
import ctypes
import os
import re

import pytest

from conftest import ROOT, read_golden


@pytest.fixture(scope="module")
def lib():
    from paper_2603_02621_gb300 import build, gb
    build.build()
    return gb.load()


def declared_symbols():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(gb_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("gb_init", "gb_destroy", "gb_sieve_segment", "gb_verify_range",
              "gb_prime_pi", "gb_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2603_02621_gb300 import gb
    assert set(declared_symbols()) <= set(gb.SIGNATURES)


def test_struct_layouts():
    from paper_2603_02621_gb300 import gb
    # sizes follow the C declarations in include/gb.h (LP64)
    assert ctypes.sizeof(gb.gb_config) == 56
    assert ctypes.sizeof(gb.gb_segment_result) == 48
    assert ctypes.sizeof(gb.gb_range_result) == 96


def test_bitset_bytes_table3(lib):
    # Table 3: dense odd-only bitset of 59 / 596 / 5,960 MB at N = 1e9, 1e10, 1e11
    from paper_2603_02621_gb300 import gb
    facts = {k: int(v) for k, v in read_golden("paper_facts.txt")}
    for N, key in [(10**9, "bitset_mib_1e9"), (10**10, "bitset_mib_1e10"), (10**11, "bitset_mib_1e11")]:
        assert gb.gb_bitset_bytes(N) // (1 << 20) == facts[key]
    assert gb.gb_bitset_bytes(3) == 8 and gb.gb_bitset_bytes(2) == 0


def test_strerror(lib):
    from paper_2603_02621_gb300 import gb
    assert gb.gb_strerror(0) == "GB_OK"
    assert "invalid" in gb.gb_strerror(gb.GB_EINVAL)


def test_init_rejects_bad_config(lib):
    from paper_2603_02621_gb300 import gb
    with pytest.raises(gb.GbError) as e:
        gb.gb_init(seg_len=1000)
    assert e.value.code == gb.GB_EINVAL
    with pytest.raises(gb.GbError):
        gb.gb_init(tile_bits=12345)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2603_02621_gb300 import gb
    with pytest.raises(ImportError):
        gb.load(str(tmp_path / "nope.so"))


def test_product_path_never_imports_oracle():
    # the library and its binding must not import, link or load the oracle
    pat = re.compile(r"^\s*(import|from)\s+oracle\b|liboracle|gb_oracle|\bor_(pmin|sieve|verify|mr|td|prime|partitions|isqrt)\w*\(", re.M)
    pkg = os.path.join(ROOT, "paper_2603_02621_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not pat.search(text), f
