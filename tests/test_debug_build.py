"""The debug build (-DGB_DEBUG, libgb_debug.so): it compiles for sm_103a,
loads, says it is the debug build, and reports no failed check before any
kernel ran; the release build reports 0.  No GPU needed."""
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_debug_build_compiles_and_loads():
    from paper_2603_02621_gb300 import build
    path = build.build(debug=True)
    assert path.endswith("libgb_debug.so") and os.path.exists(path)
    lib = ctypes.CDLL(path)
    lib.gb_debug_build.restype = ctypes.c_int
    assert lib.gb_debug_build() == 1


def test_release_build_has_no_debug_words():
    from paper_2603_02621_gb300 import gb
    lib = gb.load()
    assert lib.gb_debug_build() == 0 and lib.gb_debug_word(1) == 0
