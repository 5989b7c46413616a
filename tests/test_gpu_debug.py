"""The debug build (-DGB_DEBUG) on the GPU: the kernels' bounds checks on
their strikes and bucket entries all hold on the sieve paths (tile, slices,
carried large primes, per-chunk large primes), a range verification with the
retry pass and a batch, and its outputs equal the release build's."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, json, sys
import torch
sys.path.insert(0, sys.argv[1])
from paper_2603_02621_gb300 import gb
from paper_2603_02621_gb300.workloads import batched_ranges
lib = gb.load()
out = {"debug_build": lib.gb_debug_build()}
with gb.Context(device=0, base_limit=1 << 31, seg_len=1 << 20, p1=1 << 15, p2=1 << 20) as g:
    for A, nbits in [(4 * 10**18 - 10**11 + 1, (1 << 29) + 77), (10**14 + 1, (1 << 30) + 64),
                     (10**12 + 1, (1 << 22) + 5), (1, 5 * 10**6 + 37)]:
        q = torch.zeros(((nbits + 63) // 64,), dtype=torch.int64, device="cuda")
        pc = g.sieve_segment(A, nbits, q)
        out["sieve %d" % A] = [pc, hashlib.sha256(q.cpu().numpy().tobytes()).hexdigest()]
    r = g.verify_range(10**12, 10**12 + 2 * (1 << 22), 31, hist_cap=4096)
    out["range"] = [r["n_checked"], r["unresolved"], r["max_pmin"], r["max_pmin_n"], r["hist"].tolist()]
    b = g.verify_batch(batched_ranges(count=64, seed=3, log2_min=10, log2_max=20, start_min=10**9,
                                      start_max=10**15), hist_stride=1024)
    out["batch"] = [b["records"], b["hist"].tolist()]
out["debug_word"] = int(lib.gb_debug_word(1))
print(json.dumps(out))
"""


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, timeout=900, env=env,
                       cwd=ROOT)
    assert p.returncode == 0, p.stderr[-3000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_debug_build_checks_hold_and_outputs_match():
    from paper_2603_02621_gb300 import build
    path = build.build(debug=True)
    dbg = _run({"GB_LIBRARY": path})
    rel = _run({"GB_LIBRARY": ""})
    assert dbg.pop("debug_build") == 1 and rel.pop("debug_build") == 0
    assert dbg.pop("debug_word") == 0 and rel.pop("debug_word") == 0
    assert dbg == rel
