"""Journaled long verification (run.py, Sec. 3.6 / Tables 6-7 of the paper:
long exhaustive runs split into units) on one GPU: a 2^30-n range verified
unit by unit through gb_verify_range into a journal; a failure raised on the
host in the middle of the run; a resume that verifies only the units not yet
journaled; merged totals and histogram equal to the oracle's.  Then the CLI
itself, twice on the same journal (the second run finds every unit done)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P2 = 1 << 20


class Crash(RuntimeError):
    pass


def test_journaled_run_resumes_after_a_host_failure(tmp_path, oracle):
    from paper_2603_02621_gb300 import gb, shard
    from paper_2603_02621_gb300 import run as runmod
    lo, hi, unit = 10**12, 10**12 + 2 * (1 << 30), 1 << 27
    HL = len(oracle.primes_upto(P2))
    jpath = str(tmp_path / "j.jsonl")
    calls = []
    with gb.Context(device=0, base_limit=1 << 20, seg_len=1 << 27, p1=1 << 15, p2=P2) as ctx:
        def verify(a, b):
            calls.append((a, b))
            return shard.totals_of(ctx.verify_range(a, b, hist_cap=HL), HL)

        def failing(a, b):
            if len(calls) == 3:
                raise Crash("host failure after three units")
            return verify(a, b)

        with pytest.raises(Crash):
            runmod.run(lo, hi, unit, jpath, failing, HL, 1, 0)
        assert len(calls) == 3
        tot, ran = runmod.run(lo, hi, unit, jpath, verify, HL, 1, 0)
    assert ran == 5 and len(calls) == 8                                 # only the five units left
    summ, hist = oracle.verify_segments(lo, hi, (hi - lo) // 2, P2, HL)
    assert [tot["n_checked"], tot["unresolved"], tot["max_pmin"], tot["max_pmin_n"]] == summ[0].tolist()
    np.testing.assert_array_equal(tot["hist"], hist[0])


def test_run_cli_twice_on_one_journal(tmp_path):
    lo, hi = 10**13, 10**13 + 2 * (1 << 28)
    cmd = [sys.executable, "-m", "paper_2603_02621_gb300.run", "--lo", str(lo), "--hi", str(hi),
           "--unit", str(1 << 26), "--journal", str(tmp_path / "cli.jsonl")]
    outs = []
    for _ in range(2):
        p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
        assert p.returncode == 0, p.stderr[-2000:]
        outs.append(json.loads(p.stdout.strip().splitlines()[-1]))
    a, b = outs
    assert a["units_run_on_rank0"] == 4 and b["units_run_on_rank0"] == 0
    for k in ("n_checked", "unresolved", "max_pmin", "max_pmin_n", "hist_nonzero"):
        assert a[k] == b[k], k
    assert a["n_checked"] == (hi - lo) // 2 and a["unresolved"] == 0
