"""Host logic of multi-GPU sharding and journaled long runs (CPU only).

The verification of a unit is the CPU oracle here (the GPU path is the same
callable in production); ranks are gloo processes on 127.0.0.1.  Failures are
made on the host: a verification that raises mid-run, a torn journal line, a
rank that exits before the exchange."""
import datetime
import json
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_2603_02621_gb300 import run as runmod
from paper_2603_02621_gb300 import shard

P = 1 << 12
HL = 564                          # pi(2^12)


def _oracle_verify(a, b):
    from oracle import oracle
    summ, hist = oracle.verify_segments(a, b, (b - a) // 2, P, HL, threads=2)
    return {"n_checked": int(summ[0, 0]), "unresolved": int(summ[0, 1]), "max_pmin": int(summ[0, 2]),
            "max_pmin_n": int(summ[0, 3]), "hist": hist[0]}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_range_partitions_whole_segments():
    lo, hi, S = 10**9, 10**9 + 2 * 1000003, 4096
    for world in (1, 2, 3, 7, 300):
        parts = [shard.shard_range(lo, hi, S, world, r) for r in range(world)]
        assert parts[0][0] == lo and parts[-1][1] == hi
        for (a, b), (c, d) in zip(parts, parts[1:]):
            assert b == c                                   # contiguous, disjoint
        for a, b in parts:
            assert (a - lo) % (2 * S) == 0                  # starts on a segment boundary
    with pytest.raises(ValueError):
        shard.shard_range(5, 11, 4, 2, 0)


def test_shard_batch_is_a_balanced_partition():
    from paper_2603_02621_gb300.workloads import batched_ranges
    ranges = batched_ranges(count=500, seed=3)
    world = 4
    parts = [shard.shard_batch(ranges, world, r) for r in range(world)]
    assert sorted(i for p in parts for i in p) == list(range(len(ranges)))
    loads = [sum((ranges[i][1] - ranges[i][0]) // 2 for i in p) for p in parts]
    biggest = max((b - a) // 2 for a, b in ranges)
    assert max(loads) - min(loads) <= biggest


def test_merge_equals_whole_range(oracle):
    lo, hi = 10**8, 10**8 + 2 * 30011
    whole = _oracle_verify(lo, hi)
    parts = [_oracle_verify(a, b) for a, b in shard.units_of(lo, hi, 4099)]
    m = shard.merge(parts, HL)
    assert (m["n_checked"], m["unresolved"], m["max_pmin"], m["max_pmin_n"]) == \
        (whole["n_checked"], whole["unresolved"], whole["max_pmin"], whole["max_pmin_n"])
    np.testing.assert_array_equal(m["hist"], whole["hist"])
    # the tie-break: equal maxima keep the smaller n
    t = shard.merge([dict(whole, max_pmin_n=whole["max_pmin_n"] + 10), whole], HL)
    assert t["max_pmin_n"] == whole["max_pmin_n"]


def test_journal_resumes_after_a_crash(tmp_path, oracle):
    lo, hi, unit = 10**10, 10**10 + 2 * 20000, 3000
    path = str(tmp_path / "j.jsonl")
    calls = []

    def flaky(a, b):
        if len(calls) == 3:
            raise RuntimeError("simulated failure of the fourth unit")
        calls.append((a, b))
        return _oracle_verify(a, b)

    with pytest.raises(RuntimeError):
        shard.run_journaled(flaky, lo, hi, unit, shard.Journal(path), HL)
    assert len(shard.Journal(path).units) == 3
    with open(path, "a") as f:
        f.write('{"lo": 1, "hi": ')                       # torn write of a crashed process
    again = []

    def ok(a, b):
        again.append((a, b))
        return _oracle_verify(a, b)

    merged, ran = shard.run_journaled(ok, lo, hi, unit, shard.Journal(path), HL)
    n_units = len(shard.units_of(lo, hi, unit))
    assert ran == n_units - 3 and not set(again) & set(calls)
    whole = _oracle_verify(lo, hi)
    assert (merged["n_checked"], merged["max_pmin"], merged["max_pmin_n"]) == \
        (whole["n_checked"], whole["max_pmin"], whole["max_pmin_n"])
    np.testing.assert_array_equal(merged["hist"], whole["hist"])
    # a tampered record is rejected by its checksum
    lines = open(path).read().splitlines()
    rec = json.loads(lines[0])
    rec["n_checked"] += 1
    with open(path, "w") as f:
        f.write("\n".join([json.dumps(rec)] + lines[1:]) + "\n")
    assert len(shard.Journal(path).units) == n_units - 1


def _rank_main(rank, world, port, lo, hi, unit, jpath, out_q, fail_rank):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    try:
        if rank == fail_rank:
            raise SystemExit(3)                          # leaves before the exchange
        mine, ran = runmod.run(lo, hi, unit, jpath, _oracle_verify, HL, world, rank)
        total = shard.gather_merge(mine, HL)
        out_q.put((rank, "ok", total["n_checked"], total["max_pmin"], total["max_pmin_n"],
                   total["hist"].tolist(), ran))
    except SystemExit:
        raise
    except Exception as e:                               # noqa: BLE001 - reported to the test
        out_q.put((rank, "error", type(e).__name__))
    finally:
        if rank != fail_rank:
            try:
                dist.destroy_process_group()
            except Exception:                            # noqa: BLE001
                pass


def _spawn(world, lo, hi, unit, jpath, fail_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, lo, hi, unit, jpath, q, fail_rank))
             for r in range(world)]
    for p in procs:
        p.start()
    results = []
    for _ in range(world - (1 if fail_rank >= 0 else 0)):
        results.append(q.get(timeout=120))
    for p in procs:
        p.join(timeout=60)
    return sorted(results)


def test_two_gloo_ranks_shard_and_merge(tmp_path, oracle):
    lo, hi, unit = 10**9, 10**9 + 2 * 24000, 2500
    jpath = str(tmp_path / "run.jsonl")
    res = _spawn(2, lo, hi, unit, jpath)
    whole = _oracle_verify(lo, hi)
    assert [r[1] for r in res] == ["ok", "ok"]
    for r in res:
        assert (r[2], r[3], r[4]) == (whole["n_checked"], whole["max_pmin"], whole["max_pmin_n"])
        np.testing.assert_array_equal(np.array(r[5], dtype=np.uint64), whole["hist"])
    # a second run finds every unit in the ranks' journals and verifies none
    res2 = _spawn(2, lo, hi, unit, jpath)
    assert [r[6] for r in res2] == [0, 0]
    assert res2[0][2:6] == res[0][2:6]


def test_rank_leaving_before_the_exchange_is_detected(tmp_path):
    lo, hi, unit = 10**9, 10**9 + 2 * 4000, 1000
    res = _spawn(2, lo, hi, unit, str(tmp_path / "f.jsonl"), fail_rank=1)
    assert len(res) == 1 and res[0][0] == 0 and res[0][1] == "error"
