"""Long verifications: ``python -m paper_2603_02621_gb300.run --lo 4 --hi 1000000000002``.

One process per GPU (``torchrun --nproc-per-node N``): rank r verifies its
contiguous share of the range (whole units, ``shard.shard_range``), unit by
unit through ``gb_verify_range``, recording each finished unit in its own
journal (``<journal>.rank<r>``), so a restart resumes where it stopped; the
ranks' totals are then gathered and merged (the only exchange) and rank 0
prints them as one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

from . import shard


def run(lo: int, hi: int, unit_n: int, journal_path: str, verify, hist_len: int, world: int, rank: int):
    """Host logic of one rank: its share, journaled; returns (its totals,
    units verified in this call)."""
    a, b = shard.shard_range(lo, hi, unit_n, world, rank)
    j = shard.Journal(f"{journal_path}.rank{rank}")
    if a == b:
        return shard.empty_totals(hist_len), 0
    return shard.run_journaled(verify, a, b, unit_n, j, hist_len)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--lo", type=int, default=4)
    ap.add_argument("--hi", type=int, required=True)
    ap.add_argument("--unit", type=int, default=1 << 32, help="even n per journaled unit")
    ap.add_argument("--seg", type=int, default=1 << 27, help="even n per segment")
    ap.add_argument("--p1", type=int, default=1 << 15)
    ap.add_argument("--p2", type=int, default=1 << 20)
    ap.add_argument("--journal", default="goldbach_journal.jsonl")
    args = ap.parse_args(argv)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    from . import gb
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    hist_len = int(gb.Context(device=local, base_limit=1 << 16).prime_pi(args.p2))
    base = max(1 << 16, math.isqrt(args.hi + 4096) + 1)
    with gb.Context(device=local, base_limit=base, seg_len=args.seg, p1=args.p1, p2=args.p2) as ctx:
        def verify(a, b):
            return shard.totals_of(ctx.verify_range(a, b, hist_cap=hist_len), hist_len)
        mine, ran = run(args.lo, args.hi, args.unit, args.journal, verify, hist_len, world, rank)
    total = shard.gather_merge(mine, hist_len) if world > 1 else mine
    if rank == 0:
        print(json.dumps({"lo": args.lo, "hi": args.hi, "n_checked": total["n_checked"],
                          "unresolved": total["unresolved"], "max_pmin": total["max_pmin"],
                          "max_pmin_n": total["max_pmin_n"], "units_run_on_rank0": ran,
                          "hist_nonzero": int((total["hist"] > 0).sum())}), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
