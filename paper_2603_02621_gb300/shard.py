"""Host-side sharding, merging and journaling of long verifications.

GoldbachGPU (arXiv 2603.02621) distributes segments over GPUs (Sec. 3.6,
Tables 6-7) and runs verifications that take days; here:

* ``shard_range``: rank r of N takes a contiguous run of whole segments of
  [lo, hi) (segments are S even n from lo, so the per-segment outputs are the
  same however the range is split);
* ``shard_batch``: ranges of a batch dealt to ranks, longest first to the
  least-loaded rank (deterministic);
* ``merge``: range totals combined -- histograms and counts summed, the
  maximum p_min taken with its smallest n (the tie-break of the outputs);
* ``Journal``: an append-only JSON-lines record of finished units, each line
  carrying a checksum; a restart skips the units already recorded and a torn
  last line is ignored;
* ``run_journaled``: verify the units of a range not yet in the journal,
  appending each as it finishes, and return the merge of the whole journal;
* ``gather_merge``: every rank's totals gathered over torch.distributed (gloo
  or nccl) and merged; the only exchange of the path, a few KB.

Nothing here computes: the verification of a unit is a callable (in use,
``Context.verify_range``).
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np


def shard_range(lo: int, hi: int, S: int, world: int, rank: int):
    """[a, b) of rank `rank`: whole segments of S even n from lo, as equal in
    count as possible; an empty range (a == b) when there are fewer segments
    than ranks."""
    if lo % 2 or hi % 2 or hi < lo or S <= 0 or not 0 <= rank < world:
        raise ValueError("bad range or rank")
    nseg = ((hi - lo) // 2 + S - 1) // S
    s0 = nseg * rank // world
    s1 = nseg * (rank + 1) // world
    a = min(hi, lo + 2 * S * s0)
    b = min(hi, lo + 2 * S * s1)
    return a, b


def shard_batch(ranges, world: int, rank: int):
    """Indices of the ranges rank `rank` verifies: longest first, each to the
    rank with the fewest even n so far (ties to the lower rank)."""
    order = sorted(range(len(ranges)), key=lambda i: (-(ranges[i][1] - ranges[i][0]), i))
    load = [0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += (ranges[i][1] - ranges[i][0]) // 2
        if r == rank:
            mine.append(i)
    return sorted(mine)


def empty_totals(hist_len: int):
    return {"n_checked": 0, "unresolved": 0, "max_pmin": 0, "max_pmin_n": 0,
            "hist": np.zeros(hist_len, dtype=np.uint64)}


def totals_of(result: dict, hist_len: int):
    """Range totals from a ``verify_range`` result (dict with 'hist')."""
    h = np.zeros(hist_len, dtype=np.uint64)
    src = np.asarray(result.get("hist", np.zeros(0)), dtype=np.uint64)
    h[:min(hist_len, len(src))] = src[:hist_len]
    return {"n_checked": int(result["n_checked"]), "unresolved": int(result["unresolved"]),
            "max_pmin": int(result["max_pmin"]), "max_pmin_n": int(result["max_pmin_n"]), "hist": h}


def merge(parts, hist_len: int | None = None):
    """Combine range totals: sums, and the largest p_min with its smallest n."""
    parts = list(parts)
    if hist_len is None:
        hist_len = max([len(p["hist"]) for p in parts] or [0])
    out = empty_totals(hist_len)
    for p in parts:
        out["n_checked"] += int(p["n_checked"])
        out["unresolved"] += int(p["unresolved"])
        h = np.asarray(p["hist"], dtype=np.uint64)
        out["hist"][:len(h)] += h[:hist_len]
        pm, pn = int(p["max_pmin"]), int(p["max_pmin_n"])
        if pm and (pm > out["max_pmin"] or (pm == out["max_pmin"] and pn < out["max_pmin_n"])):
            out["max_pmin"], out["max_pmin_n"] = pm, pn
    return out


def _digest(rec: dict) -> str:
    body = json.dumps({k: rec[k] for k in sorted(rec) if k != "sha"}, sort_keys=True)
    return hashlib.sha256(body.encode()).hexdigest()[:16]


class Journal:
    """Append-only record of finished units [lo, hi) with their totals."""

    def __init__(self, path: str):
        self.path = path
        self.units = {}
        if os.path.exists(path):
            # a crash can leave a torn last line: cut the file back to its last
            # newline so that new records start on a line of their own
            with open(path, "rb+") as f:
                data = f.read()
                end = data.rfind(b"\n") + 1
                if end < len(data):
                    f.truncate(end)
            with open(path) as f:
                for line in f:
                    line = line.strip()
                    if not line:
                        continue
                    try:
                        rec = json.loads(line)
                    except json.JSONDecodeError:
                        continue                       # torn write at the end
                    if rec.get("sha") != _digest(rec):
                        continue
                    self.units[(rec["lo"], rec["hi"])] = rec

    def done(self, lo: int, hi: int) -> bool:
        return (lo, hi) in self.units

    def record(self, lo: int, hi: int, totals: dict):
        h = np.asarray(totals["hist"], dtype=np.uint64)
        nz = np.nonzero(h)[0]
        rec = {"lo": lo, "hi": hi, "n_checked": int(totals["n_checked"]),
               "unresolved": int(totals["unresolved"]), "max_pmin": int(totals["max_pmin"]),
               "max_pmin_n": int(totals["max_pmin_n"]), "hist_len": int(len(h)),
               "hist": [[int(i), int(h[i])] for i in nz]}
        rec["sha"] = _digest(rec)
        with open(self.path, "a") as f:
            f.write(json.dumps(rec) + "\n")
            f.flush()
            os.fsync(f.fileno())
        self.units[(lo, hi)] = rec

    @staticmethod
    def totals(rec: dict):
        h = np.zeros(rec["hist_len"], dtype=np.uint64)
        for i, c in rec["hist"]:
            h[i] = c
        return {"n_checked": rec["n_checked"], "unresolved": rec["unresolved"],
                "max_pmin": rec["max_pmin"], "max_pmin_n": rec["max_pmin_n"], "hist": h}

    def merged(self, lo: int, hi: int, hist_len: int):
        return merge([self.totals(r) for (a, b), r in self.units.items() if lo <= a and b <= hi], hist_len)


def units_of(lo: int, hi: int, unit_n: int):
    """[a, b) units of unit_n even n each covering [lo, hi)."""
    out = []
    a = lo
    while a < hi:
        b = min(hi, a + 2 * unit_n)
        out.append((a, b))
        a = b
    return out


def run_journaled(verify, lo: int, hi: int, unit_n: int, journal: Journal, hist_len: int):
    """Verify every unit of [lo, hi) not yet in the journal (verify(a, b) ->
    totals dict), record each, return (merged totals, units verified now)."""
    ran = 0
    for a, b in units_of(lo, hi, unit_n):
        if journal.done(a, b):
            continue
        journal.record(a, b, verify(a, b))
        ran += 1
    return journal.merged(lo, hi, hist_len), ran


def gather_merge(local: dict, hist_len: int):
    """Every rank's totals, merged, on every rank (torch.distributed must be
    initialised)."""
    import torch.distributed as dist
    payload = {"n_checked": int(local["n_checked"]), "unresolved": int(local["unresolved"]),
               "max_pmin": int(local["max_pmin"]), "max_pmin_n": int(local["max_pmin_n"]),
               "hist": np.asarray(local["hist"], dtype=np.uint64).tolist()}
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, payload)
    return merge(parts, hist_len)
