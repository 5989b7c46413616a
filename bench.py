"""Benchmark of the Goldbach verifier on the GPU (one JSON line, rank 0).

Modes (--mode), each a workload of GoldbachGPU (arXiv 2603.02621):

* exhaustive-1e12 (default): exhaustive verification of every even n in
  [4, 10^12] (Table 4's largest range, the paper's headline): one step = one
  gb_verify_range call over the range -- segments of 2^27 even n, base primes
  to 2^31, the segment sieve of the q window, the loop-inverted cover with
  P1 = 2^15, the GPU retry pass to P2 = 2^20, per-segment reductions
  (Sec. 2.3).  The same line carries, as extra keys, the 10^11-wide window
  [4e18 - 10^11, 4e18) (``window_4e18``) and the 4096-range batch against the
  per-range launch loop over the same ranges (``batched``);
* plain: [4, 10^10], segments of 2^24 even n;
* window-4e18, batched, serving: one of those workloads alone.

Multi-GPU (torchrun): plain family -- the range is cut into contiguous runs of
whole segments, one per rank (strong scaling; the ranks' totals are merged by
one gather after timing, the only exchange); batched -- each rank its own 4096
ranges (weak scaling).  The timing is the max over ranks.

--impl reference times the CPU oracle (oracle/) on seeded units of the same
workload (whole segments of the range), on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "even integers verified/sec"
UNIT = "even n/s"
P1, P2 = 1 << 15, 1 << 20
HL = 3512                           # pi(2^15): histogram row length
# the paper's number for the same workload (Table 4, one RTX 3070)
PAPER_BY_MODE = {"plain": 4999999999 / 23.547, "exhaustive-1e12": 499999999999 / 2457.040}
PAPER_CONTEXT = ("RTX 3070 (8 GB), Table 4: [4, 1e10] in 23,547 ms = 2.12e8 n/s; "
                 "[4, 1e12] in 2,457,040 ms = 2.03e8 n/s")
DEFAULT_MODE = "exhaustive-1e12"

# plain-family workloads: (range, segment length, base primes)
PLAIN_MODES = {
    "plain": dict(lo=4, hi=10**10 + 2, seg=1 << 24, base=None,
                  workload="exhaustive Goldbach verification of every even n in [4, 1e10]"),
    "exhaustive-1e12": dict(lo=4, hi=10**12 + 2, seg=1 << 27, base=1 << 31,
                            workload="exhaustive Goldbach verification of every even n in [4, 1e12]"),
    "window-4e18": dict(lo=4 * 10**18 - 10**11, hi=4 * 10**18, seg=1 << 27, base=1 << 31,
                        workload="Goldbach verification of every even n in the window [4e18 - 1e11, 4e18)"),
}
# DRAM bytes per unit of the dominant kernels (cover: even n; sieve and the
# slices: q bits), from ncu captures of the kernels as built (profiles/):
# scaled to a launch by the units it processes.  A workload without a capture
# of the current kernels reports no traffic.
NCU_TRAFFIC = {
    # 2^31 even n near 1e12 (profiles/k_cover_fast_1e12.md, k_sieve_1e12.md, k_mid_1e12.md)
    "exhaustive-1e12": {"cover": 0.12672, "sieve": 0.09678, "large": 0.22411},
}


def rank_range(mode: str, rank: int, world: int = 1):
    """[a, b) of rank `rank`: the whole range at N = 1, else a contiguous run
    of whole segments (strong scaling)."""
    from paper_2603_02621_gb300 import shard
    m = PLAIN_MODES[mode]
    return shard.shard_range(m["lo"], m["hi"], m["seg"], world, rank)


def base_for(mode: str, hi: int) -> int:
    b = PLAIN_MODES[mode]["base"] if mode in PLAIN_MODES else None
    return b or max(10**5, math.isqrt(hi + 4096) + 1)


def workload_desc(mode: str, world: int):
    if mode == "serving":
        return {"workload": "serving: Poisson stream, 2000 req/s offered, 90% ranges of 2^16..2^30 even n "
                            "at offsets uniform in [1e9, 4e18], 10% single-n queries (n < 4e18)",
                "requests": 2000, "seed": 7, "p2": P2}
    if mode == "batched":
        return {"workload": "4096 ranges per GPU, lengths log-uniform 2^10..2^26 even n, starts uniform "
                            "in [1e9, 1e15] (splitmix64 seed 1 + rank), one gb_verify_batch call",
                "ranges": 4096, "seeds": [1 + r for r in range(world)], "base_primes_to": 32 * 10**6,
                "p2": P2, "outputs": f"per-range record and p_min histogram row ({HL} entries)",
                "tuning": "gb_autotune on the same batch before timing",
                "l2": "batch q buffer ~3.1 GB > 126 MB L2; no flush needed"}
    m = PLAIN_MODES[mode]
    n = (m["hi"] - m["lo"]) // 2
    return {"workload": m["workload"], "range": [m["lo"], m["hi"]], "even_n": n,
            "rank_ranges": [list(rank_range(mode, r, world)) for r in range(world)],
            "seg_len": m["seg"], "base_primes_to": base_for(mode, m["hi"]) if m["base"] else "isqrt(hi)+ (>= 1e5)",
            "p1": P1, "p2": P2,
            "outputs": f"per-segment p_min histogram ({HL} entries), max p_min with n, unresolved",
            "l2": f"q window {min(n, 1 << 33) / 8 / 1e6:.0f} MB per slab > 126 MB L2; no flush needed"}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks, power and throttle reasons every 20 ms while running,
    each sample stamped on arrival.  The SM clock and the throttle reasons are
    taken over the samples that arrived inside the timed regions (between
    mark_start and mark_end, plus 50 ms for the output to arrive); if a region
    was too short to catch one, over the samples taken under load (GPU
    utilization >= 50 %), else over all samples."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.t_start = None
        self.t_end = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def mark_start(self):
        self.t_start = time.monotonic()

    def mark_end(self):
        self.t_end = time.monotonic()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows, mx = [], 0.0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in list(self.lines):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                clk = float(parts[0])
                mx = max(mx, float(parts[1]))
                util = float(parts[7])
            except ValueError:
                continue
            rows.append((t, clk, util, {nm for nm, v in zip(names, parts[3:7]) if v.lower() == "active"}))
        inside = []
        if self.t_start is not None and self.t_end is not None:
            inside = [r for r in rows if self.t_start <= r[0] <= self.t_end + 0.05]
        busy = [r for r in rows if r[2] >= 50.0]
        use = inside or busy or rows
        reasons = set().union(*(r[3] for r in use)) if use else set()
        return {"sm_mhz": statistics.median(r[1] for r in use) if use else None, "sm_max_mhz": mx or None,
                "samples": len(rows), "samples_in_timed_region": len(inside), "samples_under_load": len(busy),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- helpers
def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x: float, world: int, backend_ready: bool):
    if world == 1 or not backend_ready:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, backend_ready: bool):
    if world > 1 and backend_ready:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- cpu baseline
def sample_units(mode: str, seed: int = 11):
    """The workload cut into independent units (lo, hi) the oracle can verify
    one by one, in a seeded random order: the range's segments for the plain
    family, the ranges for the batched mode."""
    from paper_2603_02621_gb300 import workloads
    if mode == "batched":
        units = workloads.batched_ranges(count=4096, seed=1)
    elif mode == "serving":
        units = [(a, b) for t, kind, a, b in workloads.serving_stream(count=2000, seed=7) if kind == "range"]
    else:
        m = PLAIN_MODES[mode]
        lo, hi, seg = m["lo"], m["hi"], m["seg"]
        units = [(a, min(a + 2 * seg, hi)) for a in range(lo, hi, 2 * seg)]
    rng = workloads.SplitMix64(seed)
    order = list(range(len(units)))
    for i in range(len(order) - 1, 0, -1):          # seeded shuffle
        j = rng.below(i + 1)
        order[i], order[j] = order[j], order[i]
    return [units[i] for i in order]


def unit_kind(mode: str) -> str:
    if mode in PLAIN_MODES:
        m = PLAIN_MODES[mode]
        return "segments of %d even n of [%d, %d)" % (m["seg"], m["lo"], m["hi"])
    return {"batched": "ranges of the 4096-range batch", "serving": "range requests of the serving stream"}[mode]


class OracleRunner:
    """The oracle, as it stands, on seeded units of the workload: one unit per
    host thread at a time, each verified by the oracle in one thread."""

    def __init__(self, mode: str, seed: int = 11):
        from oracle import oracle
        import concurrent.futures as cf
        self.oracle = oracle
        self.mode = mode
        self.threads = oracle.default_threads()
        self.units = sample_units(mode, seed)
        self.used = 0
        self.ex = cf.ThreadPoolExecutor(max_workers=self.threads)
        if mode != "plain":
            hi_max = max(b for _, b in self.units)
            oracle.verify_segments(hi_max - 4, hi_max, 2, P2, 8, threads=1)   # the prime cache, untimed

    def _one(self, u):
        a, b = u
        s, _ = self.oracle.verify_segments(a, b, (b - a) // 2, P2, HL, threads=1)
        return int(s[:, 0].sum())

    def step(self):
        """One batch of `threads` units (wrapping around the sample): returns
        (even n verified, wall seconds)."""
        batch = [self.units[(self.used + k) % len(self.units)] for k in range(self.threads)]
        self.used += len(batch)
        t0 = time.perf_counter()
        n = sum(self.ex.map(self._one, batch))
        return n, time.perf_counter() - t0

    def close(self):
        self.ex.shutdown()


def cpu_baseline(mode: str = "plain", min_seconds: float = 12.0, seed: int = 11):
    """The oracle on a bounded sample of the workload's units: batches of one
    unit per host thread until min_seconds of wall time have passed."""
    r = OracleRunner(mode, seed)
    done_n, wall, steps = 0, 0.0, 0
    while wall < min_seconds and r.used < len(r.units):
        n, dt = r.step()
        done_n += n
        wall += dt
        steps += 1
    r.close()
    return {"value": done_n / wall, "unit": UNIT, "cores": r.threads, "kind": "oracle",
            "value_per_core": done_n / wall / r.threads,
            "sample": f"{r.used} seeded {unit_kind(mode)} ({done_n} n, {wall:.1f} s wall, P = 2^20)",
            "seconds": wall}


def roofline_of(prof, wk, alg_cover, steps, mode, peaks, peak_src, sms):
    """Roofline of the dominant kernel from the library's per-kernel profile
    (prof[k]: total ms, launches, work units over the timed region) and work
    counters (wk), as per-launch averages: algorithmic ALU ops per launch over
    the launch's CUDA-event time, against the ALU peak derived from the
    device's SM count, the ALU lanes per SM and the clock; DRAM bytes per
    launch from an ncu capture of the same kernel (NCU_TRAFFIC)."""
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # Both hot kernels are bound by the SM's integer ALU pipe (shifts and
    # logic ops; ncu shows it near saturation).  Its peak, from the unit counts
    # and clock: SMs x 64 ALU lanes per cycle (16 per scheduler: half the
    # issue rate, measured by a shift/or loop) x the maximum SM clock.
    alu_peak = sms * 64 * sm_max * 1e6 / 1e12            # T ALU lane-ops/s
    ncu_traffic = NCU_TRAFFIC.get(mode, {})
    per = {}
    for kern in ("sieve", "cover", "large"):
        kp = prof[kern]
        if kp["launches"] == 0:
            continue
        nl = kp["launches"]
        ms = kp["ms"] / nl
        if kern == "large":
            # primes above the tile split: 2 ALU ops per strike (word index,
            # rotated mask) issued as an atomic AND
            units = wk["large_strikes"] / nl
            ops = 2.0 * units
        elif kern == "cover" and alg_cover is not None:
            # algorithmic work: per 64-n word, the odd primes applied until
            # the word is full (counted by the generic cover, equal to the
            # oracle's count); 4 ALU ops each: the 64-bit funnel shift that
            # aligns the partner bits (2) and the OR into C (2)
            units = float(alg_cover) * steps / nl       # alg_cover is per step
            ops = 4.0 * units
        elif kern == "cover":
            # (batched mode) the block cover's own steps: 2 ops per (32-bit
            # coverage word, prime) step, 2 per probed (n, prime)
            units = wk["cover_iterations"] / nl
            ops = 2.0 * units
        else:
            # minimal ALU work: 2 ops per strike (word index, rotated mask) and
            # 6 per stamped 32-bit word (four pattern funnel shifts, two ANDs)
            units = wk["sieve_strikes"] / nl
            ops = 2.0 * units + 6.0 * (kp["units"] / nl) / 32.0
        alg_bytes = kp["units"] / nl / 8.0               # the q bits, written once / read once
        traffic = ncu_traffic[kern] * kp["units"] / nl if kern in ncu_traffic else None
        achieved = ops / (ms / 1000.0) / 1e12
        per[kern] = {"ms_per_launch": ms, "ms_total": kp["ms"], "launches": nl,
                     "achieved": achieved, "frac": achieved / alu_peak,
                     "alu_ops_per_launch": ops, "work_units_per_launch": units,
                     "dram_bytes_per_launch": traffic, "algorithmic_bytes_per_launch": alg_bytes,
                     "hbm_frac": (alg_bytes / (ms / 1000.0)) / (float(peaks.get("hbm_gbs", 6800.0)) * 1e9)}
    kern = max(per, key=lambda k: per[k]["ms_total"])
    return {"kernel": kern, "bound": "alu", "achieved": per[kern]["achieved"], "peak": alu_peak,
            "unit": "T ALU lane-ops/s", "frac": per[kern]["frac"],
            "traffic": per[kern]["dram_bytes_per_launch"],
            "peak_source": "derived: %d SMs (device attribute) x 64 ALU lanes x %.0f MHz (%s max clock)"
                           % (sms, sm_max, peak_src),
            "work": ("cover: 4 ALU ops per (64-n word, odd prime) iteration until the word is full "
                     "(algorithmic count); sieve: 2 per strike + 6 per stamped 32-bit word; "
                     "large primes: 2 per strike"),
            "kernels": per,
            "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6800.0)), "hbm_peak_source": peak_src}


def run_reference(args, world, rank):
    """The oracle as the reference arm: each step one batch of seeded units of
    the workload (one whole segment per host thread), timed on the wall clock;
    value = even n verified in the timed steps / their wall time."""
    if rank != 0:
        return 0
    mode = args.mode
    r = OracleRunner(mode)
    for _ in range(args.warmup):
        r.step()
    done_n, wall = 0, 0.0
    for _ in range(args.steps):
        n, dt = r.step()
        done_n += n
        wall += dt
    r.close()
    value = done_n / wall
    sample = (f"{args.steps} steps of {r.threads} seeded {unit_kind(mode)} each "
              f"({done_n} n verified in {wall:.1f} s wall, P = 2^20)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / max(1, args.steps),
            "n_per_step": done_n / max(1, args.steps),
            "higher_is_better": True, "scaling": "strong" if mode in PLAIN_MODES else "weak",
            "vs_baseline": value / PAPER_BY_MODE[mode] if mode in PAPER_BY_MODE else None,
            "dtype": "u64", "data": "synthetic", "mode": mode, "config": workload_desc(mode, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r.threads, "kind": "oracle",
                             "value_per_core": value / r.threads, "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_n(mode: str, rank: int = 0) -> int:
    if mode == "serving":
        from paper_2603_02621_gb300 import workloads
        return sum((b - a) // 2 for t, kind, a, b in workloads.serving_stream(count=2000, seed=7 + rank)
                   if kind == "range")
    if mode == "batched":
        from paper_2603_02621_gb300 import workloads
        return sum((b - a) // 2 for a, b in workloads.batched_ranges(count=4096, seed=1 + rank))
    m = PLAIN_MODES[mode]
    return (m["hi"] - m["lo"]) // 2


# ----------------------------------------------------------------------------- workloads on the GPU
class PlainWork:
    """One gb_verify_range call over the rank's share of the range per step."""

    def __init__(self, gb, torch, mode, rank, world, local, stream, parent=None):
        self.gb = gb
        self.mode = mode
        self.lo, self.hi = rank_range(mode, rank, world)
        self.seg = PLAIN_MODES[mode]["seg"]
        if parent is not None and parent.config()["base_limit"] >= base_for(mode, PLAIN_MODES[mode]["hi"]):
            self.ctx = parent.share(stream.cuda_stream)
            self.ctx.set_config(seg_len=self.seg, p1=P1, p2=P2)
        else:
            self.ctx = gb.Context(device=local, base_limit=base_for(mode, PLAIN_MODES[mode]["hi"]),
                                  seg_len=self.seg, p1=P1, p2=P2, stream=stream.cuda_stream)
        self.n = (self.hi - self.lo) // 2
        self.nseg = max(1, (self.n + self.seg - 1) // self.seg)
        # device-resident outputs for the device-timed value, pinned host ones for e2e
        self.d_rows = torch.zeros((self.nseg, HL), dtype=torch.int64, device="cuda")
        self.d_segs = torch.zeros((self.nseg, 6), dtype=torch.int64, device="cuda")    # 48-byte records
        self.h_rows = torch.zeros((self.nseg, HL), dtype=torch.int64).pin_memory()
        self.h_segs = torch.zeros((self.nseg, 6), dtype=torch.int64).pin_memory()
        self.h_hist = torch.zeros(HL, dtype=torch.int64).pin_memory()
        self.last = None
        self.tuned = None

    def autotune(self):
        """gb_autotune on the rank's own range (plain mode), before timing."""
        cfg, ms = self.ctx.autotune([(self.lo, self.hi)], self.gb.GB_TUNE_PLAIN, reps=1)
        # per-segment outputs follow seg_len: keep the workload's
        self.ctx.set_config(seg_len=self.seg)
        self.tuned = ({k: cfg[k] for k in ("tile_bits", "bucket_split", "cta_threads", "p1", "cover_prefix")},
                      ms)

    def _call(self, rows, segs, hist):
        gb = self.gb
        if self.n == 0:
            return None
        r = gb.gb_range_result()
        r.seg_hist = ctypes_ptr(rows)
        r.seg_hist_stride = HL
        r.seg_cap = self.nseg
        r.segs = ctypes_segs(segs)
        if hist is not None:
            r.hist = ctypes_ptr(hist)
            r.hist_cap = HL
        rc = gb.load().gb_verify_range(self.ctx.handle, self.lo, self.hi, 0, gb.ctypes.byref(r))
        if rc:
            raise gb.GbError(rc, "gb_verify_range", gb.gb_last_error())
        self.last = r
        return r

    def step_device(self):
        return self._call(self.d_rows, self.d_segs, None)

    def step_host(self):
        return self._call(self.h_rows, self.h_segs, self.h_hist)

    def totals(self):
        """The rank's totals of the last host step (for the merge)."""
        import numpy as np
        r = self.last
        if r is None:
            return {"n_checked": 0, "unresolved": 0, "max_pmin": 0, "max_pmin_n": 0,
                    "hist": np.zeros(HL, dtype=np.uint64)}
        return {"n_checked": int(r.n_checked), "unresolved": int(r.unresolved), "max_pmin": int(r.max_pmin),
                "max_pmin_n": int(r.max_pmin_n), "hist": self.h_hist.numpy().view(np.uint64).copy()}

    def algorithmic_cover_iterations(self):
        """The cover's algorithmic work for one step (untimed): the generic
        cover (cover_prefix 1) counts, per 64-n word, the odd primes applied
        until the word is full -- equal to the oracle's count from the p_min
        values (tests/test_gpu_work.py)."""
        gb = self.gb
        if self.n == 0:
            return 0
        saved = self.ctx.config()["cover_prefix"]
        self.ctx.set_config(cover_prefix=1)
        gb.gb_profile_enable(self.ctx.handle, True)
        self.step_device()
        iters = gb.gb_profile_work(self.ctx.handle)["cover_iterations"]
        gb.gb_profile_enable(self.ctx.handle, False)
        self.ctx.set_config(cover_prefix=saved)
        return iters

    def extra(self):
        if self.tuned is None:
            return {}
        return {"autotuned": self.tuned[0], "autotune_best_ms": self.tuned[1]}


class BatchWork:
    """One gb_verify_batch call over the rank's 4096 ranges per step."""

    def __init__(self, gb, torch, rank, local, stream):
        from paper_2603_02621_gb300 import workloads
        self.gb, self.torch = gb, torch
        self.mode = "batched"
        self.ranges = workloads.batched_ranges(count=4096, seed=1 + rank)
        self.count = len(self.ranges)
        self.n = sum((b - a) // 2 for a, b in self.ranges)
        self.ctx = gb.Context(device=local, base_limit=32 * 10**6, seg_len=1 << 24, p1=P1, p2=P2,
                              stream=stream.cuda_stream)
        self.lo = (gb.c_uint64 * self.count)(*[a for a, _ in self.ranges])
        self.hi = (gb.c_uint64 * self.count)(*[b for _, b in self.ranges])
        self.d_res = torch.zeros((self.count, 6), dtype=torch.int64, device="cuda")
        self.d_rows = torch.zeros((self.count, HL), dtype=torch.int64, device="cuda")
        self.h_res = torch.zeros((self.count, 6), dtype=torch.int64).pin_memory()
        self.h_rows = torch.zeros((self.count, HL), dtype=torch.int64).pin_memory()
        self.tuned, self.tune_ms = self.ctx.autotune(self.ranges, gb.GB_TUNE_BATCH, reps=1)

    def _call(self, res, rows):
        gb = self.gb
        rc = gb.load().gb_verify_batch(self.ctx.handle, self.lo, self.hi, self.count, 0,
                                       res.data_ptr(), rows.data_ptr(), HL)
        if rc:
            raise gb.GbError(rc, "gb_verify_batch", gb.gb_last_error())

    def step_device(self):
        self._call(self.d_res, self.d_rows)

    def step_host(self):
        self._call(self.h_res, self.h_rows)

    def check(self):
        import numpy as np
        raw = self.h_res.numpy().view(np.uint64)
        unres = int(raw[:, 3].sum())
        mp = (raw[:, 5] & 0xffffffff).astype(np.int64)
        k = int(np.argmax(mp))
        return {"unresolved": unres, "max_pmin": int(mp[k]), "max_pmin_n": int(raw[k, 4]),
                "n_checked": int(raw[:, 2].sum())}

    def algorithmic_cover_iterations(self):
        return None

    def extra(self):
        """The plain per-range launch loop over the same ranges, same outputs
        (per-range totals and histogram row, device-resident), timed once after
        one warm-up pass, with CUDA events on the context's stream."""
        gb, torch = self.gb, self.torch
        d_hist = torch.zeros((self.count, HL), dtype=torch.int64, device="cuda")
        lib = gb.load()

        def loop():
            for i, (a, b) in enumerate(self.ranges):
                r = gb.gb_range_result()
                r.hist = ctypes_ptr(d_hist[i])
                r.hist_cap = HL
                rc = lib.gb_verify_range(self.ctx.handle, a, b, 0, gb.ctypes.byref(r))
                if rc:
                    raise gb.GbError(rc, "gb_verify_range", gb.gb_last_error())

        loop()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record(stream)
        loop()
        ev1.record(stream)
        torch.cuda.synchronize()
        wall_s = time.perf_counter() - t0
        loop_ms = ev0.elapsed_time(ev1)
        same = bool(torch.equal(d_hist, self.d_rows))
        return {"plain_loop": {"value": self.n / (loop_ms / 1000.0), "unit": UNIT, "ms": loop_ms,
                               "wall_ms": 1000.0 * wall_s,
                               "launch": "gb_verify_range per range, same per-range histograms",
                               "same_histograms": same},
                "autotuned": {k: self.tuned[k] for k in ("tile_bits", "bucket_split", "cta_threads", "p1",
                                                         "cover_prefix")},
                "autotune_best_ms": self.tune_ms}


def measure(work, gb, torch, stream, steps, warmup, world, backend_ready, peaks, peak_src, sms, clocks=None):
    """Warm-up, then `steps` steps timed with CUDA events on the context's
    stream (device-resident outputs, per-kernel profile), then `steps` steps
    through the same public call with pinned host outputs on the wall clock
    (e2e, with the bytes the calls copied between host and device)."""
    ctx = work.ctx
    alg_cover = work.algorithmic_cover_iterations()
    torch.cuda.synchronize()
    for _ in range(warmup):
        work.step_device()
    torch.cuda.synchronize()
    # the kernels' work counts (strikes, cover steps) from one untimed step:
    # they add to the strike loops, so the timed steps run without them
    gb.gb_profile_enable(ctx.handle, True)
    work.step_device()
    wk = {k: v * steps for k, v in gb.gb_profile_work(ctx.handle).items()}
    gb.gb_profile_enable(ctx.handle, False)
    torch.cuda.synchronize()

    gb.gb_profile_enable(ctx.handle, gb.GB_PROFILE_EVENTS)
    barrier(world, backend_ready)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.mark_start()
    ev0.record(stream)
    for _ in range(steps):
        work.step_device()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world, backend_ready)
    dev_ms = ev0.elapsed_time(ev1)
    prof = gb.gb_profile_read(ctx.handle)
    launches = gb.gb_profile_kernels(ctx.handle)
    gb.gb_profile_enable(ctx.handle, False)            # (also resets the copy counters)
    max_ms = reduce_max(dev_ms, world, backend_ready)

    barrier(world, backend_ready)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        work.step_host()
    torch.cuda.synchronize()
    e2e_ms = 1000.0 * (time.perf_counter() - t0)
    if clocks:
        clocks.mark_end()
    copies = gb.gb_profile_copies(ctx.handle)
    e2e_ms = reduce_max(e2e_ms, world, backend_ready)

    n_all = workload_n(work.mode) if work.mode in PLAIN_MODES else work.n * world
    total_n = n_all * steps
    return {"value": total_n / (max_ms / 1000.0), "ms_per_step": max_ms / steps, "steps": steps, "warmup": warmup,
            "e2e": {"value": total_n / (e2e_ms / 1000.0), "unit": UNIT,
                    "h2d_bytes_per_step": copies["h2d"] / steps, "d2h_bytes_per_step": copies["d2h"] / steps,
                    "copies": "counted by the library (gb_profile_copies) over the e2e steps"},
            "roofline": roofline_of(prof, wk, alg_cover, steps, work.mode, peaks, peak_src, sms),
            "gpu_launches": int(launches), "kernel_ms": {k: prof[k]["ms"] for k in prof},
            "algorithmic_cover_iterations_per_step": alg_cover}


def merged_check(work, world, backend_ready):
    """Totals of the whole range (plain family): the ranks' totals of their
    last host step, merged by one gather (the only exchange)."""
    from paper_2603_02621_gb300 import shard
    local = work.totals()
    tot = shard.gather_merge(local, HL) if world > 1 and backend_ready else local
    return {"n_checked": int(tot["n_checked"]), "unresolved": int(tot["unresolved"]),
            "max_pmin": int(tot["max_pmin"]), "max_pmin_n": int(tot["max_pmin_n"])}


# ----------------------------------------------------------------------------- serving
def run_serving(args, gb, torch, world, rank, local, backend_ready):
    """Config-5 style serving: a Poisson stream (2000 req/s offered, seed 7 +
    rank) of 90% range verifications (2^16..2^30 even n at offsets uniform in
    [1e9, 4e18]) and 10% single-n queries, paced by arrival time into the
    continuous-batching server; value = range n verified per second of wall
    time from the first arrival to the last completion."""
    from paper_2603_02621_gb300 import workloads
    ctx = gb.Context(device=local, base_limit=1 << 32, p1=P1, p2=P2)

    def serve(reqs, lanes):
        out = [None] * len(reqs)
        with gb.Server(ctx, lanes=lanes, hbm_budget=args.hbm_budget << 30, max_batch=256) as srv:
            tickets = [None] * len(reqs)

            def submitter():
                t0 = time.perf_counter()
                for i, (t, kind, a, b) in enumerate(reqs):
                    dt = t - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                    tickets[i] = srv.submit(kind, a, b)
            th = threading.Thread(target=submitter)
            w0 = time.perf_counter()
            th.start()
            for i in range(len(reqs)):
                while tickets[i] is None:
                    time.sleep(0.0002)
                out[i] = srv.wait(tickets[i])
            th.join()
            wall = time.perf_counter() - w0
            st = srv.stats()
        return out, wall, st

    # the lanes copy the context's configuration: tune it on a sample stream first
    sample = [(a, b) for t, kind, a, b in workloads.serving_stream(count=160, seed=1000 + rank) if kind == "range"]
    tuned, tune_ms = ctx.autotune(sample, gb.GB_TUNE_BATCH, reps=1)
    serve(workloads.serving_stream(count=200, seed=1000 + rank), args.lanes)       # warm-up, arenas
    reqs = workloads.serving_stream(count=args.requests, seed=7 + rank)
    clocks = ClockSampler(local)
    barrier(world, backend_ready)
    clocks.start()
    time.sleep(0.1)
    clocks.mark_start()
    out, wall, st = serve(reqs, args.lanes)
    clocks.mark_end()
    clk = clocks.stop()
    barrier(world, backend_ready)
    bad = [r for r in out if r["status"] != 0]
    first = min(r["t_submit_us"] for r in out)
    last = max(r["t_done_us"] for r in out)
    span_s = (last - first) / 1e6
    span_s = reduce_max(span_s, world, backend_ready)
    n_range = sum((b - a) // 2 for t, kind, a, b in reqs if kind == "range")
    lat = {k: [] for k in ("range", "query")}
    for (t, kind, a, b), r in zip(reqs, out):
        lat[kind].append((r["t_done_us"] - r["t_submit_us"]) / 1000.0)
    allv = sorted(lat["range"] + lat["query"])

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(q * len(v)))] if v else None

    value = n_range * world / span_s
    n_q = sum(1 for r in reqs if r[1] == "query")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 1,
            "ms_per_step": span_s * 1000.0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic", "mode": "serving",
            "config": {"workload": "serving: Poisson stream, 2000 req/s offered, 90% ranges of 2^16..2^30 even n "
                                   "at offsets uniform in [1e9, 4e18], 10% single-n queries (n < 4e18)",
                       "requests": len(reqs), "seed": 7, "lanes": args.lanes, "hbm_budget_gib": args.hbm_budget,
                       "base_primes_to": 1 << 32, "p1": P1, "p2": P2,
                       "offered_n_per_s": n_range / reqs[-1][0]},
            "latency_ms": {"p50": pct(allv, 0.5), "p99": pct(allv, 0.99),
                           "range_p50": pct(lat["range"], 0.5), "range_p99": pct(lat["range"], 0.99),
                           "query_p50": pct(lat["query"], 0.5), "query_p99": pct(lat["query"], 0.99)},
            "roofline": None,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 16 * (len(reqs) - n_q) + 8 * n_q,
                    "d2h_bytes_per_step": 48 * (len(reqs) - n_q) + 4 * n_q},
            "clocks": clk, "gpu_launches": None, "server": st, "failed_requests": len(bad),
            "autotuned": {k: tuned[k] for k in ("tile_bits", "bucket_split", "p1", "cover_prefix")},
            "wall_s": wall, "paper_context": PAPER_CONTEXT}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# ----------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default=DEFAULT_MODE, choices=sorted(PLAIN_MODES) + ["batched", "serving"])
    ap.add_argument("--no-extras", action="store_true",
                    help="default mode: skip the window and batched measurements carried as extra keys")
    ap.add_argument("--extra-steps", type=int, default=10, help="timed steps of each extra workload")
    ap.add_argument("--requests", type=int, default=2000, help="serving: requests in the timed stream")
    ap.add_argument("--lanes", type=int, default=2, help="serving: server lanes")
    ap.add_argument("--hbm-budget", type=int, default=0, help="serving: admission budget, GiB (0: half the free HBM)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true", help="plain family: run gb_autotune on the range first")
    ap.add_argument("--lo", type=int, default=None, help="custom range start (profiling of smaller cases)")
    ap.add_argument("--hi", type=int, default=None, help="custom range end")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.lo is not None and args.hi is not None and args.mode in PLAIN_MODES:
        PLAIN_MODES[args.mode].update(lo=args.lo, hi=args.hi,
                                      workload=f"exhaustive Goldbach verification of every even n in "
                                               f"[{args.lo}, {args.hi})")
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    from paper_2603_02621_gb300 import gb

    torch.cuda.set_device(local)
    backend_ready = False
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        backend_ready = True
    stream = torch.cuda.current_stream()
    if args.mode == "serving":
        return run_serving(args, gb, torch, world, rank, local, backend_ready)
    peaks, peak_src = load_peaks()
    sms = int(torch.cuda.get_device_properties(local).multi_processor_count)
    if args.mode == "batched":
        work = BatchWork(gb, torch, rank, local, stream)
    else:
        work = PlainWork(gb, torch, args.mode, rank, world, local, stream)
        if args.autotune:
            work.autotune()

    # clocks are sampled from the warm-up through the timed and end-to-end regions
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    m = measure(work, gb, torch, stream, args.steps, args.warmup, world, backend_ready, peaks, peak_src, sms,
                clocks)
    clk = clocks.stop()
    check = work.check() if args.mode == "batched" else merged_check(work, world, backend_ready)
    plain_family = args.mode in PLAIN_MODES
    line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
            "higher_is_better": True, "scaling": "strong" if plain_family else "weak",
            "vs_baseline": m["value"] / PAPER_BY_MODE[args.mode] if args.mode in PAPER_BY_MODE else None,
            "dtype": "u64", "data": "synthetic", "mode": args.mode,
            "config": workload_desc(args.mode, world),
            "roofline": m["roofline"], "e2e": m["e2e"], "clocks": clk,
            "gpu_launches": m["gpu_launches"], "sm_count": sms, "kernel_ms": m["kernel_ms"],
            "result_check": check, "paper_context": PAPER_CONTEXT}
    line.update(work.extra())

    # the same line carries the other config-4 window and the batched mode
    if args.mode == DEFAULT_MODE and not args.no_extras:
        xs = max(1, args.extra_steps)
        wwork = PlainWork(gb, torch, "window-4e18", rank, world, local, stream, parent=work.ctx)
        wm = measure(wwork, gb, torch, stream, xs, 3, world, backend_ready, peaks, peak_src, sms)
        line["window_4e18"] = {**{k: wm[k] for k in ("value", "ms_per_step", "steps", "warmup", "e2e", "roofline",
                                                     "gpu_launches", "kernel_ms")},
                               "unit": UNIT, "scaling": "strong", "config": workload_desc("window-4e18", world),
                               "result_check": merged_check(wwork, world, backend_ready)}
        wwork.ctx.close()
        bwork = BatchWork(gb, torch, rank, local, stream)
        bm = measure(bwork, gb, torch, stream, xs, 3, world, backend_ready, peaks, peak_src, sms)
        bx = bwork.extra()
        line["batched"] = {**{k: bm[k] for k in ("value", "ms_per_step", "steps", "warmup", "e2e", "roofline",
                                                 "gpu_launches", "kernel_ms")},
                           "unit": UNIT, "scaling": "weak", "config": workload_desc("batched", world),
                           "result_check": bwork.check(), **bx,
                           "faster_than_plain_loop": bm["value"] > bx["plain_loop"]["value"]}
        bwork.ctx.close()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline(args.mode).items() if k != "seconds"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    work.ctx.close()
    if backend_ready:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def ctypes_ptr(t):
    from paper_2603_02621_gb300 import gb
    return gb.ctypes.cast(gb.ctypes.c_void_p(t.data_ptr()), gb.POINTER(gb.c_uint64))


def ctypes_segs(t):
    from paper_2603_02621_gb300 import gb
    return gb.ctypes.cast(gb.ctypes.c_void_p(t.data_ptr()), gb.POINTER(gb.gb_segment_result))


if __name__ == "__main__":
    sys.exit(main())
