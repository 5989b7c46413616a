"""Benchmark of the Goldbach verifier on the GPU (one JSON line, rank 0).

Modes (--mode), each a workload of GoldbachGPU (arXiv 2603.02621):

* plain (default): exhaustive verification of every even n in [4, 10^10]
  (Table 4's workload): one step = one gb_verify_range call: segment sieve of
  the q window, the loop-inverted cover with P1 = 2^15, the GPU retry pass to
  P2 = 2^20, per-segment reductions (Sec. 2.3);
* exhaustive-1e12: [4, 10^12] (Table 4's largest range), segments of 2^27 even n,
  base primes to 2^31;
* window-4e18: the 10^11-wide window [4e18 - 10^11, 4e18), segments of 2^27;
* batched: 4096 ranges of uneven length (log-uniform 2^10..2^26 even n) and
  offset (uniform in [10^9, 10^15]) in one gb_verify_batch call after the
  autotuner has picked tile, split, P1 and cover prefix; the plain per-range
  launch loop over the same ranges, with the same outputs, is timed beside it.

Multi-GPU (torchrun): each rank verifies its own shard (plain family: the next
range of the same width; batched: its own 4096 ranges) -- independent work, no
collective on the data path (weak scaling); the timing is the max over ranks.

--impl reference times the CPU oracle (oracle/) on a bounded sample of the
same workload, on the host cores.
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
PAPER_NPS = 4999999999 / 23.547     # Table 4: [4, 1e10] in 23,547 ms on an RTX 3070
# the paper's number for the same workload, where it has one (Table 4, RTX 3070)
PAPER_BY_MODE = {"plain": PAPER_NPS, "exhaustive-1e12": 499999999999 / 2457.040}
PAPER_CONTEXT = ("RTX 3070 (8 GB), Table 4: [4, 1e10] in 23,547 ms = 2.12e8 n/s; "
                 "[4, 1e12] in 2,457,040 ms = 2.03e8 n/s")

# plain-family workloads: (first range, shift per rank, segment length, base primes)
PLAIN_MODES = {
    "plain": dict(lo=4, hi=10**10 + 2, shift=10**10, seg=1 << 24, base=None,
                  workload="exhaustive Goldbach verification of every even n in [4, 1e10] per GPU"),
    "exhaustive-1e12": dict(lo=4, hi=10**12 + 2, shift=10**12, seg=1 << 27, base=1 << 31,
                            workload="exhaustive Goldbach verification of every even n in [4, 1e12] per GPU"),
    "window-4e18": dict(lo=4 * 10**18 - 10**11, hi=4 * 10**18, shift=-10**11, seg=1 << 27, base=1 << 31,
                        workload="Goldbach verification of the window [4e18 - 1e11, 4e18) per GPU"),
}


def rank_range(mode: str, rank: int):
    m = PLAIN_MODES[mode]
    return m["lo"] + rank * m["shift"], m["hi"] + rank * m["shift"]


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
    lo, hi = rank_range(mode, 0)
    n = (hi - lo) // 2
    return {"workload": m["workload"], "ranges": [list(rank_range(mode, r)) for r in range(world)],
            "seg_len": m["seg"], "base_primes_to": base_for(mode, hi) if m["base"] else "isqrt(hi)+ (>= 1e5)",
            "p1": P1, "p2": P2,
            "outputs": f"per-segment p_min histogram ({HL} entries), max p_min with n, unresolved",
            "l2": f"q window {n / 8 / 1e6:.0f} MB per GPU > 126 MB L2; no flush needed"}


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
    one by one, in a seeded random order: segments for the plain family,
    ranges for the batched mode."""
    from paper_2603_02621_gb300 import workloads
    if mode == "batched":
        units = workloads.batched_ranges(count=4096, seed=1)
    elif mode == "serving":
        units = [(a, b) for t, kind, a, b in workloads.serving_stream(count=2000, seed=7) if kind == "range"]
    else:
        lo, hi = rank_range(mode, 0)
        seg = PLAIN_MODES[mode]["seg"]
        units = [(a, min(a + 2 * seg, hi)) for a in range(lo, hi, 2 * seg)]
    rng = workloads.SplitMix64(seed)
    order = list(range(len(units)))
    for i in range(len(order) - 1, 0, -1):          # seeded shuffle
        j = rng.below(i + 1)
        order[i], order[j] = order[j], order[i]
    return [units[i] for i in order]


def cpu_baseline(mode: str = "plain", min_seconds: float = 12.0, seed: int = 11):
    """The oracle, as it stands, on a bounded sample of the workload's units
    (one unit per host thread at a time)."""
    from oracle import oracle
    import concurrent.futures as cf
    threads = oracle.default_threads()
    units = sample_units(mode, seed)
    if mode != "plain":
        oracle.primes_upto(3)                           # (cached small primes are built on first use)
        lo_max = max(b for _, b in units)
        oracle.verify_segments(lo_max - 4, lo_max, 2, P2, 8, threads=1)   # warm the prime cache untimed

    def one(u):
        a, b = u
        n = (b - a) // 2
        s, _ = oracle.verify_segments(a, b, n, P2, HL, threads=1)
        return int(s[:, 0].sum())

    done_n, t0, used = 0, time.perf_counter(), 0
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        while time.perf_counter() - t0 < min_seconds and used < len(units):
            batch = units[used:used + threads]
            done_n += sum(ex.map(one, batch))
            used += len(batch)
    dt = time.perf_counter() - t0
    kind = {"batched": "ranges of the 4096-range batch", "serving": "range requests of the serving stream"}.get(
        mode, "segments of %d even n of [%d, %d)" % ((PLAIN_MODES[mode]["seg"],) + tuple(rank_range(mode, 0))))
    return {"value": done_n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "value_per_core": done_n / dt / threads,
            "sample": f"{used} seeded {kind} ({done_n} n, {dt:.1f} s wall, P = 2^20)",
            "seconds": dt}


def roofline_of(prof, wk, alg_cover, steps, mode, peaks, peak_src):
    """Roofline of the dominant kernel from the library's per-kernel profile
    (prof[k]: total ms, launches, work units over the timed region) and work
    counters (wk), as per-launch averages: algorithmic ALU ops per launch over
    the launch's CUDA-event time, against the ALU peak derived from unit
    counts and the clock; DRAM bytes per launch from the ncu capture of the
    plain workload's kernels."""
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # Both hot kernels are bound by the SM's integer ALU pipe (shifts and
    # logic ops; ncu shows it near saturation).  Its peak, from the unit counts
    # and clock: 152 SMs x 64 ALU lanes per cycle (16 per scheduler: half the
    # issue rate, measured by a shift/or loop) x the maximum SM clock.
    alu_peak = 152 * 64 * sm_max * 1e6 / 1e12            # T ALU lane-ops/s
    # DRAM bytes per unit measured by ncu on [4, 2^32] (plain workload's kernels)
    ncu_traffic = {"cover": 0.1270, "sieve": 0.09678} if mode == "plain" else {}
    per = {}
    for kern in ("sieve", "cover", "large"):
        kp = prof[kern]
        if kp["launches"] == 0:
            continue
        nl = kp["launches"]
        ms = kp["ms"] / nl
        if kern == "large":
            # primes above the tile split: 2 ALU ops per strike (word index,
            # rotated mask) issued as a global atomic AND
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
    roofline = {"kernel": kern, "bound": "alu", "achieved": per[kern]["achieved"], "peak": alu_peak,
                "unit": "T ALU lane-ops/s", "frac": per[kern]["frac"],
                "traffic": per[kern]["dram_bytes_per_launch"],
                "peak_source": "derived: 152 SMs x 64 ALU lanes x %.0f MHz (%s max clock)" % (sm_max, peak_src),
                "work": ("cover: 4 ALU ops per (64-n word, odd prime) iteration until the word is full "
                         "(algorithmic count); sieve: 2 per strike + 6 per stamped 32-bit word; "
                         "large primes: 2 per strike"),
                "kernels": per,
                "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6800.0)), "hbm_peak_source": peak_src}

    return roofline


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    per_step = max(4.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(args.mode, min_seconds=1.0)
    vals = []
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(args.mode, min_seconds=per_step)
        vals.append(last["value"])
    value = statistics.mean(vals)
    n_step = workload_n(args.mode)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * n_step / value,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": value / PAPER_BY_MODE[args.mode] if args.mode in PAPER_BY_MODE else None,
            "dtype": "u64", "data": "synthetic", "mode": args.mode, "config": workload_desc(args.mode, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "value_per_core": value / last["cores"], "sample": last["sample"]},
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
    lo, hi = rank_range(mode, rank)
    return (hi - lo) // 2


# ----------------------------------------------------------------------------- workloads on the GPU
class PlainWork:
    """One gb_verify_range call over the rank's range per step."""

    def __init__(self, gb, torch, mode, rank, local, stream):
        self.gb = gb
        self.lo, self.hi = rank_range(mode, rank)
        self.seg = PLAIN_MODES[mode]["seg"]
        self.ctx = gb.Context(device=local, base_limit=base_for(mode, self.hi), seg_len=self.seg,
                              p1=P1, p2=P2, stream=stream.cuda_stream)
        self.nseg = ((self.hi - self.lo) // 2 + self.seg - 1) // self.seg
        self.n = (self.hi - self.lo) // 2
        # device-resident outputs for the device-timed value, pinned host ones for e2e
        self.d_rows = torch.zeros((self.nseg, HL), dtype=torch.int64, device="cuda")
        self.d_segs = torch.zeros((self.nseg, 6), dtype=torch.int64, device="cuda")    # 48-byte records
        self.h_rows = torch.zeros((self.nseg, HL), dtype=torch.int64).pin_memory()
        self.h_segs = torch.zeros((self.nseg, 6), dtype=torch.int64).pin_memory()
        self.h_hist = torch.zeros(HL, dtype=torch.int64).pin_memory()
        self.h2d = 0
        self.d2h = 32 + self.nseg * 48 + self.nseg * HL * 8 + HL * 8
        self.last = None
        self.tuned = None

    def autotune(self, torch):
        """gb_autotune on the rank's own range (plain mode), before timing."""
        cfg, ms = self.ctx.autotune([(self.lo, self.hi)], self.gb.GB_TUNE_PLAIN, reps=1)
        # per-segment outputs follow seg_len: keep the workload's
        self.ctx.set_config(seg_len=self.seg)
        self.tuned = ({k: cfg[k] for k in ("tile_bits", "bucket_split", "cta_threads", "p1", "cover_prefix")},
                      ms)

    def _call(self, rows, segs, hist):
        gb = self.gb
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

    def check(self):
        r = self.last
        return {"unresolved": int(r.unresolved), "max_pmin": int(r.max_pmin),
                "max_pmin_n": int(r.max_pmin_n), "n_checked": int(r.n_checked)}

    def algorithmic_cover_iterations(self):
        """The cover's algorithmic work for one step (untimed): the generic
        cover (cover_prefix 1) counts, per 64-n word, the odd primes applied
        until the word is full -- equal to the oracle's count from the p_min
        values (tests/test_gpu_work.py)."""
        gb = self.gb
        saved = self.ctx.config()["cover_prefix"]
        self.ctx.set_config(cover_prefix=1)
        gb.gb_profile_enable(self.ctx.handle, True)
        self.step_device()
        iters = gb.gb_profile_work(self.ctx.handle)["cover_iterations"]
        gb.gb_profile_enable(self.ctx.handle, False)
        self.ctx.set_config(cover_prefix=saved)
        return iters

    def extra(self, args):
        if self.tuned is None:
            return {}
        return {"autotuned": self.tuned[0], "autotune_best_ms": self.tuned[1]}


class BatchWork:
    """One gb_verify_batch call over the rank's 4096 ranges per step."""

    def __init__(self, gb, torch, mode, rank, local, stream):
        from paper_2603_02621_gb300 import workloads
        self.gb, self.torch = gb, torch
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
        self.h2d = 0                       # the range list is host memory the call reads (count x 16 B)
        self.d2h = self.count * 48 + self.count * HL * 8
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

    def extra(self, args):
        """The plain per-range launch loop over the same ranges, same outputs
        (per-range totals and histogram row, device-resident), timed once after
        one warm-up pass; and the batch without its CUDA graph."""
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
        t0 = time.perf_counter()
        loop()
        torch.cuda.synchronize()
        loop_s = time.perf_counter() - t0
        same = bool(torch.equal(d_hist, self.d_rows))
        return {"plain_loop": {"value": self.n / loop_s, "unit": UNIT, "ms": 1000.0 * loop_s,
                               "launch": "gb_verify_range per range, same per-range histograms",
                               "same_histograms": same},
                "autotuned": {k: self.tuned[k] for k in ("tile_bits", "bucket_split", "p1", "cover_prefix")},
                "autotune_best_ms": self.tune_ms}


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
    ap.add_argument("--mode", default="plain", choices=sorted(PLAIN_MODES) + ["batched", "serving"])
    ap.add_argument("--requests", type=int, default=2000, help="serving: requests in the timed stream")
    ap.add_argument("--lanes", type=int, default=2, help="serving: server lanes")
    ap.add_argument("--hbm-budget", type=int, default=0, help="serving: admission budget, GiB (0: half the free HBM)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true", help="plain family: run gb_autotune on the range first")
    ap.add_argument("--lo", type=int, default=None, help="custom range start (profiling of smaller cases)")
    ap.add_argument("--hi", type=int, default=None, help="custom range end")
    args = ap.parse_args()
    world, rank, local = dist_setup()
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
    if args.mode == "batched":
        work = BatchWork(gb, torch, args.mode, rank, local, stream)
    else:
        if args.lo is not None and args.hi is not None:
            PLAIN_MODES[args.mode].update(lo=args.lo, hi=args.hi, shift=args.hi - args.lo)
        work = PlainWork(gb, torch, args.mode, rank, local, stream)
        if args.autotune:
            work.autotune(torch)
    ctx = work.ctx

    alg_cover = work.algorithmic_cover_iterations() if isinstance(work, PlainWork) else None
    torch.cuda.synchronize()
    # clocks are sampled from the warm-up through the timed and end-to-end regions
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    for _ in range(args.warmup):
        work.step_device()
    torch.cuda.synchronize()

    # ---- device-timed region (value), per-kernel events
    gb.gb_profile_enable(ctx.handle, True)
    barrier(world, backend_ready)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark_start()
    ev0.record(stream)
    for _ in range(args.steps):
        work.step_device()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world, backend_ready)
    dev_ms = ev0.elapsed_time(ev1)
    prof = gb.gb_profile_read(ctx.handle)
    wk = gb.gb_profile_work(ctx.handle)
    launches = gb.gb_profile_kernels(ctx.handle)
    gb.gb_profile_enable(ctx.handle, False)
    max_ms = reduce_max(dev_ms, world, backend_ready)

    # ---- end-to-end region through the public call with pinned host buffers
    barrier(world, backend_ready)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        work.step_host()
    torch.cuda.synchronize()
    e2e_ms = 1000.0 * (time.perf_counter() - t0)
    clocks.mark_end()
    clk = clocks.stop()
    e2e_ms = reduce_max(e2e_ms, world, backend_ready)

    total_n = work.n * args.steps * world
    value = total_n / (max_ms / 1000.0)
    e2e_value = total_n / (e2e_ms / 1000.0)

    # ---- roofline of the dominant kernel (per-launch averages over the timed region)
    peaks, peak_src = load_peaks()
    roofline = roofline_of(prof, wk, alg_cover, args.steps, args.mode, peaks, peak_src)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": value / PAPER_BY_MODE[args.mode] if args.mode in PAPER_BY_MODE else None,
            "dtype": "u64", "data": "synthetic", "mode": args.mode,
            "config": workload_desc(args.mode, world),
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": work.h2d,
                    "d2h_bytes_per_step": work.d2h},
            "clocks": clk,
            "gpu_launches": int(launches),
            "kernel_ms": {k: prof[k]["ms"] for k in prof},
            "result_check": work.check(),
            "paper_context": PAPER_CONTEXT}
    line.update(work.extra(args))
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline(args.mode).items() if k != "seconds"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
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
