"""The bench's JSON line (reference arm, CPU only): the keys and types the
driver reads, the oracle as the reference, and the workload description."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_line():
    """The default workload ([4, 1e12], segments of 2^27 even n): each step
    one seeded segment per host thread; ms_per_step is the wall time the arm
    spent per step."""
    d = _line("--impl", "reference", "--steps", "1", "--warmup", "0")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "even integers verified/sec" and d["unit"] == "even n/s"
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1 and d["higher_is_better"] is True
    assert d["scaling"] == "strong" and d["data"] == "synthetic" and d["dtype"] == "u64"
    assert d["config"]["workload"] == "exhaustive Goldbach verification of every even n in [4, 1e12]"
    assert d["config"]["seg_len"] == 1 << 27 and d["config"]["base_primes_to"] == 1 << 31
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "sample" in cb
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert abs(d["vs_baseline"] - d["value"] / (499999999999 / 2457.040)) < 1e-6 * d["vs_baseline"]
    # the step is what the arm verified: one whole segment per host thread
    assert d["n_per_step"] == cb["cores"] * (1 << 27)
    assert abs(d["ms_per_step"] - 1000.0 * d["n_per_step"] / d["value"]) < 1e-6 * d["ms_per_step"]


def test_reference_arm_rank_nonzero_is_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert out.returncode == 0 and not [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_clock_sampler_takes_the_timed_window():
    """Clock samples are stamped on arrival; the reported SM clock and the
    throttle reasons come from the samples inside the marked timed region,
    and from the samples under load when the region caught none."""
    sys.path.insert(0, ROOT)
    import bench
    row = "{clk}, 2070, 900.0, Not Active, Not Active, Not Active, {cap}, {util}"
    c = bench.ClockSampler(0)
    c.lines = [(1.0, row.format(clk=1200, cap="Not Active", util=0)),
               (2.0, row.format(clk=2070, cap="Active", util=100)),
               (2.1, row.format(clk=2040, cap="Not Active", util=100)),
               (3.0, row.format(clk=1500, cap="Not Active", util=90))]
    c.t_start, c.t_end = 1.95, 2.06
    r = c.stop()
    assert r["samples"] == 4 and r["samples_in_timed_region"] == 2 and r["samples_under_load"] == 3
    assert r["sm_mhz"] == (2070 + 2040) / 2 and r["sm_max_mhz"] == 2070 and r["reasons"] == ["sw_power_cap"]
    c.t_start, c.t_end = 2.5, 2.6                       # a region too short to catch a sample
    r = c.stop()
    assert r["samples_in_timed_region"] == 0 and r["sm_mhz"] == 2040


def test_roofline_arithmetic():
    """The roofline of the bench line, from a synthetic profile: the dominant
    kernel by total time; achieved = algorithmic ALU ops per launch over the
    launch's time; frac = achieved / (SMs x 64 lanes x clock); traffic =
    the ncu bytes per unit times the units of one launch (workloads with a
    capture of the current kernels only)."""
    sys.path.insert(0, ROOT)
    import bench
    steps, nl = 10, 10
    prof = {"sieve": {"ms": 19.0, "launches": nl, "units": 6.25e10},      # q bits over the timed region
            "cover": {"ms": 23.3, "launches": nl, "units": 5.0e10},       # even n
            "large": {"ms": 0.0, "launches": 0, "units": 0.0}}
    wk = {"sieve_strikes": 5.3e10, "cover_iterations": 9.0e10, "large_strikes": 0.0}
    alg_cover = 3.9e9                                                       # per step
    peaks = {"sm_max_mhz": 2070.0, "hbm_gbs": 6695.5}
    sms = 152
    r = bench.roofline_of(prof, wk, alg_cover, steps, "exhaustive-1e12", peaks, "measured", sms)
    peak = sms * 64 * 2070e6 / 1e12
    assert r["kernel"] == "cover" and r["bound"] == "alu" and abs(r["peak"] - peak) < 1e-9
    ops = 4.0 * alg_cover * steps / nl
    achieved = ops / (23.3 / nl / 1000.0) / 1e12
    assert abs(r["achieved"] - achieved) < 1e-9 * achieved and abs(r["frac"] - achieved / peak) < 1e-12
    assert abs(r["traffic"] - bench.NCU_TRAFFIC["exhaustive-1e12"]["cover"] * 5.0e10 / nl) < 1e-3
    assert bench.roofline_of(prof, wk, alg_cover, steps, "plain", peaks, "measured", sms)["traffic"] is None
    s = r["kernels"]["sieve"]
    assert abs(s["alu_ops_per_launch"] - (2.0 * 5.3e10 / nl + 6.0 * 6.25e10 / nl / 32.0)) < 1.0
    assert abs(s["algorithmic_bytes_per_launch"] - 6.25e10 / nl / 8.0) < 1e-6
    assert "large" not in r["kernels"]
    # other workloads: the block cover's own steps, no ncu traffic
    r2 = bench.roofline_of(prof, wk, None, steps, "batched", peaks, "measured", sms)
    assert r2["traffic"] is None and abs(r2["kernels"]["cover"]["alu_ops_per_launch"] - 2.0 * 9.0e10 / nl) < 1.0


def _bench_rank(rank, world, port, q):
    """One gloo rank of the bench's strong-scaling host logic: its share of
    the range (bench.rank_range), verified by the oracle in place of the GPU
    call, and the merge of every rank's totals (bench.merged_check)."""
    import datetime
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        bench.PLAIN_MODES["plain"].update(lo=10**9, hi=10**9 + 2 * 50000, seg=4096)
        a, b = bench.rank_range("plain", rank, world)

        class Work:
            def totals(self):
                summ, hist = oracle.verify_segments(a, b, max(1, (b - a) // 2), bench.P2, bench.HL, threads=1)
                return {"n_checked": int(summ[:, 0].sum()), "unresolved": int(summ[:, 1].sum()),
                        "max_pmin": int(summ[0, 2]), "max_pmin_n": int(summ[0, 3]), "hist": hist[0]}
        q.put((rank, a, b, bench.merged_check(Work(), world, True)))
    finally:
        dist.destroy_process_group()


def test_strong_scaling_shards_and_merges_on_two_gloo_ranks():
    import multiprocessing as mp
    import socket
    sys.path.insert(0, ROOT)
    from oracle import oracle
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_bench_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    lo, hi = 10**9, 10**9 + 2 * 50000
    # contiguous whole-segment shares covering the range
    assert res[0][1] == lo and res[0][2] == res[1][1] and res[1][2] == hi and (res[1][1] - lo) % (2 * 4096) == 0
    summ, _ = oracle.verify_segments(lo, hi, (hi - lo) // 2, 1 << 20, 3512, threads=2)
    whole = {"n_checked": int(summ[0, 0]), "unresolved": int(summ[0, 1]), "max_pmin": int(summ[0, 2]),
             "max_pmin_n": int(summ[0, 3])}
    assert res[0][3] == whole and res[1][3] == whole
