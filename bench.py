"""Benchmark of the modulo-primes sieve on GB300 (one JSON line on rank 0).

Workload (N=1): the triangle 1 <= q < p <= 2^14 (81,599,337 coprime pairs) with the
first 64 odd primes, one range per launch (the plain form); synthetic, seeded inputs
(the ranges and prime lists of the workloads module).  A step is one pass of the hot
path over it: tile planning, the sieve with early exit and per-prime counts, survivor
compaction and the exact root test of the survivors.  The tables (built once by the
device table builder, timed separately) are resident inputs.  L2 is flushed (a 256 MiB
write) before every timed step.

Extra objects in the same line: the batched form against the plain form on the 4096
rectangles of the batched workload, the large 2^20 triangle sweep, the roofline of the
dominant kernel, the end-to-end number through the C ABI with host buffers, the oracle
timed on the host cores, and the SM clocks sampled during the timed region.

--impl reference times the oracle (the CPU restatement) on the same workload.
Multi-GPU (torchrun): every rank runs the same workload on its own GPU (replicas, weak
scaling); value = all ranks' pairs / max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "sieved coprime (p,q) pairs/s"
UNIT = "pairs/s"
# lane-ops of one prime test of one 64-value word: residue (2), address (1), three table
# loads (3), two funnel shifts (2), two ANDs (2), two popcounts (2), count add (1), two
# alive updates (2)
OPS_PER_WORD_STEP = 15


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the batched/large/e2e/cpu legs")
    ap.add_argument("--workload", default="c2", choices=["c2", "c4top"],
                    help="c2: the 2^14 triangle (the headline); c4top: the 4097 largest rows of the "
                         "2^20 triangle with 256 primes (the long-row regime, for profiling)")
    ap.add_argument("--wide-only", action="store_true",
                    help="run only the 64-bit range leg and print its JSON (for profiling)")
    ap.add_argument("--root-only", action="store_true",
                    help="run only the bulk root-test leg and print its JSON (for profiling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks sampler

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def profile_record(kernel_src: str, workload: str) -> dict:
    """The committed ncu record of the sieve kernel for this workload (DRAM bytes, warp
    instructions and issue-slot utilisation per launch), or {} when the kernel source
    changed since the capture."""
    path = os.path.join(ROOT, "profiles", "sieve_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return {}
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
    entry = rec.get(workload)
    if not entry or entry.get("sieve_cu_sha256") != sha:
        return {}
    return entry


def traffic_record(kernel_src: str, workload: str):
    """DRAM bytes per launch of the sieve kernel from a committed ncu summary, or None
    when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "sieve_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
    entry = rec.get(workload)
    if not entry or entry.get("sieve_cu_sha256") != sha:
        return None
    return entry.get("dram_bytes_per_launch")


def _tune_cache():
    """Autotuner results persist per user (device name, primes, ranges and mode are the key)."""
    d = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    try:
        os.makedirs(d, exist_ok=True)
    except OSError:
        return None
    return os.path.join(d, "cuboid_autotune.txt")


_ORACLE_TABLES = {}


def int_issue_probe(cb, torch, stream):
    """Measured 32-bit integer issue rate (lane-ops/s) of a dependency-free add/shift/xor
    stream on every SM, and the rate of the sieve's lookup mix (shared-memory load pair,
    funnel shift, and, popc, xor)."""
    sms = cb.cuboid_device_sms()
    blocks, threads, iters = sms * 8, 256, 4096
    sink = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    out = {}
    for kind, ops in ((0, 48), (1, 16 * 6)):
        for _ in range(2):
            cb.cuboid_probe_int_issue(kind, blocks, threads, iters, sink.data_ptr(), stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            cb.cuboid_probe_int_issue(kind, blocks, threads, iters, sink.data_ptr(), stream)
            b.record(stream)
        stream.synchronize()
        sec = a.elapsed_time(b) / 1e3
        out["alu_tops" if kind == 0 else "lookup_mix_tops"] = blocks * threads * iters * ops / sec / 1e12
    return out


def cpu_baseline(target_s: float = 12.0, seed: int = W.DEFAULT_SEED) -> dict:
    """The oracle as it stands, on a seeded sample of rows of the same workload."""
    import numpy as np

    import oracle as O
    cfg = W.c2()
    t0 = time.perf_counter()
    if "c2" not in _ORACLE_TABLES:
        _ORACLE_TABLES["c2"] = O.Tables(cfg["primes"], full_limit=0)
    T = _ORACLE_TABLES["c2"]
    build_s = time.perf_counter() - t0
    g = W.rng(seed)
    rows = g.permutation(np.arange(2, (1 << 14) + 1))
    pairs = 0
    t0 = time.perf_counter()
    done = 0
    for p in rows:
        n, _, _ = O.sieve_range(T, W.rect(int(p), int(p), 1, int(p) - 1, q_lt_p=True))
        pairs += n
        done += 1
        if time.perf_counter() - t0 > target_s:
            break
    dt = time.perf_counter() - t0
    return {"value": pairs / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} seeded random rows p of the 2^14 triangle ({pairs} pairs, {dt:.1f} s; "
                      f"tables built once in {build_s:.1f} s, not timed)"}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps = []
    for i in range(args.warmup):
        cpu_baseline(target_s=1.0, seed=W.DEFAULT_SEED + 1000 + i)
    per = min(10.0, max(2.0, 60.0 / max(args.steps, 1)))
    wall = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        steps.append(cpu_baseline(target_s=per, seed=W.DEFAULT_SEED + i))
        wall.append(time.perf_counter() - t0)
    v = sum(s["value"] for s in steps) / len(steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(wall) / len(wall),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": W.c2()["name"], "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": steps[-1]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    import paper_1601_00636_gb300 as cb

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    cfg = W.c2()
    if args.workload == "c4top":
        cfg = {"name": "c4top_rows2^20-4096..2^20_256primes", "primes": W.first_odd_primes(256),
               "ranges": [W.rect((1 << 20) - 4096, 1 << 20, 1, (1 << 20) - 1, q_lt_p=True)]}
    primes = cfg["primes"]
    rng = cfg["ranges"][0]
    n_primes = len(primes)
    whole_max = 1 << 14
    if world > 1 and args.workload == "c2":
        # weak scaling: the triangle grows with N (about N times the pairs of the 2^14
        # triangle) and each rank sieves one balanced shard of it
        import math
        whole_max = int(round((1 << 14) * math.sqrt(world)))
        rng, _ = cb.cuboid_shard_range(W.triangle(whole_max), world, rank)

    # table build (timed separately, once)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t = cb.cuboid_tables_build(primes, cb.ORDER_BY_RATE, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    table_ms = e0.elapsed_time(e1)

    # kernel shape picked by the autotuner on this very workload (outside the timed region)
    tune, tune_ms = cb.cuboid_autotune(t, [rng], cb.MODE_PLAIN, stream, _tune_cache())
    res = cb.cuboid_result_create(t, 1)
    arr = cb.ranges_array([rng])
    dev_ranges = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to("cuda")

    def step(mode=cb.MODE_PLAIN):
        cb.cuboid_sieve_device(res, dev_ranges.data_ptr(), 1, mode, stream)

    # parity of the timed configuration against the stored oracle result
    with open(os.path.join(ROOT, "tests", "golden", "c2_by_rate.json")) as f:
        gold = json.load(f)["results"][0]
    step()
    cb.cuboid_result_download(res, stream)
    assert cb.cuboid_result_wait(res) == cb.OK
    got = cb.cuboid_result_get(res, 0, n_primes)
    n_pairs = got["n_pairs"]
    if args.workload == "c4top":
        # every pair accounted for, and the pair total equals the sum of phi(p) over the rows
        import numpy as np
        hi = 1 << 20
        phi = np.arange(hi + 1, dtype=np.int64)
        for i in range(2, hi + 1):
            if phi[i] == i:
                phi[i::i] -= phi[i::i] // i
        bit_exact = (sum(got["counts"]) + len(got["survivors"]) == n_pairs
                     and n_pairs == int(phi[hi - 4096:hi + 1].sum()))
        n_total = n_pairs * world  # replicas of the same rows on every rank
    elif world == 1:
        bit_exact = (got["n_pairs"] == gold["n_pairs"] and got["counts"] == gold["counts"]
                     and [list(x) for x in got["survivors"]] == gold["survivors"]
                     and [list(x) for x in got["roots"]] == gold["roots"])
    else:
        # shards: every pair accounted for here, and the pair totals of all ranks add up to
        # sum phi(p) over the whole triangle (checked on rank 0)
        tot = torch.tensor([n_pairs], dtype=torch.int64, device="cuda")
        dist.all_reduce(tot)
        bit_exact = sum(got["counts"]) + len(got["survivors"]) == n_pairs
        if rank == 0:
            import numpy as np
            phi = np.arange(whole_max + 1, dtype=np.int64)
            for i in range(2, whole_max + 1):
                if phi[i] == i:
                    phi[i::i] -= phi[i::i] // i
            bit_exact = bit_exact and int(tot.item()) == int(phi[2:].sum())
        n_total = int(tot.item())

    # algorithmic work per launch (instrumented run, outside the timed region)
    cb.cuboid_sieve_device(res, dev_ranges.data_ptr(), 1, cb.MODE_PLAIN | cb.MODE_COUNT_STEPS, stream)
    cb.cuboid_result_wait(res)
    stats = cb.cuboid_result_stats(res)

    clocks = Clocks(dev)
    clocks.start()
    time.sleep(0.3)
    # bring the clocks up after the idle sampler start: ~40 ms of the L2-flush fill (not a
    # step), then the warm-up steps, then the timed steps with no idle gap
    with torch.cuda.stream(stream):
        for _ in range(600):
            flush.zero_()
    for _ in range(args.warmup):
        step()
    barrier()
    evs = []
    sieve_ms, sieve_launches = 0.0, 0
    torch.cuda.nvtx.range_push("timed")  # profilers capture only this region
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
            a.record(stream)
            step(cb.MODE_PLAIN)
            b.record(stream)
        evs.append((a, b))
    stream.synchronize()
    # the sieve kernel's own launch time, on the same steps with events around the sieve
    # launch (those events hold the sieve back from overlapping the plan kernel, so this
    # pass is timed apart from the steps above)
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            step(cb.MODE_PLAIN | cb.MODE_TIME_SIEVE)
        stream.synchronize()
        ms, nl = cb.cuboid_result_sieve_ms(res) if cb.cuboid_result_wait(res) == cb.OK else (0.0, 0)
        sieve_ms += ms
        sieve_launches += nl
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    t_max = torch.tensor([total_ms], device="cuda")
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    total_s = float(t_max.item()) / 1e3
    job_pairs = n_pairs if world == 1 else n_total
    value = job_pairs * args.steps / total_s

    # roofline of the dominant kernel (the sieve)
    pk = peaks()
    sms = cb.cuboid_device_sms()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    alu_peak = sms * 128 * sm_max * 1e6 / 1e12          # Tops/s: 32-bit integer lanes x clock
    per_launch_ms = sieve_ms / max(sieve_launches, 1)
    alg_ops = stats["word_steps"] * OPS_PER_WORD_STEP
    achieved = alg_ops / (per_launch_ms / 1e3) / 1e12
    traffic = traffic_record(os.path.join(ROOT, "paper_1601_00636_gb300", "csrc", "sieve.cu"), cfg["name"])
    probe = int_issue_probe(cb, torch, stream)
    prof = profile_record(os.path.join(ROOT, "paper_1601_00636_gb300", "csrc", "sieve.cu"), cfg["name"])
    executed = None
    if prof.get("inst_executed_per_launch"):
        # every warp instruction the kernel issues, as lane-ops, over the live launch time
        ex = prof["inst_executed_per_launch"] * 32 / (per_launch_ms / 1e3) / 1e12
        executed = {"tops": ex, "frac": ex / alu_peak, "issue_active_pct_ncu": prof.get("issue_active_pct"),
                    "note": "warp instructions per launch from the committed ncu record x 32 lanes / live launch time"}
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                "frac": achieved / alu_peak, "traffic": traffic, "probe": probe, "executed": executed,
                "kernel": "k_sieve", "launch_ms": per_launch_ms,
                "peak_note": f"{sms} SMs x 128 int32 lanes x {sm_max:.0f} MHz (sm_max_mhz of measured)",
                "work": {"word_steps": stats["word_steps"], "words": stats["words"],
                         "warp_steps": stats["warp_steps"], "ops_per_word_step": OPS_PER_WORD_STEP}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": cfg["name"] if world == 1 else f"triangle 1<=q<p<={whole_max}, 64 primes, {world} shards",
                       "pairs_per_step": job_pairs, "primes": n_primes,
                       "order": "rejection rate (CUBOID_ORDER_BY_RATE)",
                       "form": "plain (one range per launch)", "l2": "flushed (256 MiB write) before each step",
                       "parallelism": f"range shards x{world} (no data-path collective)"},
            "bit_exact": bit_exact, "table_build_ms": table_ms, "tuning": tune,
            "roofline": roofline, "clocks": clk, "gpu_launches": 2 * args.steps,
            "gpu_launches_note": "sieve + root test per timed step (a single range needs no plan kernel); the sieve-timing pass adds as many"}

    if not args.no_extras and rank == 0:
        line["e2e"] = e2e_leg(cb, torch, primes, rng, args)
        line["forms"] = forms_leg(cb, torch, stream, flush)
        line["serving"] = serving_leg(cb, torch, stream)
        line["region_section6"] = region_leg(cb, torch, stream)
        line["wide_64bit"] = wide_leg(cb, torch, stream)
        line["deep_primes"] = deep_leg(cb, torch, stream)
        line["root_test"] = root_test_leg(cb, torch, stream)
        line["cpu_baseline"] = cpu_baseline()
    elif rank == 0:
        line["e2e"] = None

    cb.cuboid_result_free(res)
    cb.cuboid_tables_free(t)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def e2e_leg(cb, torch, primes, rng, args):
    """Through the C ABI from host buffers.  Steady state (the headline): tables built once,
    then every step copies the range from pinned host memory, sieves it, runs the root
    test and reads counts, survivor and root records back (cuboid_sieve_into + wait +
    get on a reused result).  Cold: every step also builds the tables from the host prime
    list and allocates and frees the result (cuboid_tables_build + cuboid_sieve)."""
    s = torch.cuda.Stream()
    k = max(5, min(args.steps, 20))
    t = cb.cuboid_tables_build(primes, cb.ORDER_BY_RATE, s)
    cb.cuboid_autotune(t, [rng], cb.MODE_PLAIN, s, _tune_cache())
    res = cb.cuboid_result_create(t, 1)
    arr = cb.ranges_array([rng])
    times, n_pairs = [], 0
    for i in range(k + 3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cb.cuboid_sieve_into(res, None, cb.MODE_PLAIN, s, arr=arr)
        cb.cuboid_result_wait(res)
        got = cb.cuboid_result_get(res, 0, len(primes))
        dt = time.perf_counter() - t0
        n_pairs = got["n_pairs"]
        if i >= 3:
            times.append(dt)
    cb.cuboid_result_free(res)
    cb.cuboid_tables_free(t)
    times.sort()
    per = times[len(times) // 2]
    cold = []
    for i in range(7):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t = cb.cuboid_tables_build(primes, cb.ORDER_BY_RATE, s)
        r2 = cb.cuboid_sieve(t, rng["p_lo"], rng["p_hi"], rng["q_lo"], rng["q_hi"], cb.Q_LT_P, s)
        cb.cuboid_result_wait(r2)
        cb.cuboid_result_get(r2, 0, len(primes))
        cb.cuboid_result_free(r2)
        cb.cuboid_tables_free(t)
        if i >= 2:
            cold.append(time.perf_counter() - t0)
    cold.sort()
    h2d = 24  # the range, passed to the plan kernel as an argument
    d2h = 128 + 8 + 8 * len(primes)  # one copy: device header (padded), pair total, counts
    return {"value": n_pairs / per, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": per * 1e3, "steps": k,
            "includes": "host range -> device (kernel argument), plan + sieve + root test, header/counts -> host in one copy (survivor and root records when present)",
            "cold": {"value": n_pairs / cold[len(cold) // 2], "ms_per_step": 1e3 * cold[len(cold) // 2],
                     "h2d_bytes_per_step": h2d + 4 * len(primes),
                     "includes": "also table build from the host prime list and result allocation/free"}}


def serving_leg(cb, torch, stream, rates=(1e2, 3e2, 1e3, 3e3, 1e4), seconds=2.0, max_queries=4000):
    """Poisson streams of range queries (area 2^U(10,26), p, q < 2^24, 128 primes) served
    by the continuous-batching loop: latency = submit to result ready, per query."""
    import random
    c5 = W.c5()
    t = cb.cuboid_tables_build(c5["primes"], cb.ORDER_BY_RATE, stream)
    srv = cb.cuboid_server_create(t, 0, 4096)
    out = {"primes": len(c5["primes"]), "seconds_per_rate": seconds, "rates": []}
    check = []
    try:
        for ri, rate in enumerate(rates):
            n = int(min(max_queries, rate * seconds))
            qs = W.poisson_queries(rate, n, seed=W.DEFAULT_SEED + ri)
            arr = [cb.range_from_dict(q) for q in qs]
            sub, lat, pairs = {}, [], 0
            i = 0
            refused = 0
            t0 = time.perf_counter()
            while i < n or sub:
                now = time.perf_counter() - t0
                while i < n and qs[i]["t"] <= now:
                    tk = cb.cuboid_server_submit(srv, arr[i])
                    if tk is None:          # admission refused: retry on the next turn
                        refused += 1
                        break
                    sub[tk] = (i, time.perf_counter())
                    i += 1
                for tk in list(sub):
                    res = cb.cuboid_server_poll(srv, tk)
                    if res is None:
                        continue
                    qi, ts = sub.pop(tk)
                    lat.append(time.perf_counter() - ts)
                    cb.cuboid_result_wait(res)
                    got = cb.cuboid_result_get(res, 0, len(c5["primes"]))
                    pairs += got["n_pairs"]
                    if random.Random(qi * 7919 + ri).random() < 0.01:
                        check.append((qs[qi], got["counts"], got["n_pairs"]))
                    cb.cuboid_result_free(res)
                if not sub and i < n:
                    time.sleep(max(0.0, min(0.0005, qs[i]["t"] - (time.perf_counter() - t0))))
            wall = time.perf_counter() - t0
            lat.sort()
            out["rates"].append({"rate_per_s": rate, "queries": n, "pairs": pairs, "wall_s": wall,
                                 "pairs_per_s": pairs / wall, "p50_ms": 1e3 * lat[len(lat) // 2],
                                 "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                                 "refused_retries": refused})
        st = cb.cuboid_server_stats(srv)
        out["server"] = st
    finally:
        cb.cuboid_server_destroy(srv, 120000)
    # mix vs alone on the seeded 1 % sample
    same = True
    for q, counts, npairs in check:
        r = cb.cuboid_sieve(t, q["p_lo"], q["p_hi"], q["q_lo"], q["q_hi"], 0, stream)
        cb.cuboid_result_wait(r)
        g = cb.cuboid_result_get(r, 0, len(c5["primes"]))
        cb.cuboid_result_free(r)
        same &= g["counts"] == counts and g["n_pairs"] == npairs
    out["mix_equals_alone"] = {"checked": len(check), "equal": same}
    cb.cuboid_tables_free(t)
    return out


def forms_leg(cb, torch, stream, flush):
    """Plain (one launch sequence per range) vs batched (one persistent launch from a CUDA
    graph) on the 4096 rectangles of the batched workload, and the large 2^20 sweep."""
    out = {}
    c3 = W.c3()
    t = cb.cuboid_tables_build(c3["primes"], cb.ORDER_BY_RATE, stream)
    tune3, _ = cb.cuboid_autotune(t, c3["ranges"], cb.MODE_BATCHED, stream, _tune_cache())
    res = cb.cuboid_result_create(t, len(c3["ranges"]))
    arr = cb.ranges_array(c3["ranges"])
    dev = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to("cuda")
    n = len(c3["ranges"])

    def timed(mode, reps, np_):
        for _ in range(2):
            cb.cuboid_sieve_device(res, dev.data_ptr(), n, mode, stream)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.zero_()
                a.record(stream)
                cb.cuboid_sieve_device(res, dev.data_ptr(), n, mode, stream)
                b.record(stream)
            stream.synchronize()
            tot += a.elapsed_time(b)
        cb.cuboid_result_download(res, stream)
        cb.cuboid_result_wait(res)
        pairs = sum(cb.cuboid_result_get(res, i, np_)["n_pairs"] for i in range(n))
        return pairs, tot / reps

    pairs, ms_b = timed(cb.MODE_BATCHED, 5, 128)
    counts_b = [cb.cuboid_result_get(res, i, 128)["counts"] for i in range(0, n, 97)]
    _, ms_p = timed(cb.MODE_PLAIN, 2, 128)
    counts_p = [cb.cuboid_result_get(res, i, 128)["counts"] for i in range(0, n, 97)]
    out["c3_4096_rectangles"] = {"pairs": pairs, "batched_ms": ms_b, "plain_ms": ms_p, "tuning": tune3,
                                 "batched_pairs_per_s": pairs / (ms_b / 1e3),
                                 "plain_pairs_per_s": pairs / (ms_p / 1e3),
                                 "batched_equals_plain": counts_b == counts_p}
    cb.cuboid_result_free(res)
    cb.cuboid_tables_free(t)

    c4 = W.c4()
    t = cb.cuboid_tables_build(c4["primes"], cb.ORDER_BY_RATE, stream)
    # tuned on the 4097 longest rows (the full sweep takes ~60 ms a pass)
    sub = [W.rect((1 << 20) - 4096, 1 << 20, 1, (1 << 20) - 1, q_lt_p=True)]
    tune4, _ = cb.cuboid_autotune(t, sub, cb.MODE_BATCHED, stream, _tune_cache())
    res = cb.cuboid_result_create(t, 1)
    arr = cb.ranges_array(c4["ranges"])
    dev = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to("cuda")
    n = 1
    pairs, ms = timed(cb.MODE_BATCHED, 3, 256)
    out["c4_triangle_2^20"] = {"pairs": pairs, "ms": ms, "pairs_per_s": pairs / (ms / 1e3), "tuning": tune4}
    cb.cuboid_result_free(res)
    cb.cuboid_tables_free(t)
    return out


def region_leg(cb, torch, stream, p_to=154000):
    """The search of section 5 over the rows p = 1..154000 of Eq. 1.2 with the 96 primes
    11..541 in ascending order (the run of section 6), through cuboid_region_scan: wall
    clock, pairs/s, survivors and the deepest prime needed."""
    primes = W.primes_between(11, 541)
    t = cb.cuboid_tables_build(primes, cb.ORDER_AS_GIVEN, stream)
    cb.cuboid_region_scan(t, 1, 2000, stream=stream)          # warm-up (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, rep, counts, surv, roots = cb.cuboid_region_scan(t, 1, p_to, stream=stream)
    wall = time.perf_counter() - t0
    cb.cuboid_tables_free(t)
    return {"rows": [1, p_to], "primes": "11..541 (96, ascending)", "status": st, "pairs": rep["pairs"],
            "wall_s": wall, "pairs_per_s": rep["pairs"] / wall, "n_surv": rep["n_surv"],
            "depth": rep["depth"], "r_max": rep["r_max"],
            "paper": "4130 min on its machine for the same rows (section 6; context only)"}


def root_test_leg(cb, torch, stream, n_max=1024, reps=3):
    """The exact root test in bulk: the tables of 3, 5 and 7 are all zero (section 2), so
    every coprime pair of the triangle 1 <= q < p <= 1024 survives the sieve and goes
    through the root test.  CUDA events around the whole run (sieve, root test, copies)
    and around the sieve launch alone (CUBOID_MODE_TIME_SIEVE); the root test's share is
    the difference."""
    t = cb.cuboid_tables_build([3, 5, 7], cb.ORDER_AS_GIVEN, stream)
    res = cb.cuboid_result_create(t, 1, 1 << 20, 1 << 12)
    rng = W.triangle(n_max)
    runs = []
    for i in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            cb.cuboid_sieve_into(res, [rng], cb.MODE_PLAIN | cb.MODE_TIME_SIEVE, stream)
            b.record(stream)
        st = cb.cuboid_result_wait(res)
        sieve_ms, _ = cb.cuboid_result_sieve_ms(res)
        if i:
            runs.append((a.elapsed_time(b), sieve_ms))
    got = cb.cuboid_result_get(res, 0, 3)
    cb.cuboid_result_free(res)
    cb.cuboid_tables_free(t)
    runs.sort()
    total, sieve = runs[len(runs) // 2]
    n = len(got["survivors"])
    return {"workload": f"triangle 1 <= q < p <= {n_max}, primes 3, 5, 7 (every coprime pair survives)",
            "status": st, "survivors": n, "roots": len(got["roots"]), "ms_total": total, "ms_sieve": sieve,
            "ms_root_test": total - sieve, "survivors_per_s": n / ((total - sieve) / 1e3),
            "thread_us_per_survivor": (total - sieve) * 1e3 / max(n, 1) * (cb.cuboid_device_sms() * 2 * 256),
            "note": "root-test grid: 2 CTAs of 256 threads per SM; thread-us per survivor = root-test time x threads / survivors"}


def deep_leg(cb, torch, stream, reps=5):
    """Every prime below the bound of Eq. 2.7 (the 1192 primes from 11 to 9689; 4.4 GB of
    window rows, far more than the 129 MB L2): table build time and device bytes, then the
    2^14 triangle sieved with them (plain single-range runs, device time per run with CUDA
    events around the sieve and root test) in ascending order (the paper's) and in
    rejection-rate order, beside the 64-prime headline on the same triangle."""
    primes = W.primes_between(11, 9696)
    rng = W.c2()["ranges"][0]
    out = {"primes": f"11..9689 ({len(primes)})", "workload": "triangle 1 <= q < p <= 16384"}
    for name, flag in (("ascending", cb.ORDER_AS_GIVEN), ("rate", cb.ORDER_BY_RATE)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t = cb.cuboid_tables_build(primes, flag, stream)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        n, dev_bytes, _ = cb.cuboid_tables_info(t)
        order = cb.cuboid_tables_order(t)
        res = cb.cuboid_result_create(t, 1)
        times = []
        for i in range(reps + 2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                a.record(stream)
                cb.cuboid_sieve_into(res, [rng], cb.MODE_PLAIN, stream)
                b.record(stream)
            cb.cuboid_result_wait(res)
            if i >= 2:
                times.append(a.elapsed_time(b))
        got = cb.cuboid_result_get(res, 0, n)
        cb.cuboid_result_free(res)
        cb.cuboid_tables_free(t)
        times.sort()
        ms = times[len(times) // 2]
        used = [primes[i] for i, c in enumerate(got["counts"]) if c]
        out[name] = {"table_bytes": dev_bytes, "table_build_s": build_s, "pairs": got["n_pairs"], "ms": ms,
                     "pairs_per_s": got["n_pairs"] / (ms / 1e3), "n_surv": len(got["survivors"]),
                     "first_primes_tried": [primes[i] for i in order[:6]],
                     "largest_prime_rejecting": max(used) if used else None,
                     "sums_ok": sum(got["counts"]) + len(got["survivors"]) == got["n_pairs"]}
    return out


def wide_leg(cb, torch, stream, rows=16):
    """64-bit ranges: 16 rows of the region of Eq. 1.2 (every q from q_lo(p) to 59 p) with
    the 96 primes 11..541 ascending, through cuboid_sieve_wide: the rows from p = 10^8
    (q up to 5.9 10^9: per row a 32-bit piece of 4.3 10^9 q and a based piece of 1.6 10^9),
    the rows p_max + 1 .. p_max + 16 just beyond the 32-bit limit of section 6 (p_max =
    72796055; the based pieces hold a few q), and the 16 rows just below p_max (32-bit
    pieces only) through the same call.  Device time (CUDA events around the enqueue,
    copies back included) and pairs/s; each row's counts and survivors must add up to its
    pair total."""
    p_max = 72796055
    primes = W.primes_between(11, 541)
    t = cb.cuboid_tables_build(primes, cb.ORDER_AS_GIVEN, stream)
    out = {}
    for name, p0 in (("rows_from_1e8", 10 ** 8), ("beyond_p_max", p_max + 1), ("below_p_max", p_max - rows + 1)):
        rngs = [W.rect(p, p, cb.cuboid_region_qmin(p), 59 * p) for p in range(p0, p0 + rows)]
        for it in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                a.record(stream)
                res = cb.cuboid_sieve_wide(t, rngs, stream=stream)
                b.record(stream)
            st = cb.cuboid_result_wait(res)
            ms = a.elapsed_time(b)
            got = [cb.cuboid_result_get_wide(res, i, len(primes)) for i in range(rows)]
            cb.cuboid_result_free(res)
        pairs = sum(g["n_pairs"] for g in got)
        out[name] = {"rows": [p0, p0 + rows - 1], "q": "q_lo(p) .. 59 p (Eq. 1.2)", "status": st,
                     "pieces": sum(len(cb.cuboid_wide_pieces(r)) for r in rngs), "pairs": pairs, "ms": ms,
                     "pairs_per_s": pairs / (ms / 1e3), "n_surv": sum(len(g["survivors"]) for g in got),
                     "q_max": 59 * (p0 + rows - 1),
                     "sums_ok": all(sum(g["counts"]) + len(g["survivors"]) == g["n_pairs"] for g in got)}
    cb.cuboid_tables_free(t)
    out["primes"] = "11..541 (96, ascending)"
    return out


def main():
    args = parse()
    if args.wide_only:
        import torch
        import paper_1601_00636_gb300 as cb
        torch.cuda.set_device(0)
        print(json.dumps({"wide_64bit": wide_leg(cb, torch, torch.cuda.current_stream())}), flush=True)
        return
    if args.root_only:
        import torch
        import paper_1601_00636_gb300 as cb
        torch.cuda.set_device(0)
        print(json.dumps({"root_test": root_test_leg(cb, torch, torch.cuda.current_stream())}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
