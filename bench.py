"""Benchmark of the modulo-primes sieve on GB300 (one JSON line on rank 0).

Workload (N=1, the headline): the triangle 1 <= q < p <= 2^20 (334,211,599,245 coprime
pairs) with the first 256 odd primes in rejection-rate order, sieved by the batched form:
one persistent sieve launch with a device tile queue, replayed from a captured CUDA graph
(plan, sieve with early exit and per-prime counts, survivor compaction, exact root test of
the survivors).  Synthetic, seeded inputs (the workloads module).  A step is one pass of
the hot path over the whole triangle.  The tables (built once by the device table builder,
timed separately) are resident inputs; L2 is flushed (a 256 MiB write) before every timed
step.  The line's own bit_exact check: the pair total equals sum phi(p) over the triangle,
every pair is counted or a survivor, and 64 seeded full rows sieved in the same process
with the same tables equal the oracle's stored results.

Extra objects in the same line: the 2^14 triangle in the plain form (one range per
launch) with the same fields, the batched form against the plain form on the 4096
rectangles of the batched workload, the serving loop, the section 6 region scan, 64-bit
ranges, every prime below the Eq. 2.7 bound, the bulk root test, the roofline of the
dominant kernel, the end-to-end number through the C ABI with host buffers, the oracle
and the C/OpenMP restatement of the paper's loop timed on every host core, and the SM
clocks sampled during the timed region.

--impl reference times the oracle (the CPU restatement) on every host core on the same
workload.  Multi-GPU (torchrun): the triangle grows with N (about N times the pairs) and
each rank sieves one balanced row shard (weak scaling, no data-path collective); value =
all ranks' pairs / max over ranks of the timed region.
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
# 32-bit integer logic issues to the ALU pipe at 16 lanes per clock per SM sub-partition
# (four per SM): 64 lane-ops per clock per SM
INT_LANES_PER_SM_CLK = 64
C4_PAIRS = 334211599245  # sum of phi(p) for p = 2 .. 2^20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip every leg beside the headline")
    ap.add_argument("--workload", default="c4", choices=["c4", "c2", "c4top"],
                    help="c4: the 2^20 triangle, 256 primes, batched (the headline); c2: the 2^14 triangle, "
                         "64 primes, plain; c4top: the 4097 largest rows of the 2^20 triangle (for profiling)")
    ap.add_argument("--serving-seconds", type=float, default=60.0, help="longest run per offered rate")
    ap.add_argument("--serving-queries", type=int, default=10000, help="most queries per offered rate")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample length (wall clock)")
    ap.add_argument("--wide-only", action="store_true",
                    help="run only the 64-bit range leg and print its JSON (for profiling)")
    ap.add_argument("--root-only", action="store_true",
                    help="run only the bulk root-test leg and print its JSON (for profiling)")
    ap.add_argument("--probe-only", action="store_true",
                    help="run only the integer issue probes and print their JSON")
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

def _tune_cache():
    """Autotuner results persist per user (device name, primes, ranges and mode are the key)."""
    d = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    try:
        os.makedirs(d, exist_ok=True)
    except OSError:
        return None
    return os.path.join(d, "cuboid_autotune.txt")


def profile_record(workload: str) -> dict:
    """The committed ncu record of the sieve kernel for this workload (DRAM bytes, warp
    instructions and issue-slot utilisation per launch), or {} when the kernel source
    changed since the capture."""
    src = os.path.join(ROOT, "paper_1601_00636_gb300", "csrc", "sieve.cu")
    try:
        with open(os.path.join(ROOT, "profiles", "sieve_traffic.json")) as f:
            rec = json.load(f)
    except OSError:
        return {}
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    entry = rec.get(workload)
    if not entry or entry.get("sieve_cu_sha256") != sha:
        return {}
    return entry


def host_cpu() -> dict:
    """Core count and model of this host (the GPU machine's host cores)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.strip().lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    import platform
    return {"cores": os.cpu_count(), "model": model or platform.processor() or platform.machine(),
            "machine": __import__("platform").machine()}


def phi_sum(n_max: int, lo: int = 2) -> int:
    """sum phi(p) for p = lo .. n_max (totient sieve)."""
    import numpy as np
    phi = np.arange(n_max + 1, dtype=np.int64)
    for i in range(2, n_max + 1):
        if phi[i] == i:
            phi[i::i] -= phi[i::i] // i
    return int(phi[lo:].sum())


PROBE_KINDS = {0: ("alu_tops", 48), 1: ("lookup_mix_tops", 96), 2: ("lop3", 16), 3: ("funnel_shift", 16),
               4: ("popc_plus_mad", 32), 5: ("mad_lo", 16), 6: ("mad_wide", 16), 7: ("mad_hi", 16),
               8: ("add_min", 16)}


def int_issue_probe(cb, torch, stream, sm_mhz: float = 2070.0):
    """Measured integer issue rates: a dependency-free add/shift/xor stream on every SM
    (alu_tops), the sieve's lookup mix (shared-memory load pair, funnel shift, and, popc,
    xor), and one-instruction streams (lop3, funnel shift, popc + mad, mad.lo, mad.wide,
    mad.hi, the add-then-minimum of the residue steps) as lane-ops per clock per SM at the
    given clock."""
    sms = cb.cuboid_device_sms()
    blocks, threads, iters = sms * 8, 256, 4096
    sink = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    out, per_clk = {}, {}
    for kind, (name, ops) in PROBE_KINDS.items():
        for _ in range(2):
            cb.cuboid_probe_int_issue(kind, blocks, threads, iters, sink.data_ptr(), stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            cb.cuboid_probe_int_issue(kind, blocks, threads, iters, sink.data_ptr(), stream)
            b.record(stream)
        stream.synchronize()
        sec = a.elapsed_time(b) / 1e3
        rate = blocks * threads * iters * ops / sec
        if kind < 2:
            out[name] = rate / 1e12
        per_clk[name] = rate / (sms * sm_mhz * 1e6)
    out["lane_ops_per_clk_per_sm"] = per_clk
    return out


# ------------------------------------------------------------------ CPU baselines (oracle, paper loop)

_WORKER = {}


def _cpu_init(T):
    _WORKER["T"] = T


def _cpu_ready(_):
    return os.getpid()


def _cpu_rows(args):
    """Worker: the oracle over whole rows p of the triangle (q < p) until the deadline."""
    import oracle as O
    rows, deadline = args
    T = _WORKER["T"]
    pairs = done = 0
    for p in rows:
        if time.time() > deadline:
            break
        n, _, _ = O.sieve_range(T, W.rect(int(p), int(p), 1, int(p) - 1, q_lt_p=True))
        pairs += n
        done += 1
    return pairs, done


class OraclePool:
    """The oracle as it stands on every host core: spawned processes (never forked after a
    GPU call), each holding the oracle's tables of the workload's primes in rejection-rate
    order, sieving seeded random rows of the workload's triangle."""

    def __init__(self, primes, workers=None):
        import multiprocessing as mp

        import oracle as O
        self.workers = workers or os.cpu_count() or 1
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(self.workers) as pool:  # the reduced tables, one prime per task
            reduced = pool.map(O.reduced_table, primes)
        T = O.Tables(primes, "rate", full_limit=0, reduced=reduced)
        self.pool = ctx.Pool(self.workers, initializer=_cpu_init, initargs=(T,))
        self.pool.map(_cpu_ready, range(4 * self.workers))  # every worker up before timing
        self.setup_s = time.perf_counter() - t0

    def time_rows(self, n_max: int, seconds: float, seed: int) -> dict:
        import numpy as np
        rows = W.rng(seed).permutation(np.arange(2, n_max + 1))[:200000]
        chunks = [rows[i::self.workers] for i in range(self.workers)]
        t0 = time.perf_counter()
        deadline = time.time() + seconds
        res = self.pool.map(_cpu_rows, [(c, deadline) for c in chunks], chunksize=1)
        dt = time.perf_counter() - t0
        pairs = sum(r[0] for r in res)
        done = sum(r[1] for r in res)
        return {"value": pairs / dt, "pairs": pairs, "rows": done, "seconds": dt}

    def close(self):
        self.pool.terminate()
        self.pool.join()


def cpu_baseline(cfg_name: str, primes, n_max: int, seconds: float, seed: int = W.DEFAULT_SEED) -> dict:
    """The oracle on every host core on a bounded sample of the workload (seeded random full
    rows of the triangle), and the C/OpenMP restatement of the paper's loop
    (oracle/paper_loop.c) on C2 and C3 in full and on seeded rows of C4."""
    cpu = host_cpu()
    pool = OraclePool(primes)
    try:
        r = pool.time_rows(n_max, seconds, seed)
    finally:
        pool.close()
    out = {"value": r["value"], "unit": UNIT, "cores": pool.workers, "kind": "oracle",
           "sample": f"{r['rows']} seeded random full rows p of the {cfg_name} triangle ({r['pairs']} pairs, "
                     f"{r['seconds']:.1f} s wall on {pool.workers} processes; tables built once in "
                     f"{pool.setup_s:.1f} s, not timed)",
           "cpu_model": cpu["model"], "os_cpu_count": cpu["cores"], "machine": cpu["machine"]}
    try:
        out["paper_loop"] = paper_loop_baseline(seed)
    except Exception as e:  # the C baseline is context; its failure must not hide the rest
        out["paper_loop"] = {"error": repr(e)[:300]}
    return out


def paper_loop_baseline(seed: int = W.DEFAULT_SEED) -> dict:
    """The section 5 loop in C with OpenMP over Eq. 2.6 tables on every host core: C2 and
    C3 in full (checked against the oracle's stored results where they exist) and 2048
    seeded rows of C4 (pairs/s extrapolated to the whole triangle, labelled as such)."""
    import gzip

    import numpy as np

    import oracle as O
    from oracle.paper_loop import PaperLoop, max_threads
    out = {"kind": "paper loop (section 5) in C with OpenMP, 32-bit residues, Eq. 2.6 tables",
           "threads": max_threads()}
    c2 = W.c2()
    L = PaperLoop(c2["primes"])
    T2 = O.Tables(c2["primes"], "rate", full_limit=0)
    t0 = time.perf_counter()
    n, counts, surv = L.sieve(T2.order, c2["ranges"][0])
    dt = time.perf_counter() - t0
    with open(os.path.join(ROOT, "tests", "golden", "c2_by_rate.json")) as f:
        g = json.load(f)["results"][0]
    out["c2_full"] = {"pairs": n, "seconds": dt, "pairs_per_s": n / dt,
                      "equals_oracle": n == g["n_pairs"] and counts == g["counts"]
                      and surv == [tuple(x) for x in g["survivors"]]}
    L.close()
    c3 = W.c3()
    gold3 = os.path.join(ROOT, "tests", "golden", "c3_all_rects.json.gz")
    order3 = None
    if os.path.exists(gold3):
        with gzip.open(gold3, "rt") as f:
            G3 = json.load(f)
        order3 = G3["order"]
    else:
        G3 = None
        order3 = O.Tables(c3["primes"], "rate", full_limit=0).order
    L = PaperLoop(c3["primes"])
    t0 = time.perf_counter()
    res = L.sieve_many(order3, c3["ranges"])
    dt = time.perf_counter() - t0
    pairs = sum(x[0] for x in res)
    eq = None
    if G3 is not None:
        eq = all(x[0] == g_["n_pairs"] and x[1] == _dense(g_["counts_nz"], len(c3["primes"]))
                 and x[2] == [tuple(y) for y in g_["survivors"]] for x, g_ in zip(res, G3["results"]))
    out["c3_full"] = {"pairs": pairs, "seconds": dt, "pairs_per_s": pairs / dt, "equals_oracle": eq}
    L.close()
    c4 = W.c4()
    L = PaperLoop(c4["primes"])
    with open(os.path.join(ROOT, "tests", "golden", "c4_rows_by_rate.json")) as f:
        order4 = json.load(f)["order"]  # the oracle's rejection-rate order of the 256 primes
    rows = sorted(int(p) for p in W.rng(seed).permutation(np.arange(2, (1 << 20) + 1))[:2048])
    rngs = [W.rect(p, p, 1, p - 1, q_lt_p=True) for p in rows]
    t0 = time.perf_counter()
    res = L.sieve_many(order4, rngs)
    dt = time.perf_counter() - t0
    pairs = sum(x[0] for x in res)
    out["c4_rows"] = {"rows": len(rows), "pairs": pairs, "seconds": dt, "pairs_per_s": pairs / dt,
                      "c4_extrapolated_s": C4_PAIRS / (pairs / dt),
                      "note": "2048 seeded random full rows of the 2^20 triangle; the whole-triangle time is "
                              "extrapolated from their pairs/s"}
    L.close()
    return out


def _dense(nz, n):
    out = [0] * n
    for i, c in nz:
        out[i] = c
    return out


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    """The oracle as it stands on every host core, each step a bounded sample (seeded
    random full rows) of the same workload as our arm."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    name, primes, n_max = _cpu_workload(args.workload)
    pool = OraclePool(primes)
    try:
        per = min(10.0, max(2.0, 60.0 / max(args.steps, 1)))
        for i in range(args.warmup):
            pool.time_rows(n_max, 0.5, W.DEFAULT_SEED + 1000 + i)
        steps = [pool.time_rows(n_max, per, W.DEFAULT_SEED + i) for i in range(args.steps)]
    finally:
        pool.close()
    pairs = sum(s["pairs"] for s in steps)
    secs = sum(s["seconds"] for s in steps)
    v = pairs / secs
    cpu = host_cpu()
    sample = (f"{sum(s['rows'] for s in steps)} seeded random full rows p of the {name} triangle over "
              f"{args.steps} steps of {per:.1f} s ({pairs} pairs); {pool.workers} processes")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(steps),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": name, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.workers, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu["model"], "os_cpu_count": cpu["cores"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _cpu_workload(workload: str):
    if workload == "c2":
        return W.c2()["name"], W.c2()["primes"], 1 << 14
    return W.c4()["name"], W.c4()["primes"], 1 << 20


# ------------------------------------------------------------------ our arm

def _spec(cb, workload: str, world: int, rank: int):
    """The timed workload: name, primes, this rank's range, the form, and the pair total
    of the whole job when it has a closed form."""
    import math
    if workload == "c4top":
        return {"name": "c4top_rows2^20-4096..2^20_256primes", "primes": W.first_odd_primes(256),
                "range": W.rect((1 << 20) - 4096, 1 << 20, 1, (1 << 20) - 1, q_lt_p=True),
                "mode": cb.MODE_PLAIN, "form": "plain (one range per launch)", "side": 1 << 20,
                "whole_pairs": None, "launches_per_step": 2}
    if workload == "c2":
        side, cfg, mode, form = 1 << 14, W.c2(), cb.MODE_PLAIN, "plain (one range per launch)"
        lps = 2
    else:
        side, cfg, mode = 1 << 20, W.c4(), cb.MODE_BATCHED
        form = "batched (persistent kernel, device tile queue, replayed CUDA graph)"
        lps = 4
    name = cfg["name"]
    rng = cfg["ranges"][0]
    if world > 1:  # weak scaling: the triangle grows with N, each rank sieves one balanced shard
        side = int(round(side * math.sqrt(world)))
        rng, _ = cb.cuboid_shard_range(W.triangle(side), world, rank)
        name = f"triangle 1<=q<p<={side}, {len(cfg['primes'])} primes, {world} shards"
    return {"name": name, "primes": cfg["primes"], "range": rng, "mode": mode, "form": form, "side": side,
            "whole_pairs": "phi", "launches_per_step": lps}


def measure(cb, torch, dist, stream, flush, spec, args, world, rank, tables=None):
    """One workload: table build, autotune, parity of the timed configuration, K timed
    steps (CUDA events on the launching stream, max over ranks), the sieve kernel's own
    launch time in a second pass, and the roofline of that kernel."""
    primes = spec["primes"]
    n_primes = len(primes)
    rng = spec["range"]
    mode = spec["mode"]
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t = tables or cb.cuboid_tables_build(primes, cb.ORDER_BY_RATE, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    table_ms = e0.elapsed_time(e1)
    # kernel shape picked by the autotuner on this very workload (outside the timed region;
    # a few seconds for the 2^20 triangle, cached)
    tune, _ = cb.cuboid_autotune(t, [rng], mode, stream, _tune_cache())
    res = cb.cuboid_result_create(t, 1)
    arr = cb.ranges_array([rng])
    dev_ranges = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to("cuda")

    def step(m=mode):
        cb.cuboid_sieve_device(res, dev_ranges.data_ptr(), 1, m, stream)

    # parity of the timed configuration (outside the timed region)
    step()
    cb.cuboid_result_download(res, stream)
    st = cb.cuboid_result_wait(res)
    got = cb.cuboid_result_get(res, 0, n_primes)
    n_pairs = got["n_pairs"]
    check = {"status_ok": st == cb.OK, "counts_plus_survivors_equal_pairs":
             sum(got["counts"]) + len(got["survivors"]) == n_pairs}
    if world > 1:
        tot = torch.tensor([n_pairs], dtype=torch.int64, device="cuda")
        dist.all_reduce(tot)
        n_total = int(tot.item())
    else:
        n_total = n_pairs
    if spec["name"].startswith("c2_") and world == 1:
        with open(os.path.join(ROOT, "tests", "golden", "c2_by_rate.json")) as f:
            gold = json.load(f)["results"][0]
        check["equals_stored_oracle_result"] = (n_pairs == gold["n_pairs"] and got["counts"] == gold["counts"]
                                               and [list(x) for x in got["survivors"]] == gold["survivors"]
                                               and [list(x) for x in got["roots"]] == gold["roots"])
    if spec["whole_pairs"] == "phi" and rank == 0:
        want = C4_PAIRS if spec["side"] == (1 << 20) else phi_sum(spec["side"])
        check["pair_total_equals_sum_phi"] = n_total == want
    elif spec["name"].startswith("c4top"):
        check["pair_total_equals_sum_phi"] = n_pairs == phi_sum(1 << 20, (1 << 20) - 4096)
    if spec["name"].startswith("c4_") and world == 1:
        check["sampled_rows"] = c4_rows_check(cb, t, stream, n_primes)

    # algorithmic work per launch (instrumented run, outside the timed region)
    cb.cuboid_sieve_device(res, dev_ranges.data_ptr(), 1, mode | cb.MODE_COUNT_STEPS, stream)
    cb.cuboid_result_wait(res)
    stats = cb.cuboid_result_stats(res)

    dev = torch.cuda.current_device()
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
    _barrier(torch, dist, world)
    evs = []
    torch.cuda.nvtx.range_push("timed")  # profilers capture only this region
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
        evs.append((a, b))
    stream.synchronize()
    # the sieve kernel's own launch time, on the same steps with events around the sieve
    # launch (those events keep the sieve from overlapping the kernel before it, so this
    # pass is timed apart from the steps above)
    sieve_ms, sieve_launches = 0.0, 0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            step(mode | cb.MODE_TIME_SIEVE)
        stream.synchronize()
        ms, nl = cb.cuboid_result_sieve_ms(res) if cb.cuboid_result_wait(res) == cb.OK else (0.0, 0)
        sieve_ms += ms
        sieve_launches += nl
    torch.cuda.nvtx.range_pop()
    _barrier(torch, dist, world)
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    t_max = torch.tensor([total_ms], device="cuda")
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    total_s = float(t_max.item()) / 1e3
    value = n_total * args.steps / total_s

    # roofline of the dominant kernel (the sieve): algorithmic integer lane-ops per launch
    # over its average launch time, against the 32-bit integer logic pipe's peak
    sms = cb.cuboid_device_sms()
    sm_max = float(clk.get("sm_max_mhz") or 2070.0)
    peak = sms * INT_LANES_PER_SM_CLK * sm_max * 1e6 / 1e12
    per_launch_ms = sieve_ms / max(sieve_launches, 1)
    alg_ops = stats["word_steps"] * OPS_PER_WORD_STEP
    achieved = alg_ops / (per_launch_ms / 1e3) / 1e12
    probe = int_issue_probe(cb, torch, stream, sm_max)
    prof = profile_record(spec["name"])
    executed = None
    if prof.get("inst_executed_per_launch"):
        # every executed instruction, on any pipe, against the issue slots (one warp
        # instruction per clock per SM sub-partition): not against the ALU pipe alone
        ex = prof["inst_executed_per_launch"] * 32 / (per_launch_ms / 1e3) / 1e12
        issue_peak = sms * 4 * 32 * sm_max * 1e6 / 1e12
        executed = {"tops": ex, "issue_peak_tops": issue_peak, "frac_of_issue_slots": ex / issue_peak,
                    "issue_active_pct_ncu": prof.get("issue_active_pct"),
                    "alu_pipe_pct_ncu": prof.get("alu_pipe_pct"),
                    "note": "warp instructions per launch from the committed ncu record x 32 lanes / live launch "
                            "time, against 4 issue slots x 32 lanes per clock per SM (instructions of every pipe)"}
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": prof.get("dram_bytes_per_launch"), "kernel": "k_sieve", "launch_ms": per_launch_ms,
                "peak_note": f"{sms} SMs x {INT_LANES_PER_SM_CLK} int32 logic lanes per clock (16 per SM "
                             f"sub-partition, the ALU pipe) x {sm_max:.0f} MHz (maximum SM clock seen)",
                "probe": probe, "frac_of_probe": achieved / probe["alu_tops"], "executed": executed,
                "work": {"word_steps": stats["word_steps"], "words": stats["words"],
                         "warp_steps": stats["warp_steps"], "ops_per_word_step": OPS_PER_WORD_STEP,
                         "pairs": n_pairs}}
    out = {"value": value, "ms_per_step": total_ms / args.steps, "pairs_per_step": n_total,
           "bit_exact": all(v if not isinstance(v, dict) else v.get("equal", False) for v in check.values()),
           "checks": check, "table_build_ms": table_ms, "tuning": tune, "roofline": roofline, "clocks": clk,
           "gpu_launches": spec["launches_per_step"] * args.steps}
    cb.cuboid_result_free(res)
    return out, t


def c4_rows_check(cb, t, stream, n_primes) -> dict:
    """64 seeded full rows of the 2^20 triangle sieved with the headline's tables (one
    batched run) against the oracle's stored results (rejection-rate order)."""
    path = os.path.join(ROOT, "tests", "golden", "c4_rows_by_rate.json")
    with open(path) as f:
        gold = json.load(f)
    order = cb.cuboid_tables_order(t)
    res = cb.cuboid_result_create(t, len(gold["ranges"]))
    try:
        cb.cuboid_sieve_into(res, gold["ranges"], cb.MODE_BATCHED, stream)
        st = cb.cuboid_result_wait(res)
        bad = []
        for i, g in enumerate(gold["results"]):
            got = cb.cuboid_result_get(res, i, n_primes)
            if not (got["n_pairs"] == g["n_pairs"] and got["counts"] == g["counts"]
                    and [list(x) for x in got["survivors"]] == g["survivors"]
                    and [list(x) for x in got["roots"]] == g["roots"]):
                bad.append(gold["ranges"][i]["p_lo"])
    finally:
        cb.cuboid_result_free(res)
    return {"rows": len(gold["ranges"]), "equal": st == cb.OK and not bad and order == gold["order"],
            "mismatched_rows": bad, "pairs": sum(g["n_pairs"] for g in gold["results"])}


def _barrier(torch, dist, world):
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    import paper_1601_00636_gb300 as cb

    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    spec = _spec(cb, args.workload, world, rank)
    head, t = measure(cb, torch, dist, stream, flush, spec, args, world, rank)
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": spec["name"], "pairs_per_step": head["pairs_per_step"],
                       "primes": len(spec["primes"]), "order": "rejection rate (CUBOID_ORDER_BY_RATE)",
                       "form": spec["form"], "l2": "flushed (256 MiB write) before each step",
                       "parallelism": f"range shards x{world} (no data-path collective)"},
            "bit_exact": head["bit_exact"], "checks": head["checks"], "table_build_ms": head["table_build_ms"],
            "tuning": head["tuning"], "roofline": head["roofline"], "clocks": head["clocks"],
            "gpu_launches": 2 * head["gpu_launches"],
            "gpu_launches_note": ("per timed step: reset, plan, sieve and root test (one graph); the "
                                  "sieve-timing pass adds as many" if spec["mode"] == cb.MODE_BATCHED else
                                  "sieve + root test per timed step (a single range needs no plan kernel); "
                                  "the sieve-timing pass adds as many")}
    if not args.no_extras and rank == 0:
        line["e2e"] = e2e_leg(cb, torch, spec, args)
        if args.workload == "c4":
            c2s = _spec(cb, "c2", 1, 0)
            c2, t2 = measure(cb, torch, dist, stream, flush, c2s, args, 1, 0)
            c2["e2e"] = e2e_leg(cb, torch, c2s, args, cold=True)
            c2["workload"] = c2s["name"]
            c2["form"] = c2s["form"]
            line["c2_plain"] = c2
            cb.cuboid_tables_free(t2)
        line["forms"] = forms_leg(cb, torch, stream, flush)
        line["serving"] = serving_leg(cb, torch, stream, args)
        line["region_section6"] = region_leg(cb, torch, stream)
        line["wide_64bit"] = wide_leg(cb, torch, stream)
        line["deep_primes"] = deep_leg(cb, torch, stream)
        line["root_test"] = root_test_leg(cb, torch, stream)
        name, primes, n_max = _cpu_workload(args.workload)
        line["cpu_baseline"] = cpu_baseline(name, primes, n_max, args.cpu_seconds)
    elif rank == 0:
        line["e2e"] = None
    cb.cuboid_tables_free(t)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def e2e_leg(cb, torch, spec, args, cold=False):
    """Through the C ABI from host buffers, steady state: tables built once, then every
    step copies the range from pinned host memory to the device, runs the whole path
    (the workload's form) and reads the header, pair total and counts (and any survivor
    and root records) back (cuboid_sieve_into + wait + get on a reused result); wall clock,
    median.  cold: every step also builds the tables from the host prime list and
    allocates and frees the result (cuboid_tables_build + cuboid_sieve)."""
    primes, rng, mode = spec["primes"], spec["range"], spec["mode"]
    s = torch.cuda.Stream()
    k = max(5, min(args.steps, 20))
    t = cb.cuboid_tables_build(primes, cb.ORDER_BY_RATE, s)
    cb.cuboid_autotune(t, [rng], mode, s, _tune_cache())
    res = cb.cuboid_result_create(t, 1)
    arr = cb.ranges_array([rng])
    times, n_pairs, ok = [], 0, True
    for i in range(k + 3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cb.cuboid_sieve_into(res, None, mode, s, arr=arr)
        ok &= cb.cuboid_result_wait(res) == cb.OK
        got = cb.cuboid_result_get(res, 0, len(primes))
        dt = time.perf_counter() - t0
        n_pairs = got["n_pairs"]
        if i >= 3:
            times.append(dt)
    cb.cuboid_result_free(res)
    cb.cuboid_tables_free(t)
    times.sort()
    per = times[len(times) // 2]
    h2d = 24  # the range (one cuboid_range)
    d2h = 128 + 8 + 8 * len(primes)  # one copy: device header (padded), pair total, counts
    out = {"value": n_pairs / per, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": per * 1e3, "steps": k, "status_ok": ok,
           "includes": ("host range -> device (pinned copy), reset + plan + persistent sieve + root test "
                        "(one graph), header/counts -> host in one copy (survivor and root records when present)"
                        if mode == cb.MODE_BATCHED else
                        "host range -> device (kernel argument), sieve + root test, header/counts -> host in one "
                        "copy (survivor and root records when present)")}
    if cold:
        ct = []
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
                ct.append(time.perf_counter() - t0)
        ct.sort()
        out["cold"] = {"value": n_pairs / ct[len(ct) // 2], "ms_per_step": 1e3 * ct[len(ct) // 2],
                       "h2d_bytes_per_step": h2d + 4 * len(primes),
                       "includes": "also table build from the host prime list and result allocation/free"}
    return out


def serving_leg(cb, torch, stream, args, rates=(1e2, 3e2, 1e3, 3e3, 1e4), beyond=(3e4, 1e5, 3e5, 1e6, 3e6, 1e7)):
    """Poisson streams of range queries (area 2^U(10,26), p, q < 2^24, 128 primes) served
    by the continuous-batching loop.  Each offered rate runs for min(serving_seconds,
    serving_queries / rate) seconds of arrivals, replayed by the library's native load
    loop (cuboid_server_replay) so that the host language does not limit the offered
    load; latency = admission to result on the host, per query (p50/p99).  The rates past
    1e4/s (up to 1e7/s) look for saturation: the first offered rate whose achieved query rate falls below
    90 % of it.  Served-in-mix = run-alone (pair totals, counts, survivors and roots) on a
    seeded 1 % of the queries of every rate."""
    import random
    c5 = W.c5()
    n_primes = len(c5["primes"])
    t = cb.cuboid_tables_build(c5["primes"], cb.ORDER_BY_RATE, stream)
    srv = cb.cuboid_server_create(t, 0, 4096)
    out = {"primes": n_primes, "seconds_per_rate": args.serving_seconds, "queries_per_rate": args.serving_queries,
           "rates": [], "latency": "admission to result on the host (native replay loop)"}
    check = []
    saturated = None
    try:
        for ri, rate in enumerate(tuple(rates) + tuple(beyond)):
            n = int(max(200, min(args.serving_queries, rate * args.serving_seconds)))
            qs = W.poisson_queries(rate, n, seed=W.DEFAULT_SEED + ri)
            r = cb.cuboid_server_replay(srv, qs, [q["t"] for q in qs])
            lat = sorted(r["latency_s"])
            pairs = sum(r["npairs"])
            g = random.Random(7919 + ri)
            pick = {i for i in range(n) if g.random() < 0.01}
            for i, tk in enumerate(r["tickets"]):
                res = cb.cuboid_server_poll(srv, tk)
                if i in pick:
                    cb.cuboid_result_wait(res)
                    got = cb.cuboid_result_get(res, 0, n_primes)
                    check.append((qs[i], got))
                cb.cuboid_result_free(res)
            offered_span = qs[-1]["t"]
            row = {"rate_per_s": rate, "queries": n, "pairs": pairs, "wall_s": r["wall_s"],
                   "achieved_queries_per_s": n / r["wall_s"], "pairs_per_s": pairs / r["wall_s"],
                   "offered_span_s": offered_span, "p50_ms": 1e3 * lat[len(lat) // 2],
                   "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                   "refused_retries": r["refused"], "errors": sum(1 for x in r["status"] if x != cb.OK)}
            out["rates"].append(row)
            if saturated is None and row["achieved_queries_per_s"] < 0.9 * rate:
                saturated = row
        out["server"] = cb.cuboid_server_stats(srv)
    finally:
        cb.cuboid_server_destroy(srv, 120000)
    best = max(out["rates"], key=lambda x: x["achieved_queries_per_s"])
    out["saturation"] = {"first_saturated_offered_rate_per_s": saturated["rate_per_s"] if saturated else None,
                         "at_saturation": saturated,
                         "max_achieved_queries_per_s": best["achieved_queries_per_s"],
                         "max_pairs_per_s": max(x["pairs_per_s"] for x in out["rates"]),
                         "rule": "first offered rate whose achieved query rate is below 90 % of it"}
    # mix vs alone on the seeded 1 % sample
    same = True
    for q, g in check:
        r = cb.cuboid_sieve(t, q["p_lo"], q["p_hi"], q["q_lo"], q["q_hi"], 0, stream)
        cb.cuboid_result_wait(r)
        a = cb.cuboid_result_get(r, 0, n_primes)
        cb.cuboid_result_free(r)
        same &= (a["n_pairs"], a["counts"], a["survivors"], a["roots"]) == \
                (g["n_pairs"], g["counts"], g["survivors"], g["roots"])
    out["mix_equals_alone"] = {"checked": len(check), "equal": same,
                               "compared": "pair totals, per-prime counts, survivors and roots"}
    cb.cuboid_tables_free(t)
    return out


def forms_leg(cb, torch, stream, flush, warm=3, reps=10):
    """Plain (one launch sequence per range) vs batched (one persistent launch replayed
    from a CUDA graph) on the 4096 rectangles of the batched workload: 3 warm-ups, then
    the median of 10 (CUDA events, L2 flushed before each), the host time to enqueue the
    plain form's 4096 launch sequences beside it, batched = plain on every rectangle, and
    both against the oracle's stored results for all 4096 rectangles."""
    import gzip
    out = {}
    c3 = W.c3()
    n_primes = len(c3["primes"])
    t = cb.cuboid_tables_build(c3["primes"], cb.ORDER_BY_RATE, stream)
    tune3, _ = cb.cuboid_autotune(t, c3["ranges"], cb.MODE_BATCHED, stream, _tune_cache())
    res = cb.cuboid_result_create(t, len(c3["ranges"]))
    arr = cb.ranges_array(c3["ranges"])
    dev = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to("cuda")
    n = len(c3["ranges"])

    def timed(mode):
        for _ in range(warm):
            cb.cuboid_sieve_device(res, dev.data_ptr(), n, mode, stream)
        torch.cuda.synchronize()
        ms, host = [], []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.zero_()
                a.record(stream)
                h0 = time.perf_counter()
                cb.cuboid_sieve_device(res, dev.data_ptr(), n, mode, stream)
                host.append(time.perf_counter() - h0)
                b.record(stream)
            stream.synchronize()
            ms.append(a.elapsed_time(b))
        cb.cuboid_result_download(res, stream)
        st = cb.cuboid_result_wait(res)
        got = [cb.cuboid_result_get(res, i, n_primes) for i in range(n)]
        ms.sort()
        host.sort()
        return got, ms[len(ms) // 2], host[len(host) // 2] * 1e3, st

    got_b, ms_b, host_b, st_b = timed(cb.MODE_BATCHED)
    got_p, ms_p, host_p, st_p = timed(cb.MODE_PLAIN)
    pairs = sum(g["n_pairs"] for g in got_b)
    key = lambda g: (g["n_pairs"], g["counts"], g["survivors"], g["roots"])  # noqa: E731
    same = all(key(a) == key(b) for a, b in zip(got_b, got_p))
    oracle_eq = None
    gold = os.path.join(ROOT, "tests", "golden", "c3_all_rects.json.gz")
    if os.path.exists(gold):
        with gzip.open(gold, "rt") as f:
            G = json.load(f)
        oracle_eq = all(g["n_pairs"] == w["n_pairs"] and g["counts"] == _dense(w["counts_nz"], n_primes)
                        and [list(x) for x in g["survivors"]] == w["survivors"]
                        and [list(x) for x in g["roots"]] == w["roots"] for g, w in zip(got_b, G["results"]))
    out["c3_4096_rectangles"] = {"pairs": pairs, "batched_ms": ms_b, "plain_ms": ms_p, "tuning": tune3,
                                 "batched_pairs_per_s": pairs / (ms_b / 1e3),
                                 "plain_pairs_per_s": pairs / (ms_p / 1e3),
                                 "batched_over_plain": ms_p / ms_b,
                                 "plain_host_enqueue_ms": host_p, "batched_host_enqueue_ms": host_b,
                                 "status_ok": st_b == cb.OK and st_p == cb.OK,
                                 "batched_equals_plain": same, "equals_oracle_all_4096": oracle_eq,
                                 "timing": f"{warm} warm-ups, median of {reps}, CUDA events, L2 flushed"}
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
    if args.probe_only:
        import torch
        import paper_1601_00636_gb300 as cb
        torch.cuda.set_device(0)
        print(json.dumps({"probe": int_issue_probe(cb, torch, torch.cuda.current_stream())}), flush=True)
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
