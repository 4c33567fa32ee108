"""Writes the stored expected values of the GPU parity tests.  Calls only the oracle and
the seeded workload generators (no GPU code).  Run from the repository root:

    python tests/golden/make_golden.py [sieve] [paper_files] [region] [c3_all] [c5_full] [c4_rate]

Each output is JSON: {"config", "primes", "order", "ranges": [...], "results": [...]},
one result per range: n_pairs, counts (caller order), survivors, roots.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def dump(name, config, primes, ranges, by_density=False):
    t0 = time.time()
    T = O.Tables(primes, by_density, full_limit=0)
    res = O.run(primes, ranges, by_density, tables=T)
    out = {"config": config, "primes": primes, "by_density": by_density, "order": res["order"],
           "ranges": ranges, "results": res["ranges"]}
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(f"{name}: {time.time() - t0:.1f} s")


def dump_paper_files(name, primes):
    """SHA-256 and sizes of the paper's two table files for these primes (section 2)."""
    import hashlib
    t0 = time.time()
    blob, recs = O.paper_table_files(primes)
    out = {"primes": primes, "bit_tables_bytes": len(blob), "primes_bytes": len(recs),
           "bit_tables_sha256": hashlib.sha256(blob).hexdigest(),
           "primes_sha256": hashlib.sha256(recs).hexdigest()}
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)
    print(f"{name}: {time.time() - t0:.1f} s")


def dump_region(name, p_from, p_to, primes):
    """Section 5 region scan of rows p_from..p_to (every q of Eq. 1.2) by the oracle."""
    t0 = time.time()
    T = O.Tables(primes, full_limit=0)
    r = O.region_scan(T, p_from, p_to)
    out = {"rows": [p_from, p_to], "primes": primes, "pairs": r["pairs"], "counts": r["counts"],
           "survivors": r["survivors"], "roots": r["roots"], "depth": r["depth"], "r_max": r["r_max"]}
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(f"{name}: {time.time() - t0:.1f} s")


def _sieve_chunk(args):
    """Worker: oracle results of a list of (index, range) with the worker's tables."""
    items = args
    out = []
    for k, rng in items:
        n_pairs, counts, surv = O.sieve_range(_WORKER["T"], rng)
        surv = sorted(surv)
        roots = sorted((p, q, t) for (p, q) in surv for t in O.integer_roots(p, q))
        out.append((k, {"n_pairs": n_pairs, "counts_nz": [[i, c] for i, c in enumerate(counts) if c],
                        "survivors": surv, "roots": roots}))
    return out


_WORKER = {}


def _init_worker(T):
    _WORKER["T"] = T


def dump_many(name, config, primes, ranges, mode, workers=None):
    """Like dump, for thousands of ranges: rows sieved over every host core (spawned
    processes, tables built once by the oracle and handed to each), counts stored sparse
    as [[caller index, count], ...] (every other count is 0), gzip-compressed JSON."""
    import gzip
    import multiprocessing as mp
    t0 = time.time()
    ctx = mp.get_context("spawn")
    workers = workers or os.cpu_count() or 1
    with ctx.Pool(workers) as pool:
        reduced = pool.map(O.reduced_table, primes)
    T = O.Tables(primes, mode, full_limit=0, reduced=reduced)
    # biggest first, dealt round robin in small chunks
    idx = sorted(range(len(ranges)), key=lambda k: -W.lattice_points(ranges[k]))
    chunks = [[(k, ranges[k]) for k in idx[j::workers * 8]] for j in range(workers * 8)]
    results = [None] * len(ranges)
    with ctx.Pool(workers, initializer=_init_worker, initargs=(T,)) as pool:
        for part in pool.imap_unordered(_sieve_chunk, chunks):
            for k, r in part:
                results[k] = r
    out = {"config": config, "primes": primes, "by_density": mode, "order": list(T.order),
           "ranges": ranges, "results": results}
    with gzip.open(os.path.join(HERE, name), "wt") as f:
        json.dump(out, f, separators=(",", ":"))
    print(f"{name}: {time.time() - t0:.1f} s")


def main(which):
    if "c3_all" in which:
        c3 = W.c3()
        dump_many("c3_all_rects.json.gz", "c3: all 4096 rectangles", c3["primes"], c3["ranges"], "rate")
    if "c5_full" in which:
        q = W.poisson_queries(1e3, 24, seed=W.DEFAULT_SEED + 77)
        dump_many("c5_full_queries.json.gz", "c5: 24 queries of the full distribution (area 2^U(10,26), p, q < 2^24)",
                  W.first_odd_primes(128), q, "rate")
    if "c4_rate" in which:
        dump("c4_rows_by_rate.json", "c4 sampled rows, rejection-rate order", W.first_odd_primes(256),
             W.sampled_rows(1 << 20, 64), by_density="rate")
    if "region" in which:
        dump_region("region_112600_112699.json", 112600, 112699, W.primes_between(11, 541))
    if "paper_files" in which:
        dump_paper_files("paper_files_11_541.json", W.primes_between(11, 541))
    if "sieve" not in which:
        return
    c2 = W.c2()
    dump("c2_as_given.json", c2["name"], c2["primes"], c2["ranges"])
    dump("c2_by_density.json", c2["name"], c2["primes"], c2["ranges"], by_density=True)
    dump("c2_by_rate.json", c2["name"], c2["primes"], c2["ranges"], by_density="rate")
    dump("c4_rows.json", "c4 sampled rows", W.first_odd_primes(256), W.sampled_rows(1 << 20, 64))
    rects = [r for r in W.c3()["ranges"] if (r["p_hi"] - r["p_lo"] + 1) * (r["q_hi"] - r["q_lo"] + 1) <= 1 << 16][:64]
    dump("c3_small_rects.json", "c3 rectangles of area <= 2^16", W.first_odd_primes(128), rects)
    c5 = W.poisson_queries(1e3, 48, log2_area=(10.0, 16.0))
    dump("c5_small_queries.json", "c5-shaped queries of area <= 2^16", W.first_odd_primes(128), c5)


if __name__ == "__main__":
    main(sys.argv[1:] or ["sieve", "paper_files", "region", "c3_all", "c5_full", "c4_rate"])
