"""Writes the stored expected values of the GPU parity tests.  Calls only the oracle and
the seeded workload generators (no GPU code).  Run from the repository root:

    python tests/golden/make_golden.py [sieve] [paper_files] [region]

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


def main(which):
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
    main(sys.argv[1:] or ["sieve", "paper_files", "region"])
