"""The CUBOID_DEBUG build: the sieve kernel checks every shared- and global-memory table
window (the window must stay inside the row of (x mod r): s < r and its last word before
the row's end, so the replicated padding of a row is never read as bits of another), every
coprimality-mask entry, factor record and per-warp queue slot.  A failed check is recorded
in the result header and reported as CUBOID_EINDEX; the access is skipped (no trap).

This runs, in a separate process with CUBOID_DEBUG=1 (which loads libcuboid_debug.so),
the small configurations, the edge and ragged ranges, weak sieves, the 64 sampled rows of
the 2^20 triangle, every prime below the Eq. 2.7 bound on a small triangle, 64-bit ranges
and each lanes-per-row build, and requires status OK and the oracle's results throughout.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import gzip, json, os, sys
sys.path.insert(0, os.getcwd())
sys.path.insert(0, os.path.join(os.getcwd(), "tests"))
import torch
torch.cuda.set_device(0)
import paper_1601_00636_gb300 as cb
assert cb.DEBUG and cb.LIB_PATH.endswith("libcuboid_debug.so"), cb.LIB_PATH
import oracle as O
import workloads as W
from test_gpu_parity import _edge_ranges

s = torch.cuda.current_stream()
checked = 0


def run(t, n, ranges, mode, surv_cap=0):
    res = cb.cuboid_result_create(t, len(ranges), surv_cap, 0)
    cb.cuboid_sieve_into(res, ranges, mode, s)
    st = cb.cuboid_result_wait(res)
    out = [cb.cuboid_result_get(res, i, n) for i in range(len(ranges))]
    cb.cuboid_result_free(res)
    assert st == cb.OK, cb.STATUS_NAMES.get(st, st)
    return out


def same(got, want):
    global checked
    for g, w in zip(got, want):
        assert g["n_pairs"] == w["n_pairs"] and list(g["counts"]) == list(w["counts"])
        assert [tuple(x) for x in g["survivors"]] == [tuple(x) for x in w["survivors"]]
        assert [tuple(x) for x in g["roots"]] == [tuple(x) for x in w["roots"]]
        checked += 1


# C1 in every order and form; the edge ranges with each lanes-per-row build
primes = W.first_odd_primes(24)
for flag, mode_o in ((cb.ORDER_AS_GIVEN, False), (cb.ORDER_BY_DENSITY, True), (cb.ORDER_BY_RATE, "rate")):
    t = cb.cuboid_tables_build(primes, flag, s)
    want = O.run(primes, [W.triangle(200)], by_density=mode_o)["ranges"]
    for mode in (cb.MODE_PLAIN, cb.MODE_BATCHED):
        same(run(t, 24, [W.triangle(200)], mode), want)
    cb.cuboid_tables_free(t)
t = cb.cuboid_tables_build(primes, 0, s)
edge = _edge_ranges()
want = O.run(primes, edge)["ranges"]
for lanes in (32, 16, 8):
    cb.cuboid_tables_set_tuning(t, row_lanes=lanes)
    for mode in (cb.MODE_PLAIN, cb.MODE_BATCHED):
        same(run(t, 24, edge, mode), want)
# the diagonal's roots through the root test
diag = [W.rect(1, 60, 1, 60, allow_diagonal=True)]
same(run(t, 24, diag, cb.MODE_BATCHED), O.run(primes, diag)["ranges"])
# a 64-bit range across 2^32
wide = W.rect(72796056, 72796057, (1 << 32) - 700, (1 << 32) + 900)
res = cb.cuboid_sieve_wide(t, [wide], s)
assert cb.cuboid_result_wait(res) == cb.OK
g = cb.cuboid_result_get_wide(res, 0, 24)
cb.cuboid_result_free(res)
n_pairs, counts, surv = O.sieve_range(O.Tables(primes), wide)
assert (g["n_pairs"], g["counts"], g["survivors"]) == (n_pairs, counts, sorted(surv))
cb.cuboid_tables_free(t)

# weak sieves: survivors through the queue and the compaction
for wp, rng in (([3, 5, 7], W.triangle(200)), ([13], W.rect(1, 150, 1, 150))):
    t = cb.cuboid_tables_build(wp, 0, s)
    same(run(t, len(wp), [rng], cb.MODE_PLAIN), O.run(wp, [rng])["ranges"])
    cb.cuboid_tables_free(t)

# stored oracle results: the 2^14 triangle (rate order), 64 rows of the 2^20 triangle
for name, n in (("c2_by_rate.json", 64), ("c4_rows_by_rate.json", 256)):
    with open(os.path.join("tests", "golden", name)) as f:
        gold = json.load(f)
    t = cb.cuboid_tables_build(gold["primes"], cb.ORDER_BY_RATE, s)
    for mode in (cb.MODE_PLAIN, cb.MODE_BATCHED):
        same(run(t, n, gold["ranges"], mode), gold["results"])
    cb.cuboid_tables_free(t)

# every prime below the Eq. 2.7 bound, the deep tables read from global memory
deep = W.primes_between(11, 9696)
t = cb.cuboid_tables_build(deep, cb.ORDER_BY_RATE, s)
got = run(t, len(deep), [W.triangle(2048)], cb.MODE_PLAIN)[0]
assert got["n_pairs"] == sum(len(O.row_pairs(p, W.triangle(2048))) for p in range(2, 2049))
assert sum(got["counts"]) + len(got["survivors"]) == got["n_pairs"]
cb.cuboid_tables_free(t)
torch.cuda.synchronize()
print("DEBUG-BUILD-OK", checked)
"""


def test_debug_build_index_checks_stay_clean():
    import __graft_entry__
    __graft_entry__._builder().build(debug=True)
    env = dict(os.environ, CUBOID_DEBUG="1")
    p = subprocess.run([sys.executable, "-c", SCRIPT], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1200)
    assert p.returncode == 0, p.stdout[-3000:] + p.stderr[-3000:]
    assert "DEBUG-BUILD-OK" in p.stdout
