"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit-exact.

Survivor sets, roots, per-prime counts and pair totals must equal the oracle's on the
same seeded inputs.  Stored expected values under tests/golden/ were written by
tests/golden/make_golden.py, which calls only the oracle.
"""
import gzip
import json
import math
import os
import random

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def cb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1601_00636_gb300 as cb
    torch.cuda.set_device(0)
    return cb


@pytest.fixture(scope="module")
def stream():
    import torch
    return torch.cuda.current_stream()


def _order_flag(cb, by_density):
    return {False: cb.ORDER_AS_GIVEN, True: cb.ORDER_BY_DENSITY, "rate": cb.ORDER_BY_RATE}[by_density]


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _norm(res):
    return {"n_pairs": res["n_pairs"], "counts": list(res["counts"]),
            "survivors": [tuple(x) for x in res["survivors"]],
            "roots": [tuple(x) for x in res["roots"]]}


def _run(cb, t, n_primes, ranges, mode, stream, surv_cap=0):
    res = cb.cuboid_result_create(t, len(ranges), surv_cap, 0)
    try:
        cb.cuboid_sieve_into(res, ranges, mode, stream)
        st = cb.cuboid_result_wait(res)
        out = [cb.cuboid_result_get(res, i, n_primes) for i in range(len(ranges))]
    finally:
        cb.cuboid_result_free(res)
    return st, out


def _check_against(got, want):
    assert len(got) == len(want)
    for i, (g, w) in enumerate(zip(got, want)):
        g, w = _norm(g), _norm(w)
        assert g["n_pairs"] == w["n_pairs"], (i, g["n_pairs"], w["n_pairs"])
        assert g["counts"] == w["counts"], (i, g["counts"], w["counts"])
        assert g["survivors"] == w["survivors"], i
        assert g["roots"] == w["roots"], i


@pytest.fixture(scope="module")
def c1_tables(cb, stream):
    t = cb.cuboid_tables_build(W.first_odd_primes(24), cb.ORDER_AS_GIVEN, stream)
    yield t
    cb.cuboid_tables_free(t)


# ---------------------------------------------------------------- K1: tables

@pytest.mark.parametrize("build", ["reduced", "full"])
def test_c1_tables_bit_exact(cb, stream, build):
    primes = W.first_odd_primes(24)
    t = cb.cuboid_tables_build(primes, cb.BUILD_FULL if build == "full" else cb.BUILD_REDUCED, stream)
    try:
        for i, r in enumerate(primes):
            assert cb.cuboid_tables_copy_bits(t, i) == O.pack_table_bytes(O.unsolvable_table(r)), r
            assert np.array_equal(np.frombuffer(cb.cuboid_tables_copy_reduced(t, i, r), np.uint8),
                                  O.reduced_table(r)), r
    finally:
        cb.cuboid_tables_free(t)


def test_u11_matches_paper_through_gpu(cb, stream):
    """Eq. 2.6 bytes of u_11 straight from the device."""
    t = cb.cuboid_tables_build([11], 0, stream)
    try:
        b = cb.cuboid_tables_copy_bits(t, 0)
    finally:
        cb.cuboid_tables_free(t)
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "u11_bytes_eq2_6.txt")) if ln[0].isdigit()]
    assert len(b) == 16
    for idx, bits in rows:
        assert format(b[int(idx)], "08b") == bits


def _unpack(b, r):
    bits = np.unpackbits(np.frombuffer(b, np.uint8), bitorder="little")[: r * r]
    return bits.reshape(r, r)


def test_full_equals_reduced_all_256_primes(cb, stream):
    """Brute force over every t equals the homogeneity reduction, for every prime of the
    256-prime list; each table is symmetric; every v_r equals the oracle's."""
    primes = W.first_odd_primes(256)
    tf = cb.cuboid_tables_build(primes, cb.BUILD_FULL, stream)
    tr = cb.cuboid_tables_build(primes, cb.BUILD_REDUCED, stream)
    try:
        for i, r in enumerate(primes):
            bf, br = cb.cuboid_tables_copy_bits(tf, i), cb.cuboid_tables_copy_bits(tr, i)
            assert bf == br, r
            u = _unpack(bf, r)
            assert np.array_equal(u, u.T), r
            assert not u[0].any() and not u[:, 0].any()
            if i % 16 == 0 or r > 1500:
                assert np.array_equal(np.frombuffer(cb.cuboid_tables_copy_reduced(tr, i, r), np.uint8),
                                      O.reduced_table(r)), r
    finally:
        cb.cuboid_tables_free(tf)
        cb.cuboid_tables_free(tr)


def test_c2_primes_full_tables_vs_oracle(cb, stream):
    primes = [r for r in W.first_odd_primes(64) if r > 97][::4]
    t = cb.cuboid_tables_build(primes, cb.BUILD_FULL, stream)
    try:
        for i, r in enumerate(primes):
            assert cb.cuboid_tables_copy_bits(t, i) == O.pack_table_bytes(O.unsolvable_table(r)), r
    finally:
        cb.cuboid_tables_free(t)


@pytest.mark.parametrize("n", [24, 64, 128, 256])
def test_effective_order(cb, stream, n):
    primes = W.first_odd_primes(n)
    for flag, dens in ((cb.ORDER_AS_GIVEN, False), (cb.ORDER_BY_DENSITY, True), (cb.ORDER_BY_RATE, "rate")):
        t = cb.cuboid_tables_build(primes, flag, stream)
        try:
            got = cb.cuboid_tables_order(t)
        finally:
            cb.cuboid_tables_free(t)
        want = O.effective_order(primes, [int(O.reduced_table(r).sum()) for r in primes], dens)
        assert got == want


# ---------------------------------------------------------------- K2-K4: sieve

@pytest.mark.parametrize("mode", ["plain", "batched"])
@pytest.mark.parametrize("dens", [False, True, "rate"])
def test_c1_parity(cb, stream, mode, dens):
    cfg = W.c1()
    primes = cfg["primes"]
    t = cb.cuboid_tables_build(primes, _order_flag(cb, dens), stream)
    try:
        st, got = _run(cb, t, len(primes), cfg["ranges"],
                       cb.MODE_BATCHED if mode == "batched" else cb.MODE_PLAIN, stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == cb.OK
    want = O.run(primes, cfg["ranges"], dens)["ranges"]
    _check_against(got, want)
    assert got[0]["n_pairs"] == 12231


def test_c1_single_range_call(cb, stream, c1_tables):
    """cuboid_sieve(p_lo, p_hi, q_lo, q_hi) as the paper states the problem."""
    res = cb.cuboid_sieve(c1_tables, 2, 200, 1, 199, cb.Q_LT_P, stream)
    assert cb.cuboid_result_wait(res) == cb.OK
    got = cb.cuboid_result_get(res, 0, 24)
    cb.cuboid_result_free(res)
    want = O.run(W.first_odd_primes(24), [W.triangle(200)])["ranges"][0]
    _check_against([got], [want])


@pytest.mark.parametrize("name", ["c2_as_given.json", "c2_by_density.json", "c2_by_rate.json"])
@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_c2_parity(cb, stream, name, mode):
    g = _golden(name)
    t = cb.cuboid_tables_build(g["primes"], _order_flag(cb, g["by_density"]), stream)
    try:
        assert cb.cuboid_tables_order(t) == g["order"]
        st, got = _run(cb, t, len(g["primes"]), g["ranges"],
                       cb.MODE_BATCHED if mode == "batched" else cb.MODE_PLAIN, stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == cb.OK
    _check_against(got, g["results"])
    assert got[0]["n_pairs"] == 81599337


def test_weak_sieve_every_pair_survives(cb, stream):
    """Primes 3, 5, 7 have all-zero tables: every pair reaches the exact root test."""
    primes = [3, 5, 7]
    ranges = [W.triangle(80), W.rect(1, 40, 1, 40, allow_diagonal=True), W.rect(95, 130, 7, 61)]
    t = cb.cuboid_tables_build(primes, 0, stream)
    try:
        for mode in (cb.MODE_PLAIN, cb.MODE_BATCHED):
            st, got = _run(cb, t, 3, ranges, mode, stream)
            assert st == cb.OK
            want = O.run(primes, ranges)["ranges"]
            _check_against(got, want)
            assert got[1]["roots"] == [(k, k, k * k) for k in range(1, 41)]
    finally:
        cb.cuboid_tables_free(t)


def test_weak_sieve_13(cb, stream):
    primes = [13]
    ranges = [W.triangle(150), W.rect(1, 90, 1, 90, allow_diagonal=True)]
    t = cb.cuboid_tables_build(primes, 0, stream)
    try:
        st, got = _run(cb, t, 1, ranges, cb.MODE_BATCHED, stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == cb.OK
    _check_against(got, O.run(primes, ranges)["ranges"])


def _edge_ranges():
    R = W.rect
    top = (1 << 32) - 1
    return [
        R(5, 5, 3, 3), R(7, 7, 1, 1), R(1, 1, 1, 1, allow_diagonal=True), R(2, 2, 1, 1, q_lt_p=True),
        R(1000, 1000, 1, 4096), R(31, 33, 30, 34), R(63, 65, 1, 200, q_lt_p=True),
        R(1, 300, 97, 97), R(100, 101, 1, 1 << 14), R(1 << 16, (1 << 16) + 3, 1, 70000, q_lt_p=True),
        R(top - 40, top, top - 70, top), R(top - 2, top, 1, 3000), R(4000, 4100, top - 500, top),
        R(999983, 999983, 999000, 1000100, allow_diagonal=True),
        R(2 * 3 * 5 * 7 * 11 * 13 * 17 * 19 * 23, 2 * 3 * 5 * 7 * 11 * 13 * 17 * 19 * 23, 1, 5000),
        R(65521 * 65519, 65521 * 65519, 65000, 66000),
        R(4294967294, 4294967294, 1, 3000), R(200, 260, 1, 5000, q_lt_p=True),
        R(61, 61, 1, 20000), R(122, 122, 1, 20000), R(61 * 67, 61 * 67, 1, 20000), R(183, 183, 1, 9000),
        R(4294967291, 4294967291, 1, 70000), R(2 * 2147483647, 2 * 2147483647, 65536, 140000), R(1, 5000, 200, 210), R(3, 3000, 2, 3001, q_lt_p=True, allow_diagonal=True),
    ]


@pytest.mark.parametrize("rows", [0, "p", "q"])
def test_edge_and_ragged_ranges(cb, stream, c1_tables, rows):
    primes = W.first_odd_primes(24)
    ranges = []
    for r in _edge_ranges():
        r = dict(r)
        r["flags"] = {0: 0, "p": cb.ROWS_P, "q": cb.ROWS_Q}[rows]
        ranges.append(r)
    st, got = _run(cb, c1_tables, 24, ranges, cb.MODE_BATCHED, stream)
    assert st == cb.OK
    _check_against(got, O.run(primes, ranges)["ranges"])
    st, got2 = _run(cb, c1_tables, 24, ranges, cb.MODE_PLAIN, stream)
    assert st == cb.OK and got2 == got


def test_transposed_rectangles(cb, stream, c1_tables):
    """Reflection symmetry u_r(a, b) = u_r(b, a): swapping the p and q ranges transposes
    the survivors and keeps every count."""
    g = random.Random(7)
    ranges, trans = [], []
    for _ in range(40):
        a, b = g.randint(1, 5000), g.randint(1, 5000)
        h, w = g.randint(1, 300), g.randint(1, 300)
        ranges.append(W.rect(a, a + h, b, b + w))
        trans.append(W.rect(b, b + w, a, a + h))
    st1, g1 = _run(cb, c1_tables, 24, ranges, cb.MODE_BATCHED, stream)
    st2, g2 = _run(cb, c1_tables, 24, trans, cb.MODE_BATCHED, stream)
    assert st1 == st2 == cb.OK
    for x, y in zip(g1, g2):
        assert x["counts"] == y["counts"] and x["n_pairs"] == y["n_pairs"]
        assert sorted((q, p) for p, q in x["survivors"]) == y["survivors"]


@pytest.mark.parametrize("lanes,tpw", [(8, 0), (16, 0), (8, 1), (16, 64), (8, 16)])
def test_lanes_per_row_edge_ranges(cb, stream, lanes, tpw):
    """Rows shared by 8 or 16 lanes (4 or 2 rows a warp): the edge and ragged ranges, the
    small batched rectangles and random row orientations equal the oracle, both forms."""
    primes = W.first_odd_primes(24)
    t = cb.cuboid_tables_build(primes, cb.ORDER_AS_GIVEN, stream)
    try:
        cb.cuboid_tables_set_tuning(t, row_lanes=lanes, tiles_per_warp=tpw)
        ranges = []
        for i, r in enumerate(_edge_ranges()):
            r = dict(r)
            r["flags"] = (0, cb.ROWS_P, cb.ROWS_Q)[i % 3]
            ranges.append(r)
        want = O.run(primes, ranges)["ranges"]
        for mode in (cb.MODE_BATCHED, cb.MODE_PLAIN):
            st, got = _run(cb, t, 24, ranges, mode, stream)
            assert st == cb.OK
            _check_against(got, want)
    finally:
        cb.cuboid_tables_free(t)


TUNINGS = [dict(), dict(block_threads=256, ctas_per_sm=1), dict(block_threads=1024, ctas_per_sm=1),
           dict(smem_primes=1), dict(smem_primes=64, ctas_per_sm=1, block_threads=512),
           dict(tiles_per_warp=1), dict(tiles_per_warp=64, ctas_per_sm=4, block_threads=128),
           dict(hot_primes=0), dict(hot_primes=2), dict(hot_primes=6, smem_primes=10),
           dict(hot_primes=6, smem_primes=3), dict(row_lanes=8), dict(row_lanes=16),
           dict(row_lanes=8, tiles_per_warp=1, block_threads=512, ctas_per_sm=1, hot_primes=5),
           dict(row_lanes=16, tiles_per_warp=64, ctas_per_sm=4, block_threads=128, hot_primes=0),
           dict(row_lanes=8, block_threads=1024, ctas_per_sm=1, hot_primes=6),
           dict(block_threads=320, ctas_per_sm=2), dict(block_threads=640, ctas_per_sm=1, row_lanes=8),
           dict(block_threads=320, ctas_per_sm=2, row_lanes=16, hot_primes=5, tiles_per_warp=1)]


@pytest.mark.parametrize("tune", TUNINGS)
@pytest.mark.parametrize("name", ["c2_as_given.json", "c2_by_rate.json"])
def test_tuning_invariance_c2(cb, stream, tune, name):
    g = _golden(name)
    t = cb.cuboid_tables_build(g["primes"], _order_flag(cb, g["by_density"]), stream)
    try:
        cb.cuboid_tables_set_tuning(t, **tune)
        st, got = _run(cb, t, 64, g["ranges"], cb.MODE_BATCHED, stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == cb.OK
    _check_against(got, g["results"])


def test_c3_small_rectangles_vs_oracle(cb, stream):
    g = _golden("c3_small_rects.json")
    t = cb.cuboid_tables_build(g["primes"], 0, stream)
    try:
        for mode in (cb.MODE_PLAIN, cb.MODE_BATCHED):
            st, got = _run(cb, t, 128, g["ranges"], mode, stream)
            assert st == cb.OK
            _check_against(got, g["results"])
    finally:
        cb.cuboid_tables_free(t)


def _golden_gz(name):
    """A gzip-compressed golden with sparse counts ([[caller index, count], ...])."""
    with gzip.open(os.path.join(GOLDEN, name), "rt") as f:
        g = json.load(f)
    n = len(g["primes"])
    for r in g["results"]:
        c = [0] * n
        for i, v in r.pop("counts_nz"):
            c[i] = v
        r["counts"] = c
    return g


def test_c3_all_rectangles_vs_oracle(cb, stream):
    """All 4096 rectangles of the batched workload (1.05e9 pairs, 128 primes in
    rejection-rate order), element by element against the oracle's stored results, in one
    persistent launch and in 4096 separate launches."""
    g = _golden_gz("c3_all_rects.json.gz")
    cfg = W.c3()
    assert g["ranges"] == cfg["ranges"]
    t = cb.cuboid_tables_build(g["primes"], cb.ORDER_BY_RATE, stream)
    try:
        assert cb.cuboid_tables_order(t) == g["order"]
        st1, a = _run(cb, t, 128, cfg["ranges"], cb.MODE_BATCHED, stream)
        st2, b = _run(cb, t, 128, cfg["ranges"], cb.MODE_PLAIN, stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st1 == st2 == cb.OK
    _check_against(a, g["results"])
    _check_against(b, g["results"])


def test_c5_full_size_queries_vs_oracle(cb, stream):
    """24 queries of the serving distribution at full size (areas up to 2^26, p, q < 2^24,
    128 primes in rejection-rate order) against the oracle's stored results: batched
    together, and one by one."""
    g = _golden_gz("c5_full_queries.json.gz")
    t = cb.cuboid_tables_build(g["primes"], cb.ORDER_BY_RATE, stream)
    try:
        st, a = _run(cb, t, 128, g["ranges"], cb.MODE_BATCHED, stream)
        assert st == cb.OK
        _check_against(a, g["results"])
        for q, want in zip(g["ranges"], g["results"]):
            st, one = _run(cb, t, 128, [q], cb.MODE_PLAIN, stream)
            assert st == cb.OK
            _check_against(one, [want])
    finally:
        cb.cuboid_tables_free(t)


def test_c4_sampled_rows_rate_order(cb, stream):
    """The 64 seeded C4 rows in the benchmark's order (rejection rate) against the oracle."""
    g = _golden("c4_rows_by_rate.json")
    t = cb.cuboid_tables_build(g["primes"], cb.ORDER_BY_RATE, stream)
    try:
        assert cb.cuboid_tables_order(t) == g["order"]
        st, got = _run(cb, t, 256, g["ranges"], cb.MODE_BATCHED, stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == cb.OK
    _check_against(got, g["results"])


def test_c4_sampled_rows(cb, stream):
    g = _golden("c4_rows.json")
    t = cb.cuboid_tables_build(g["primes"], 0, stream)
    try:
        st, got = _run(cb, t, 256, g["ranges"], cb.MODE_BATCHED, stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == cb.OK
    _check_against(got, g["results"])


def _phi_sum(n):
    phi = np.arange(n + 1, dtype=np.int64)
    for i in range(2, n + 1):
        if phi[i] == i:
            phi[i::i] -= phi[i::i] // i
    return int(phi[2:].sum())


def test_c4_full_triangle_totals(cb, stream):
    """The full 1 <= q < p <= 2^20 triangle with 256 primes: pairs = sum of phi(p), every
    pair accounted for, and the same counts under two kernel shapes."""
    cfg = W.c4()
    t = cb.cuboid_tables_build(cfg["primes"], 0, stream)
    try:
        st, a = _run(cb, t, 256, cfg["ranges"], cb.MODE_BATCHED, stream)
        cb.cuboid_tables_set_tuning(t, block_threads=256, ctas_per_sm=4, smem_primes=40, tiles_per_warp=2)
        st2, b = _run(cb, t, 256, cfg["ranges"], cb.MODE_PLAIN, stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == st2 == cb.OK
    assert a == b
    x = a[0]
    assert x["n_pairs"] == _phi_sum(1 << 20)
    assert sum(x["counts"]) + len(x["survivors"]) == x["n_pairs"]
    assert x["survivors"] == []


# ---------------------------------------------------------------- K4 on given pairs

def test_verify_pairs_diagonal_and_large(cb, stream):
    ks = list(range(1, 60)) + [1 << 20, (1 << 20) - 3, (1 << 31) + 11, (1 << 32) - 1, 4294967291]
    got = cb.cuboid_verify_pairs(ks, ks, stream)
    assert got == sorted((k, k, k * k) for k in ks)


def test_verify_pairs_vs_oracle(cb, stream):
    g = random.Random(11)
    pairs = [(p, q) for p in range(1, 30) for q in range(1, 30)]
    pairs += [(g.randint(1, 5000), g.randint(1, 5000)) for _ in range(300)]
    pairs += [(l * a, l * b) for (a, b) in [(2, 3), (5, 7), (1, 4)] for l in (6, 30, 210)]
    pairs += [(g.randint(1, (1 << 32) - 1), g.randint(1, (1 << 32) - 1)) for _ in range(4)]
    pairs += [(1, (1 << 32) - 1), ((1 << 32) - 1, 1), (65536, 65535)]
    got = cb.cuboid_verify_pairs([p for p, _ in pairs], [q for _, q in pairs], stream)
    want = sorted((p, q, t) for p, q in pairs for t in O.integer_roots(p, q))
    assert got == want


# ---------------------------------------------------------------- contract and status codes

def test_survivor_overflow_keeps_counts(cb, stream):
    primes = [3, 5, 7]
    t = cb.cuboid_tables_build(primes, 0, stream)
    try:
        st, got = _run(cb, t, 3, [W.triangle(100)], cb.MODE_BATCHED, stream, surv_cap=100)
    finally:
        cb.cuboid_tables_free(t)
    assert st == cb.EOVERFLOW
    want = O.run(primes, [W.triangle(100)])["ranges"][0]
    assert got[0]["n_pairs"] == want["n_pairs"] and got[0]["counts"] == want["counts"]


def test_status_codes(cb, stream, c1_tables):
    lib = cb._lib
    for bad in ([4], [11, 11], [9697], [1], [], [2] * 1025, W.primes_between(11, 10600)):
        with pytest.raises(cb.CuboidError) as e:
            cb.cuboid_tables_build(bad, 0, stream)
        assert e.value.status == cb.EINVAL
    for args in ((0, 5, 1, 5), (5, 4, 1, 5), (1, 5, 0, 5), (1, 5, 6, 5)):
        with pytest.raises(cb.CuboidError) as e:
            cb.cuboid_sieve(c1_tables, *args, 0, stream)
        assert e.value.status == cb.ERANGE
    with pytest.raises(cb.CuboidError) as e:
        cb.cuboid_sieve(c1_tables, 1, 5, 1, 5, cb.ROWS_P | cb.ROWS_Q, stream)
    assert e.value.status == cb.EINVAL
    srv = cb.cuboid_server_create(c1_tables, 0, 64)
    try:
        assert cb.cuboid_tables_free(c1_tables) == cb.EBUSY
    finally:
        assert cb.cuboid_server_destroy(srv, 10000) == cb.OK
    assert lib.cuboid_result_get(None, 0, None, None, None, None, None, None) == cb.EINVAL


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_device_resident_ranges_modes(cb, stream, c1_tables, mode):
    """Plain launches read the caller's device ranges in place, batched ones copy them;
    both equal the oracle, twice in a row on the same result."""
    import torch
    ranges = [W.triangle(200), W.rect(300, 400, 1, 800), W.rect(7, 7, 1, 5000)]
    arr = cb.ranges_array(ranges)
    dev = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).cuda()
    m = cb.MODE_PLAIN if mode == "plain" else cb.MODE_BATCHED
    want = O.run(W.first_odd_primes(24), ranges)["ranges"]
    res = cb.cuboid_result_create(c1_tables, 3)
    try:
        for _ in range(2):
            cb.cuboid_sieve_device(res, dev.data_ptr(), 3, m, stream)
            cb.cuboid_result_download(res, stream)
            assert cb.cuboid_result_wait(res) == cb.OK
            _check_against([cb.cuboid_result_get(res, i, 24) for i in range(3)], want)
    finally:
        cb.cuboid_result_free(res)


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_sieve_timing_events(cb, stream, c1_tables, mode):
    """CUBOID_MODE_TIME_SIEVE times the sieve launches in both forms (inside the captured
    graph through event-record nodes) without changing the results."""
    rng = [W.triangle(3000), W.rect(100, 900, 1, 4000)]
    m = (cb.MODE_PLAIN if mode == "plain" else cb.MODE_BATCHED) | cb.MODE_TIME_SIEVE
    res = cb.cuboid_result_create(c1_tables, 2)
    try:
        cb.cuboid_sieve_into(res, rng, m, stream)
        assert cb.cuboid_result_wait(res) == cb.OK
        ms, launches = cb.cuboid_result_sieve_ms(res)
        got = [cb.cuboid_result_get(res, i, 24) for i in range(2)]
    finally:
        cb.cuboid_result_free(res)
    assert launches == (2 if mode == "plain" else 1)
    assert 0.0 < ms < 1000.0
    _check_against(got, O.run(W.first_odd_primes(24), rng)["ranges"])


def test_device_resident_ranges(cb, stream, c1_tables):
    import torch
    ranges = [W.triangle(200), W.rect(300, 400, 1, 800)]
    arr = cb.ranges_array(ranges)
    dev = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).cuda()
    res = cb.cuboid_result_create(c1_tables, 2)
    try:
        cb.cuboid_sieve_device(res, dev.data_ptr(), 2, cb.MODE_BATCHED, stream)
        cb.cuboid_result_download(res, stream)
        assert cb.cuboid_result_wait(res) == cb.OK
        got = [cb.cuboid_result_get(res, i, 24) for i in range(2)]
    finally:
        cb.cuboid_result_free(res)
    _check_against(got, O.run(W.first_odd_primes(24), ranges)["ranges"])


def test_count_steps_instrumentation(cb, stream, c1_tables):
    rng = [W.triangle(2000)]
    res = cb.cuboid_result_create(c1_tables, 1)
    try:
        cb.cuboid_sieve_into(res, rng, cb.MODE_BATCHED | cb.MODE_COUNT_STEPS, stream)
        assert cb.cuboid_result_wait(res) == cb.OK
        got = cb.cuboid_result_get(res, 0, 24)
        s = cb.cuboid_result_stats(res)
    finally:
        cb.cuboid_result_free(res)
    _check_against([got], O.run(W.first_odd_primes(24), rng)["ranges"])
    assert s["words"] > 0 and s["tiles"] > 0
    assert s["words"] <= s["word_steps"] <= 32 * s["warp_steps"]


def test_repeat_is_deterministic(cb, stream, c1_tables):
    rng = [W.rect(1, 3000, 1, 3000, q_lt_p=True), W.rect(5000, 6000, 1, 20)]
    a = _run(cb, c1_tables, 24, rng, cb.MODE_BATCHED, stream)
    b = _run(cb, c1_tables, 24, rng, cb.MODE_BATCHED, stream)
    assert a == b


def test_deep_primes_near_eq_2_7_bound(cb, stream):
    """Primes up to the largest the table bound below Eq. 2.7 allows (9689 < 9697): the
    reduced tables equal the oracle's, and sieving with the large primes first equals
    the oracle on long rows."""
    primes = [9689, 9679, 9677, 7919, 4999, 11, 13, 17]
    t = cb.cuboid_tables_build(primes, cb.ORDER_AS_GIVEN, stream)
    try:
        for i, r in enumerate(primes[:3]):
            assert cb.cuboid_tables_copy_reduced(t, i, r) == bytes(O.reduced_table(r))
        ranges = [W.rect(100000, 100003, 1, 200000), W.rect(9689 * 7, 9689 * 7, 1, 100000),
                  W.rect(1, 30000, 9677, 9679)]
        T = O.Tables(primes, full_limit=0)
        want = O.run(primes, ranges, tables=T)["ranges"]
        for mode in (cb.MODE_BATCHED, cb.MODE_PLAIN):
            st, got = _run(cb, t, len(primes), ranges, mode, stream, surv_cap=1 << 20)
            assert st == cb.OK
            _check_against(got, want)
    finally:
        cb.cuboid_tables_free(t)


def test_every_prime_below_eq_2_7_bound(cb, stream):
    """All 1192 primes from 11 to 9689 (every prime the bound below Eq. 2.7 admits), 4.4 GB
    of window rows.  Ascending order: the table at the highest offset (r = 9689) has the
    oracle's bits (sampled: the reduced-table lookup and Definition 1.1 pair by pair); the
    first ten primes' counts and survivors equal the oracle's sieve with those ten, and
    every survivor of the ten meets the remaining primes in order through Definition 1.1
    evaluated pair by pair, which fixes the deep counts and the final survivors exactly.
    Descending order: the deepest primes are tried first, from global memory (no shared-
    memory prefix holds a 12 MB table); every pair's first rejecter by Definition 1.1."""
    primes = W.primes_between(11, 9696)
    assert len(primes) == 1192 and primes[-1] == 9689
    ranges = [W.rect(100000, 100030, 1, 60000), W.rect(9689 * 3, 9689 * 3 + 2, 9677, 200000)]
    t = cb.cuboid_tables_build(primes, cb.ORDER_AS_GIVEN, stream)
    try:
        n, dev_bytes, _ = cb.cuboid_tables_info(t)
        assert n == 1192 and dev_bytes > 4 * 10 ** 9
        r = primes[-1]
        blob = cb.cuboid_tables_copy_bits(t, len(primes) - 1)
        assert len(blob) == (r * r + 7) // 8
        st, got = _run(cb, t, len(primes), ranges, cb.MODE_PLAIN, stream, surv_cap=1 << 20)
    finally:
        cb.cuboid_tables_free(t)
    bit = lambda a, b: (blob[(a * r + b) >> 3] >> ((a * r + b) & 7)) & 1
    T1 = O.Tables([r], full_limit=0)
    g = random.Random(7)
    for _ in range(3000):
        a, b = g.randrange(r), g.randrange(r)
        assert bit(a, b) == T1.bit(0, a, b)
    for _ in range(12):
        a, b = g.randrange(r), g.randrange(r)
        assert bit(a, b) == (0 if O.is_solvable(a, b, r) else 1)
    assert st == cb.OK
    k = 10
    T = O.Tables(primes[:k])
    for res, rng in zip(got, ranges):
        n_pairs, c_pre, surv_pre = O.sieve_range(T, rng)
        want = c_pre + [0] * (len(primes) - k)
        want_surv = []
        for (p, q) in surv_pre:
            for i in range(k, len(primes)):
                if not O.is_solvable(p % primes[i], q % primes[i], primes[i]):
                    want[i] += 1
                    break
            else:
                want_surv.append((p, q))
        assert surv_pre and sum(want[k:]) > 0
        assert res["n_pairs"] == n_pairs and res["counts"] == want
        assert sorted(res["survivors"]) == sorted(want_surv)

    desc = primes[::-1]
    rng = W.rect(10 ** 6, 10 ** 6 + 1, 1, 45)
    t = cb.cuboid_tables_build(desc, cb.ORDER_AS_GIVEN, stream)
    try:
        st, (res,) = _run(cb, t, len(desc), [rng], cb.MODE_PLAIN, stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == cb.OK
    want = [0] * len(desc)
    pairs = list(O.pairs_in_range(rng))
    for (p, q) in pairs:
        i = next(i for i, rr in enumerate(desc) if not O.is_solvable(p % rr, q % rr, rr))
        want[i] += 1
    assert res["n_pairs"] == len(pairs) and res["counts"] == want and res["survivors"] == []


def test_staging_wait_gives_up_and_reports(cb, stream, c1_tables):
    """Failure detection without a fault: with CUBOID_MODE_STAGE_TIMEOUT every CTA's
    bounded wait for its shared-memory staging gives up at once; the run reports
    ETIMEOUT, and the next run on the same result and context is exact again."""
    rng = [W.triangle(2000)]
    res = cb.cuboid_result_create(c1_tables, 1)
    try:
        cb.cuboid_sieve_into(res, rng, cb.MODE_PLAIN | cb.MODE_STAGE_TIMEOUT, stream)
        assert cb.cuboid_result_wait(res) == cb.ETIMEOUT
        with pytest.raises(cb.CuboidError):
            cb.cuboid_sieve_into(res, rng, cb.MODE_BATCHED | cb.MODE_STAGE_TIMEOUT, stream)
        cb.cuboid_sieve_into(res, rng, cb.MODE_PLAIN, stream)
        assert cb.cuboid_result_wait(res) == cb.OK
        got = cb.cuboid_result_get(res, 0, 24)
    finally:
        cb.cuboid_result_free(res)
    _check_against([got], O.run(W.first_odd_primes(24), rng)["ranges"])


def test_single_range_result_alternating_forms(cb, stream, c1_tables):
    """A one-range result alternates between the plan-free single-range run (two result
    blocks, each cleared by the other run's root test) and the planned forms; every run
    equals the oracle, including after a run whose staging gave up."""
    import torch
    rngs = [W.triangle(1500), W.rect(700, 900, 1, 3000), W.rect(5, 5, 1, 100000)]
    want = [O.run(W.first_odd_primes(24), [r])["ranges"][0] for r in rngs]
    dev = [torch.frombuffer(bytearray(bytes(cb.ranges_array([r]))), dtype=torch.uint8).cuda() for r in rngs]
    res = cb.cuboid_result_create(c1_tables, 1)
    try:
        seq = [("host", cb.MODE_PLAIN), ("host", cb.MODE_BATCHED), ("dev", cb.MODE_PLAIN),
               ("host", cb.MODE_PLAIN | cb.MODE_STAGE_TIMEOUT), ("host", cb.MODE_PLAIN),
               ("dev", cb.MODE_BATCHED), ("host", cb.MODE_PLAIN | cb.MODE_COUNT_STEPS),
               ("dev", cb.MODE_PLAIN | cb.MODE_TIME_SIEVE), ("host", cb.MODE_PLAIN)]
        for i, (src, mode) in enumerate(seq):
            k = i % 3
            if src == "host":
                cb.cuboid_sieve_into(res, [rngs[k]], mode, stream)
            else:
                cb.cuboid_sieve_device(res, dev[k].data_ptr(), 1, mode, stream)
                cb.cuboid_result_download(res, stream)
            st = cb.cuboid_result_wait(res)
            if mode & cb.MODE_STAGE_TIMEOUT:
                assert st == cb.ETIMEOUT
                continue
            assert st == cb.OK, (i, src, mode)
            _check_against([cb.cuboid_result_get(res, 0, 24)], [want[k]])
    finally:
        cb.cuboid_result_free(res)


def test_multi_range_result_alternating_single_and_batched(cb, stream, c1_tables):
    """A three-range result alternates single-range runs (plan-free, two blocks) with
    batched and plain three-range runs; every run equals the oracle."""
    rngs = [W.triangle(1200), W.rect(700, 900, 1, 3000), W.rect(5, 5, 1, 100000)]
    want = O.run(W.first_odd_primes(24), rngs)["ranges"]
    res = cb.cuboid_result_create(c1_tables, 3)
    try:
        seq = [[0], rngs, [1], [2], rngs, [0], "plain3", [1]]
        for item in seq:
            if item == "plain3":
                cb.cuboid_sieve_into(res, rngs, cb.MODE_PLAIN, stream)
                assert cb.cuboid_result_wait(res) == cb.OK
                _check_against([cb.cuboid_result_get(res, i, 24) for i in range(3)], want)
            elif item is rngs:
                cb.cuboid_sieve_into(res, rngs, cb.MODE_BATCHED, stream)
                assert cb.cuboid_result_wait(res) == cb.OK
                _check_against([cb.cuboid_result_get(res, i, 24) for i in range(3)], want)
            else:
                k = item[0]
                cb.cuboid_sieve_into(res, [rngs[k]], cb.MODE_PLAIN, stream)
                assert cb.cuboid_result_wait(res) == cb.OK
                _check_against([cb.cuboid_result_get(res, 0, 24)], [want[k]])
    finally:
        cb.cuboid_result_free(res)


@pytest.mark.parametrize("lanes", [8, 16])
def test_grouped_rows_many_short_ranges(cb, stream, c1_tables, lanes):
    """Thousands of one-row ranges with 8 or 16 lanes per row: the pair totals of every row
    equal the oracle's, three times over (groups that idle at the end of a range must
    leave no state behind for the rows their warp sieves next)."""
    rows = [W.rect(x, x, 2, 3001, q_lt_p=True, allow_diagonal=True) for x in range(3, 3001)]
    for i, r in enumerate(rows):
        r["flags"] = (cb.ROWS_P, 0)[i % 2]
    want = [len(O.row_pairs(r["p_lo"], r)) for r in rows]
    t = cb.cuboid_tables_build(W.first_odd_primes(24), cb.ORDER_AS_GIVEN, stream)
    try:
        cb.cuboid_tables_set_tuning(t, row_lanes=lanes)
        for _ in range(3):
            res = cb.cuboid_result_create(t, len(rows))
            try:
                cb.cuboid_sieve_into(res, rows, cb.MODE_BATCHED, stream)
                assert cb.cuboid_result_wait(res) == cb.OK
                got = [cb.cuboid_result_get(res, i, 24)["n_pairs"] for i in range(len(rows))]
            finally:
                cb.cuboid_result_free(res)
            assert got == want
    finally:
        cb.cuboid_tables_free(t)
