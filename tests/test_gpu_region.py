"""GPU: the region search of section 5 (Theorem 1.2, Eq. 5.1/5.2) through the C ABI.

The synchronous scan must equal the oracle's region scan row block by row block (pairs,
per-prime counts, survivors, roots, depth and r_max, bit-exact); the asynchronous search
(start / current / stop / resume) must add up to the synchronous scan of the same rows;
the start call must give the six return codes of section 5; and the scan of p <= 154000
with the 96 primes 11..541 must reproduce section 6: no survivor, deepest prime 137.
"""
import time

import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


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


def _tables(cb, primes, flags):
    return cb.cuboid_tables_build(primes, flags)


def _compare(got, want, primes_order):
    st, rep, counts, surv, roots = got
    assert st == 0
    assert rep["pairs"] == want["pairs"]
    assert counts == want["counts"]
    assert sorted(surv) == sorted(want["survivors"])
    assert rep["n_surv"] == len(want["survivors"])
    assert sorted(roots) == want["roots"] and rep["n_roots"] == len(want["roots"])
    assert (rep["depth"], rep["r_max"]) == (want["depth"], want["r_max"])


@pytest.mark.parametrize("order", ["given", "rate"])
def test_region_rows_1_to_1000(cb, stream, order):
    """Rows 1..1000: Eq. 5.1 below 152, Eq. 5.2 above, batch edges at every hundred."""
    primes = W.primes_between(11, 53)
    flag = cb.ORDER_AS_GIVEN if order == "given" else cb.ORDER_BY_RATE
    T = O.Tables(primes, by_density={"given": False, "rate": "rate"}[order])
    want = O.region_scan(T, 1, 1000)
    assert want["survivors"]                       # the survivor path is exercised
    t = _tables(cb, primes, flag)
    try:
        got = cb.cuboid_region_scan(t, 1, 1000, stream=stream)
        _compare(got, want, T.order)
        rep = got[1]
        assert (rep["p"], rep["q"]) == (1001, O.region_q_bounds(1001)[0])
    finally:
        cb.cuboid_tables_free(t)


@pytest.mark.parametrize("p_from,q_from,p_to", [(152, 100, 310), (151, 8000, 153), (199, 3, 201),
                                                (1, 30, 1), (250, 14750, 250)])
def test_region_mid_row_starts(cb, stream, p_from, q_from, p_to):
    """A scan resumed inside a row starts at q_from; rows after it start at their q_lo."""
    primes = W.primes_between(11, 61)
    T = O.Tables(primes)
    want = O.region_scan(T, p_from, p_to, q_from)
    t = _tables(cb, primes, cb.ORDER_AS_GIVEN)
    try:
        _compare(cb.cuboid_region_scan(t, p_from, p_to, q_from=q_from, stream=stream), want, T.order)
    finally:
        cb.cuboid_tables_free(t)


def test_region_scan_errors(cb, stream):
    t = _tables(cb, W.primes_between(11, 31), cb.ORDER_AS_GIVEN)
    try:
        for args, code in [((0, 5), cb.ERANGE), ((10, 9), cb.ERANGE), ((5, 72796056), cb.EPMAX)]:
            with pytest.raises(cb.CuboidError) as e:
                cb.cuboid_region_scan(t, *args, stream=stream)
            assert e.value.status == code
        with pytest.raises(cb.CuboidError) as e:
            cb.cuboid_region_scan(t, 152, 160, q_from=2, stream=stream)
        assert e.value.status == cb.EQLOW
        with pytest.raises(cb.CuboidError) as e:
            cb.cuboid_region_scan(t, 152, 160, q_from=59 * 152 + 1, stream=stream)
        assert e.value.status == cb.EQHIGH
    finally:
        cb.cuboid_tables_free(t)


def test_search_return_codes(cb):
    """Section 5's codes of the start call: 0 started, 1 already running (and the tables
    cannot be released meanwhile), 2 p < 152, 3 p > 72796055, 4 q below Eq. 5.2, 5 q
    above 59 p, 6 no tables."""
    t = _tables(cb, W.primes_between(11, 541), cb.ORDER_AS_GIVEN)
    try:
        assert cb.cuboid_search_start_status(None, 152, 3)[0] == 6
        assert cb.cuboid_search_start_status(t, 151, 3)[0] == 2
        assert cb.cuboid_search_start_status(t, 72796056, 5000)[0] == 3
        assert cb.cuboid_search_start_status(t, 152, 2)[0] == 4
        assert cb.cuboid_search_start_status(t, 152, 0)[0] == 4
        assert cb.cuboid_search_start_status(t, 152, 59 * 152 + 1)[0] == 5
        st, s = cb.cuboid_search_start_status(t, 152, 3)
        assert st == 0
        try:
            assert cb.cuboid_search_start_status(t, 152, 3)[0] == 1
            assert cb.cuboid_tables_free(t) == cb.EBUSY
        finally:
            st2, rep, _ = cb.cuboid_search_stop(s, 96)
        assert st2 == 0 and rep["p"] >= 152
    finally:
        assert cb.cuboid_tables_free(t) == 0


def _run_search(cb, t, p, q, until_p, n):
    s = cb.cuboid_search_start(t, p, q)
    deadline = time.time() + 120
    seen = []
    while time.time() < deadline:
        cur, rmax = cb.cuboid_search_current(s)
        seen.append((cur, rmax))
        if cur >= until_p:
            break
        time.sleep(0.02)
    st, rep, counts = cb.cuboid_search_stop(s, n)
    assert st == 0
    return rep, counts, seen


def test_search_stop_resume_equals_scan(cb, stream):
    """Start at (152, 3), stop, resume from the report's (p, q), stop again: the two
    reports add up to the synchronous scan of the same rows, and the progress probe moves
    in steps of 100 rows with r_max no deeper than the list."""
    primes = W.primes_between(11, 541)
    t = _tables(cb, primes, cb.ORDER_AS_GIVEN)
    try:
        rep1, c1, seen = _run_search(cb, t, 152, 3, 3000, len(primes))
        assert rep1["p"] > 152 and rep1["p"] % 100 == 0
        assert rep1["q"] == cb.cuboid_region_qmin(rep1["p"])
        assert all(cur % 100 == 0 for cur, _ in seen)
        assert all(r == 0 or r in primes for _, r in seen)
        rep2, c2, _ = _run_search(cb, t, rep1["p"], rep1["q"], rep1["p"] + 2000, len(primes))
        assert rep2["p"] > rep1["p"]
        st, whole, counts, surv, roots = cb.cuboid_region_scan(t, 152, rep2["p"] - 1, q_from=3, stream=stream)
        assert st == 0
        assert [a + b for a, b in zip(c1, c2)] == counts
        assert rep1["pairs"] + rep2["pairs"] == whole["pairs"]
        assert rep1["n_surv"] + rep2["n_surv"] == whole["n_surv"] == 0
        assert whole["pairs"] == O.region_pair_count(152, rep2["p"] - 1)
    finally:
        cb.cuboid_tables_free(t)


def test_section6_region_to_154000(cb, stream):
    """Section 6: rows p = 1..154000, every q of Eq. 1.2, the 96 primes 11..541 in
    ascending order.  No pair passes the sieve, and the deepest prime needed is the 29th,
    137.  The number of coprime pairs sieved equals the Moebius count of the oracle."""
    primes = W.primes_between(11, 541)
    assert len(primes) == 96 and primes[28] == 137
    t = _tables(cb, primes, cb.ORDER_AS_GIVEN)
    try:
        st, rep, counts, surv, roots = cb.cuboid_region_scan(t, 1, 154000, stream=stream)
        assert st == 0
        assert rep["n_surv"] == 0 and surv == [] and roots == []
        assert rep["pairs"] == O.region_pair_count(1, 154000)
        assert sum(counts) == rep["pairs"]
        assert rep["depth"] <= 29 and rep["r_max"] <= 137
        print(f"section 6 scan: depth {rep['depth']} r_max {rep['r_max']} pairs {rep['pairs']}")
        assert (rep["depth"], rep["r_max"]) == (29, 137)
        # the per-prime counts of the first rows agree with the oracle
        T = O.Tables(primes, full_limit=0)
        st2, rep2, c2, _, _ = cb.cuboid_region_scan(t, 152, 260, stream=stream)
        want = O.region_scan(T, 152, 260)
        assert c2 == want["counts"] and rep2["pairs"] == want["pairs"]
    finally:
        cb.cuboid_tables_free(t)


def test_theorem11_on_found_roots(cb, stream):
    """Roots the device finds (the diagonal pairs p = q, t = p^2, sieved with the diagonal
    allowed) are flagged by Theorem 1.1 exactly as the oracle flags them: none is a cuboid."""
    primes = W.first_odd_primes(6)
    T = O.Tables(primes)
    rng = {"p_lo": 1, "p_hi": 300, "q_lo": 1, "q_hi": 300, "q_lt_p": True, "allow_diagonal": True}
    want = O.run(primes, [rng], tables=T)["ranges"][0]
    assert want["roots"]
    t = _tables(cb, primes, cb.ORDER_AS_GIVEN)
    try:
        res = cb.cuboid_sieve(t, 1, 300, 1, 300, cb.Q_LT_P | cb.ALLOW_DIAGONAL, stream)
        try:
            cb.cuboid_result_wait(res)
            got = cb.cuboid_result_get(res, 0, len(primes))
        finally:
            cb.cuboid_result_free(res)
    finally:
        cb.cuboid_tables_free(t)
    assert sorted(got["roots"]) == want["roots"]
    flags = cb.cuboid_theorem11_flags(got["roots"])
    assert flags == [O.theorem_1_1_holds(*r) for r in got["roots"]] and not any(flags)
    assert got["cuboids"] == []


def test_region_hundred_near_stop_example(cb, stream):
    """The hundred of rows 112600..112699 (the hundred of the stop report printed in
    section 5), every q of Eq. 1.2, primes 11..541 ascending: per-prime counts, pair
    total and depth equal the oracle's stored scan (tests/golden/make_golden.py)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "region_112600_112699.json")))
    t = _tables(cb, g["primes"], cb.ORDER_AS_GIVEN)
    try:
        st, rep, counts, surv, roots = cb.cuboid_region_scan(t, 112600, 112699, stream=stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == 0 and counts == g["counts"] and rep["pairs"] == g["pairs"]
    assert sorted(surv) == [tuple(x) for x in g["survivors"]] and roots == []
    assert (rep["depth"], rep["r_max"]) == (g["depth"], g["r_max"]) == (27, 127)
