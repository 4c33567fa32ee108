"""GPU: 64-bit ranges beyond the 32-bit limit of section 6 (p_max = 2^32 / 59), through
the C ABI, against the oracle.

Small windows are compared pair set by pair set with the oracle's sieve (counts per
prime, pair totals, survivors, roots; bit-exact).  A row whose q span needs three pieces
(more than 2^33 values) is checked by properties that hold at any size: the pair total
equals the oracle's Moebius count, the counts and survivors add up to it, and every
survivor the device reports passes every table prime in the oracle.
"""
import math
import random

import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TWO32 = 1 << 32
P_MAX = 72796055  # section 6: 2^32 / 59


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


def _run(cb, t, ranges, n_primes, stream):
    res = cb.cuboid_sieve_wide(t, ranges, stream=stream)
    try:
        st = cb.cuboid_result_wait(res)
        return st, [cb.cuboid_result_get_wide(res, i, n_primes) for i in range(len(ranges))]
    finally:
        cb.cuboid_result_free(res)


def _compare(got, want):
    assert got["n_pairs"] == want["n_pairs"]
    assert got["counts"] == want["counts"]
    assert got["survivors"] == want["survivors"]
    assert got["roots"] == want["roots"]


def _window_cases():
    return [
        # rows of p just beyond p_max, q across 2^32: a 32-bit piece and one based piece
        W.rect(P_MAX + 1, P_MAX + 4, TWO32 - 3000, TWO32 + 5000),
        # the same rows, q entirely above 2^32 (one based piece, unaligned ends)
        W.rect(P_MAX + 1, P_MAX + 3, TWO32 + 77, TWO32 + 4000),
        # rows of q, p near 2^39 (q prime to p decided from the factors of q)
        W.rect(2 ** 39 - 1500, 2 ** 39 + 700, 1, 30),
        # rows of q with q < p everywhere: the restriction keeps all pairs
        W.rect(2 ** 36 + 5, 2 ** 36 + 2000, 2 ** 31, 2 ** 31 + 12, q_lt_p=True),
        # rows of p, q < p: only the 32-bit piece remains
        W.rect(TWO32 - 9, TWO32 - 1, TWO32 - 400, TWO32 + 400, q_lt_p=True),
        # the diagonal crossing 2^32 - 5 (a prime): roots t = p^2 from the 32-bit piece
        W.rect(TWO32 - 5, TWO32 - 5, TWO32 - 40, TWO32 + 30, allow_diagonal=True),
        # an ordinary 32-bit range through the 64-bit entry point
        W.rect(1000, 1100, 3000, 3400),
    ]


def test_wide_windows_match_oracle(cb, stream):
    primes = W.primes_between(11, 53)
    T = O.Tables(primes)
    ranges = _window_cases()
    t = cb.cuboid_tables_build(primes, cb.ORDER_AS_GIVEN)
    try:
        st, got = _run(cb, t, ranges, len(primes), stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == cb.OK
    for g, rng in zip(got, ranges):
        n_pairs, counts, surv = O.sieve_range(T, rng)
        surv = sorted(surv)
        want = {"n_pairs": n_pairs, "counts": counts, "survivors": surv,
                "roots": sorted((p, q, tt) for (p, q) in surv for tt in O.integer_roots(p, q))}
        _compare(g, want)
    assert got[5]["roots"] == [(TWO32 - 5, TWO32 - 5, (TWO32 - 5) ** 2)]
    assert got[5]["cuboids"] == []


def test_wide_survivor_path_few_primes(cb, stream):
    """Six primes leave many survivors in based pieces (rows of p beyond p_max with q
    above 2^32; rows of q with p near 2^38): survivors and counts are exact; the roots the
    device reports are zeros of Q_pq, and those of a sample of survivors (the oracle's
    divisor search) are among them."""
    primes = W.primes_between(11, 29)
    T = O.Tables(primes)
    ranges = [W.rect(P_MAX + 1, P_MAX + 2, TWO32 + 1, TWO32 + 30000),
              W.rect(2 ** 38, 2 ** 38 + 3000, 7, 20)]
    t = cb.cuboid_tables_build(primes, cb.ORDER_AS_GIVEN)
    try:
        st, got = _run(cb, t, ranges, len(primes), stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == cb.OK
    for g, rng in zip(got, ranges):
        n_pairs, counts, surv = O.sieve_range(T, rng)
        assert (g["n_pairs"], g["counts"], g["survivors"]) == (n_pairs, counts, sorted(surv))
        assert len(surv) > 50
        for (pp, qq, tt) in g["roots"]:
            assert (pp, qq) in set(surv) and O.q_value(pp, qq, tt) == 0
        for (pp, qq) in random.Random(9).sample(surv, 6):
            assert all((pp, qq, tt) in g["roots"] for tt in O.integer_roots(pp, qq))


@pytest.mark.parametrize("order", ["rate", "density"])
def test_wide_rows_of_p_effective_orders(cb, stream, order):
    """Rows p = p_max + 1 .. p_max + 6, q across 2^32, 26 primes in a reordered list."""
    primes = W.primes_between(11, 113)
    flag = cb.ORDER_BY_RATE if order == "rate" else cb.ORDER_BY_DENSITY
    T = O.Tables(primes, by_density=order)
    rng = W.rect(P_MAX + 1, P_MAX + 6, TWO32 - 20000, TWO32 + 20000)
    t = cb.cuboid_tables_build(primes, flag)
    try:
        st, (g,) = _run(cb, t, [rng], len(primes), stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == cb.OK
    n_pairs, counts, surv = O.sieve_range(T, rng)
    assert (g["n_pairs"], g["counts"], g["survivors"]) == (n_pairs, counts, sorted(surv))


def test_wide_row_three_pieces_properties(cb, stream):
    """One row p = p_max + 2 with q from 2^33 - 1000 to 2^34 + 1000 (three based pieces):
    the pair total is the Moebius count, counts and survivors add up to it, every
    reported survivor passes every prime in the oracle and is coprime to p, and the
    pieces' boundaries hold no gap: the same row cut into four ranges by hand gives the
    same totals."""
    p = P_MAX + 2
    primes = W.primes_between(11, 71)  # 16 primes: about 2 10^4 survivors in the row
    T = O.Tables(primes)
    q_lo, q_hi = 2 ** 33 - 1000, 2 ** 34 + 1000
    t = cb.cuboid_tables_build(primes, cb.ORDER_AS_GIVEN)
    try:
        st, (g,) = _run(cb, t, [W.rect(p, p, q_lo, q_hi)], len(primes), stream)
        cuts = [q_lo, 2 ** 33 + 12345, 3 * 2 ** 32 + 64, 3 * 2 ** 32 + 65, q_hi + 1]
        parts = [W.rect(p, p, a, b - 1) for a, b in zip(cuts, cuts[1:])]
        st2, gp = _run(cb, t, parts, len(primes), stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == st2 == cb.OK
    assert g["n_pairs"] == O.coprime_count(p, q_lo, q_hi)
    assert sum(g["counts"]) + len(g["survivors"]) == g["n_pairs"]
    assert sum(x["n_pairs"] for x in gp) == g["n_pairs"]
    assert [sum(c) for c in zip(*[x["counts"] for x in gp])] == g["counts"]
    assert sorted(s for x in gp for s in x["survivors"]) == g["survivors"]
    sample = random.Random(3).sample(g["survivors"], min(400, len(g["survivors"])))
    for (pp, qq) in sample:
        assert pp == p and q_lo <= qq <= q_hi and math.gcd(pp, qq) == 1
        assert not any(T.bit(i, pp, qq) for i in range(len(primes)))
    assert g["survivors"]
    for (pp, qq, tt) in g["roots"]:
        assert O.q_value(pp, qq, tt) == 0


def test_wide_errors(cb, stream):
    t = cb.cuboid_tables_build(W.primes_between(11, 31), cb.ORDER_AS_GIVEN)
    try:
        for rng, code in [(W.rect(TWO32, TWO32 + 1, TWO32, TWO32 + 1), cb.ERANGE),
                          (W.rect(1, 2, 1, 1 << 40), cb.ERANGE),
                          (W.rect(0, 2, 1, 5), cb.ERANGE)]:
            with pytest.raises(cb.CuboidError) as e:
                cb.cuboid_sieve_wide(t, [rng], stream=stream)
            assert e.value.status == code
        # a wide result is read with the wide getter only
        res = cb.cuboid_sieve_wide(t, [W.rect(3, 4, TWO32 + 1, TWO32 + 99)], stream=stream)
        try:
            assert cb.cuboid_result_wait(res) == cb.OK
            with pytest.raises(cb.CuboidError):
                cb.cuboid_result_get(res, 0, 7)
        finally:
            cb.cuboid_result_free(res)
        # an empty range (q < p leaves nothing): zero pairs, no records
        st, (g,) = _run(cb, t, [W.rect(3, 4, TWO32 + 1, TWO32 + 99, q_lt_p=True)], 7, stream)
        assert st == cb.OK and g["n_pairs"] == 0 and g["survivors"] == [] and sum(g["counts"]) == 0
    finally:
        cb.cuboid_tables_free(t)


def test_verify_pairs_wide_matches_oracle(cb, stream):
    """The exact root test at p, q up to 2^40 - 1: the diagonal roots t = k^2 (t up to
    2^80, two 64-bit limbs) and no root for coprime pairs of large primes, as the
    oracle's divisor search finds."""
    ks = [2 ** 40 - 87, 2 ** 39 + 1, TWO32 + 15, 3, 1]
    pairs = [(k, k) for k in ks] + [(2 ** 40 - 87, 2 ** 32 - 5), (2 ** 32 - 5, 2 ** 40 - 87), (2 ** 40 - 87, 1)]
    got = cb.cuboid_verify_pairs_wide([p for p, _ in pairs], [q for _, q in pairs], stream=stream)
    want = sorted((p, q, tt) for p, q in pairs for tt in O.integer_roots(p, q))
    assert got == want
    assert (2 ** 40 - 87, 2 ** 40 - 87, (2 ** 40 - 87) ** 2) in got
    with pytest.raises(cb.CuboidError) as e:
        cb.cuboid_verify_pairs_wide([1 << 40], [3], stream=stream)
    assert e.value.status == cb.ERANGE


# ---------------------------------------------------------------- the region scan past p_max

def test_region_scan_wide_equals_32bit_scan(cb, stream):
    """Below p_max the 64-bit scan equals the 32-bit scan of section 5 (itself checked
    against the oracle's region scan): rows 140..400 across the switch of Eq. 5.1 to
    Eq. 5.2, and the last six rows below p_max whose q reach 2^32 - 1."""
    primes = W.primes_between(11, 61)
    t = cb.cuboid_tables_build(primes, cb.ORDER_AS_GIVEN)
    try:
        for p_from, q_from, p_to in [(140, 0, 400), (P_MAX - 5, 0, P_MAX), (250, 14000, 260)]:
            a = cb.cuboid_region_scan(t, p_from, p_to, q_from=q_from, stream=stream)
            b = cb.cuboid_region_scan_wide(t, p_from, p_to, q_from=q_from, stream=stream)
            assert a[0] == b[0] == cb.OK
            assert a[2] == b[2] and a[3] == b[3] and a[4] == b[4]
            for k in ("pairs", "n_surv", "n_roots", "depth", "r_max", "p"):
                assert a[1][k] == b[1][k], k
            # the 32-bit scan cannot resume past p_max and reports q = 0 there
            assert b[1]["q"] == O.region_q_bounds(p_to + 1)[0]
            assert a[1]["q"] == (b[1]["q"] if p_to < P_MAX else 0)
    finally:
        cb.cuboid_tables_free(t)


def test_region_scan_wide_past_p_max(cb, stream):
    """Rows p_max - 3 .. p_max + 4 with the 96 primes 11..541 ascending (section 6's list):
    the pair total is the oracle's Moebius count of every row's segment of Eq. 1.2, counts
    and survivors add up to it, depth and r_max follow from the counts as the oracle reads
    them, the report points at the next row's first q, the counts equal those of the same
    rows through cuboid_sieve_wide, and a scan stopped at p_max and resumed from the report
    adds up to the whole."""
    primes = W.primes_between(11, 541)
    T = O.Tables(primes, full_limit=0)
    a, b = P_MAX - 3, P_MAX + 4
    t = cb.cuboid_tables_build(primes, cb.ORDER_AS_GIVEN)
    try:
        st, rep, counts, surv, roots = cb.cuboid_region_scan_wide(t, a, b, stream=stream)
        rows = [W.rect(p, p, O.region_q_bounds(p)[0], O.region_q_bounds(p)[1]) for p in range(a, b + 1)]
        st_w, got = _run(cb, t, rows, len(primes), stream)
        st1, rep1, c1, s1, r1 = cb.cuboid_region_scan_wide(t, a, P_MAX, stream=stream)
        st2, rep2, c2, s2, r2 = cb.cuboid_region_scan_wide(t, rep1["p"], b, q_from=rep1["q"], stream=stream)
    finally:
        cb.cuboid_tables_free(t)
    assert st == st_w == st1 == st2 == cb.OK
    want_pairs = sum(O.coprime_count(p, *O.region_q_bounds(p)) for p in range(a, b + 1))
    assert rep["pairs"] == want_pairs == sum(g["n_pairs"] for g in got)
    assert sum(counts) + rep["n_surv"] == rep["pairs"]
    assert counts == [sum(c) for c in zip(*[g["counts"] for g in got])]
    assert sorted(surv) == sorted(s for g in got for s in g["survivors"]) and roots == []
    assert (rep["depth"], rep["r_max"]) == O.deepest_prime(T, counts, rep["n_surv"])
    assert (rep["p"], rep["q"]) == (b + 1, O.region_q_bounds(b + 1)[0])
    assert (rep1["p"], rep1["q"]) == (P_MAX + 1, O.region_q_bounds(P_MAX + 1)[0])
    assert [x + y for x, y in zip(c1, c2)] == counts and rep1["pairs"] + rep2["pairs"] == rep["pairs"]
    assert rows[-1]["q_hi"] > TWO32 > rows[0]["q_hi"]


def test_region_scan_wide_errors(cb, stream):
    t = cb.cuboid_tables_build(W.primes_between(11, 31), cb.ORDER_AS_GIVEN)
    try:
        for args, kw, code in [((0, 5), {}, cb.ERANGE), ((10, 9), {}, cb.ERANGE), ((5, TWO32), {}, cb.ERANGE),
                               ((P_MAX + 10, P_MAX + 11), {"q_from": 3}, cb.EQLOW),
                               ((P_MAX + 10, P_MAX + 11), {"q_from": 59 * (P_MAX + 10) + 1}, cb.EQHIGH)]:
            with pytest.raises(cb.CuboidError) as e:
                cb.cuboid_region_scan_wide(t, *args, stream=stream, **kw)
            assert e.value.status == code
    finally:
        cb.cuboid_tables_free(t)
