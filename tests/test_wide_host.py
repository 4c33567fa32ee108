"""Host logic of 64-bit ranges (CPU, no CUDA call): the cut of a range into pieces and the
Theorem 1.1 flags of 64-bit roots.

Section 6 bounds the paper's 32-bit code at p_max = 2^32 / 59; the library's 64-bit ranges
keep the row coordinate below 2^32 and cut the other into 32-bit pieces relative to
64-bit bases.  The pieces must hold exactly the pairs of the range: same rows, the y
values split into disjoint consecutive intervals, every relative bound in 32 bits, and
the q < p restriction decided per piece.
"""
import random

import pytest

import oracle as O

TWO32 = 1 << 32


@pytest.fixture(scope="module")
def cb():
    import paper_1601_00636_gb300 as cb
    return cb


def _absolute(cb, rng):
    """(rows, [(y_lo, y_hi, flags)]) of the pieces in absolute coordinates."""
    pieces = cb.cuboid_wide_pieces(rng)
    rows, ys = None, []
    for pc, bp, bq in pieces:
        rows_q = bool(pc["flags"] & cb.ROWS_Q)
        assert bool(pc["flags"] & cb.ROWS_P) != rows_q or (bp == bq == 0 and not pc["flags"] & (cb.ROWS_P | cb.ROWS_Q))
        for v in (pc["p_lo"], pc["p_hi"], pc["q_lo"], pc["q_hi"]):
            assert 1 <= v < TWO32
        if rows_q:
            assert bq == 0
            x, y, base = (pc["q_lo"], pc["q_hi"]), (pc["p_lo"], pc["p_hi"]), bp
        else:
            assert bp == 0
            x, y, base = (pc["p_lo"], pc["p_hi"]), (pc["q_lo"], pc["q_hi"]), bq
        if base:
            assert base % 64 == 0 and base >= TWO32 - 64 and 64 <= y[0] < 128
            assert not pc["flags"] & (cb.Q_LT_P | cb.ALLOW_DIAGONAL)
        rows = x if rows is None else rows
        assert rows == x
        ys.append((y[0] + base, y[1] + base, pc["flags"]))
    return rows, ys


@pytest.mark.parametrize("seed", range(6))
def test_pieces_partition_the_range(cb, seed):
    g = random.Random(seed)
    for _ in range(60):
        rows_p = g.random() < 0.5
        x_lo = g.randrange(1, TWO32 - 1000)
        x_hi = x_lo + g.randrange(0, 1000)
        y_lo = g.choice([g.randrange(1, TWO32), g.randrange(TWO32, 1 << 39)])
        y_hi = min(y_lo + g.choice([0, 63, 64, 5000, TWO32 - 65, TWO32 - 64, 3 * TWO32 + 17]), (1 << 40) - 1)
        tri = g.random() < 0.3
        rng = ({"p_lo": x_lo, "p_hi": x_hi, "q_lo": y_lo, "q_hi": y_hi} if rows_p
               else {"p_lo": y_lo, "p_hi": y_hi, "q_lo": x_lo, "q_hi": x_hi})
        rng["q_lt_p"] = tri
        if y_hi < TWO32:
            rng["flags"] = cb.ROWS_P if rows_p else cb.ROWS_Q
        rows, ys = _absolute(cb, rng)
        # the y values kept: all of [y_lo, y_hi], except that q < p (rows of p) drops y >= 2^32
        keep_hi = min(y_hi, TWO32 - 1) if (tri and rows_p) else y_hi
        if y_lo > keep_hi:
            assert ys == []
            continue
        assert rows == (x_lo, x_hi)
        assert ys[0][0] == y_lo and ys[-1][1] == keep_hi
        for (a0, a1, _), (b0, b1, _) in zip(ys, ys[1:]):
            assert a1 + 1 == b0 and a0 <= a1
        for a0, a1, fl in ys:
            assert (a1 < TWO32) == (a0 < TWO32)           # no piece straddles 2^32
            if a0 < TWO32:
                assert bool(fl & cb.Q_LT_P) == tri          # the 32-bit piece keeps the restriction
        # pieces above 2^32 hold at most 2^32 - 64 values
        assert all(a1 - a0 + 1 <= TWO32 - 64 for a0, a1, _ in ys if a0 >= TWO32)


def test_32bit_range_is_one_piece(cb):
    rng = {"p_lo": 5, "p_hi": 900, "q_lo": 7, "q_hi": 70000, "q_lt_p": True, "allow_diagonal": True}
    ((pc, bp, bq),) = cb.cuboid_wide_pieces(rng)
    assert (bp, bq) == (0, 0)
    assert (pc["p_lo"], pc["p_hi"], pc["q_lo"], pc["q_hi"]) == (5, 900, 7, 70000)
    assert pc["flags"] == cb.Q_LT_P | cb.ALLOW_DIAGONAL


def test_rows_follow_the_32bit_coordinate(cb):
    (pc, bp, bq), = cb.cuboid_wide_pieces({"p_lo": TWO32 + 5, "p_hi": TWO32 + 9, "q_lo": 3, "q_hi": 4})
    assert pc["flags"] == cb.ROWS_Q and bq == 0 and bp + pc["p_lo"] == TWO32 + 5
    (pc, bp, bq), = cb.cuboid_wide_pieces({"p_lo": 3, "p_hi": 4, "q_lo": TWO32 + 5, "q_hi": TWO32 + 9})
    assert pc["flags"] == cb.ROWS_P and bp == 0 and bq + pc["q_lo"] == TWO32 + 5
    # q < p with rows of q and every p above 2^32: the restriction holds everywhere
    (pc, bp, bq), = cb.cuboid_wide_pieces({"p_lo": TWO32, "p_hi": TWO32 + 9, "q_lo": 3, "q_hi": 4, "q_lt_p": True})
    assert pc["flags"] == cb.ROWS_Q
    # q < p with rows of p and every q above 2^32: nothing is left
    assert cb.cuboid_wide_pieces({"p_lo": 3, "p_hi": 4, "q_lo": TWO32, "q_hi": TWO32 + 9, "q_lt_p": True}) == []


@pytest.mark.parametrize("rng,code", [
    ({"p_lo": 0, "p_hi": 4, "q_lo": 1, "q_hi": 2}, "ERANGE"),
    ({"p_lo": 5, "p_hi": 4, "q_lo": 1, "q_hi": 2}, "ERANGE"),
    ({"p_lo": 1, "p_hi": 4, "q_lo": 1, "q_hi": 1 << 40}, "ERANGE"),
    ({"p_lo": TWO32, "p_hi": TWO32, "q_lo": TWO32, "q_hi": TWO32}, "ERANGE"),
    ({"p_lo": 1, "p_hi": TWO32, "q_lo": 1, "q_hi": TWO32}, "ERANGE"),
    ({"p_lo": 1, "p_hi": 2, "q_lo": TWO32, "q_hi": TWO32 + 1, "flags": 8}, "ERANGE"),   # rows of q forced
    ({"p_lo": 1, "p_hi": 2, "q_lo": 1, "q_hi": 2, "flags": 0x10}, "EINVAL"),
    ({"p_lo": 1, "p_hi": 2, "q_lo": 1, "q_hi": 2, "flags": 0xC}, "EINVAL"),
    ({"p_lo": 1, "p_hi": 2, "q_lo": 1, "q_hi": 2, "reserved": 1}, "EINVAL"),
])
def test_piece_errors(cb, rng, code):
    with pytest.raises(cb.CuboidError) as e:
        cb.cuboid_wide_pieces(rng)
    assert e.value.status == getattr(cb, code)


def test_theorem11_wide_matches_oracle(cb):
    """Theorem 1.1 in 256-bit integers at p, q near 2^40 and t near the window's edges."""
    g = random.Random(5)
    roots = []
    for _ in range(400):
        p = g.randrange(1, 1 << 40)
        q = g.randrange(1, 1 << 40)
        base = max(p * p, p * q, q * q)
        t = base + g.choice([-1, 0, 1, g.randrange(1, 1 << 20), base, 2 * base, 3 * base, 4 * base])
        t = max(t, 0)
        if t >= 1 << 128:
            continue
        roots.append((p, q, t))
    flags = cb.cuboid_theorem11_flags_wide(roots)
    assert flags == [O.theorem_1_1_holds(*r) for r in roots]
    assert any(flags) and not all(flags)
    with pytest.raises(cb.CuboidError):
        cb.cuboid_theorem11_flags_wide([(1 << 40, 1, 5)])


def test_device_root_bound_covers_oracle_bound():
    """The root test isolates the roots of R(u) = Q(sqrt u) in [0, 45 M^4], M = max(p, q);
    for pairs up to 2^40 (64-bit ranges) that interval holds the oracle's bound on every
    positive root, and 45 M^4 stays below the 2^166 the device's three 64-bit limbs use."""
    g = random.Random(17)
    cases = [(1, 1), (2, 1), (1, 2), ((1 << 40) - 1, 1), (1, (1 << 40) - 1), ((1 << 40) - 1, (1 << 40) - 1)]
    cases += [(g.randrange(1, 1 << 40), g.randrange(1, 1 << 40)) for _ in range(300)]
    for p, q in cases:
        M = max(p, q)
        assert O.root_bound_u(p, q) <= 45 * M ** 4 < 1 << 166
