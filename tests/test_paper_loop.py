"""The C/OpenMP restatement of the paper's section 5 loop (oracle/paper_loop.c), the timed
CPU baseline, against the paper's printed bytes, the literal C1 results and the Python
oracle (CPU only)."""
import json
import os
import random

import pytest

import oracle as O
import workloads as W
from oracle.paper_loop import PaperLoop

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def loop24():
    return PaperLoop(W.first_odd_primes(24))


def test_u11_bytes_are_the_printed_eq_2_6(loop24):
    """Eq. 2.6: the 16 bytes printed for u_11 (highest bit leftmost)."""
    b = loop24.table_bytes(W.first_odd_primes(24).index(11))
    with open(os.path.join(GOLDEN, "u11_bytes_eq2_6.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(b) == 16
    for idx, bits in rows:
        assert format(b[int(idx)], "08b") == bits


def test_packed_tables_equal_brute_force_definition():
    """Definition 1.1 by trying every t (the oracle's full tables) for every r <= 313."""
    primes = W.first_odd_primes(64)
    L = PaperLoop(primes)
    for i, r in enumerate(primes):
        if r > 200:  # the slow oracle tables above 200 are pinned by the reduced-vs-full test
            break
        assert L.table_bytes(i) == O.pack_table_bytes(O.unsolvable_table(r)), r


def test_c1_literal(loop24):
    """C1 in the paper's ascending order: 12,231 pairs, no survivor, and the first-rejecter
    counts 11:8153 13:1164 17:1940 19:612 23:255 29:75 31:19 37:8 41:3 43:2."""
    from test_oracle_pins import C1_COUNTS, C1_PAIRS
    primes = W.first_odd_primes(24)
    n, counts, surv = loop24.sieve(list(range(24)), W.triangle(200))
    assert n == C1_PAIRS and surv == []
    assert counts == [C1_COUNTS.get(r, 0) for r in primes]


@pytest.mark.parametrize("mode", [False, True, "rate"])
def test_matches_oracle_on_rectangles(mode):
    primes = W.first_odd_primes(24)
    L = PaperLoop(primes)
    T = O.Tables(primes, mode)
    g = random.Random(7)
    ranges = [W.triangle(300), W.rect(300, 340, 1, 700), W.rect(1, 50, 1, 3000)]
    for _ in range(6):
        p, q = g.randint(1, 1 << 20), g.randint(1, 1 << 20)
        ranges.append(W.rect(p, p + g.randint(0, 20), q, q + g.randint(0, 2000), q_lt_p=g.random() < 0.5))
    for rng in ranges:
        n, counts, surv = L.sieve(T.order, rng)
        want = O.sieve_range(T, rng)
        assert (n, counts, surv) == (want[0], want[1], sorted(want[2])), rng


def test_weak_sieve_survivors():
    """Primes 13, 17, 19 leave survivors: the same survivor list as the oracle."""
    L = PaperLoop([13, 17, 19])
    T = O.Tables([13, 17, 19])
    rng = W.rect(1, 150, 1, 150)
    n, counts, surv = L.sieve(T.order, rng)
    want = O.sieve_range(T, rng)
    assert surv and (n, counts, surv) == (want[0], want[1], sorted(want[2]))


def test_c2_in_full_equals_stored_oracle_result():
    """The 2^14 triangle with 64 primes in rejection-rate order, all 81,599,337 pairs,
    against the oracle's stored result; one thread and all threads agree."""
    with open(os.path.join(GOLDEN, "c2_by_rate.json")) as f:
        gold = json.load(f)
    L = PaperLoop(gold["primes"])
    for threads in (0, 1):
        n, counts, surv = L.sieve(gold["order"], gold["ranges"][0], threads=threads)
        r = gold["results"][0]
        assert n == r["n_pairs"] and counts == r["counts"] and surv == [tuple(x) for x in r["survivors"]]


def test_many_ranges_in_one_call_equal_one_by_one():
    """The multi-range call (rows of all ranges as work items) equals per-range calls and
    the oracle on seeded rectangles of the batched workload's shape."""
    primes = W.first_odd_primes(24)
    L = PaperLoop(primes)
    T = O.Tables(primes, "rate")
    ranges = W.batched_rectangles(40, log2_area=(4.0, 12.0)) + [W.rect(1, 60, 1, 60)]
    many = L.sieve_many(T.order, ranges)
    for rng, got in zip(ranges, many):
        assert got == L.sieve(T.order, rng)
        want = O.sieve_range(T, rng)
        assert got == (want[0], want[1], sorted(want[2]))
