"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

Each test ties an oracle function to something other than the oracle itself: a table
or byte string printed in the paper, a closed form, an algebraic identity, a library
routine, a brute-force evaluation on tiny inputs, or a count with an independent
formula.
"""
import math
import os
import random

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


def _polymul(a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _coeff_list(p, q):
    """Oracle coefficients as a dense list indexed by power of t."""
    c = O.q_coefficients(p, q)
    return [c.get(k, 0) for k in range(11)]


# ---------------------------------------------------------------- Eq. 2.5 / Eq. 2.6

def test_u11_matches_printed_table():
    """Eq. 2.5: the 121 bits of u_11 printed in the paper."""
    rows = _read_rows("u11_eq2_5.txt")
    want = np.array([[int(ch) for ch in row] for row in rows], dtype=np.uint8)
    assert want.shape == (11, 11)
    assert np.array_equal(O.unsolvable_table(11), want)


def test_u11_bytes_match_printed_packing():
    """Eq. 2.6: the printed bytes of u_11 (highest bit leftmost, zero padding)."""
    packed = O.pack_table_bytes(O.unsolvable_table(11))
    assert len(packed) == 16
    for row in _read_rows("u11_bytes_eq2_6.txt"):
        idx, bits = row.split()
        assert format(packed[int(idx)], "08b") == bits, idx


@pytest.mark.parametrize("r", [2, 3, 5, 7])
def test_small_prime_tables_vanish(r):
    """Section 2, after Eq. 2.4: u_2, u_3, u_5 and u_7 are identically zero."""
    assert int(O.unsolvable_table(r).sum()) == 0


@pytest.mark.parametrize("r", [11, 13, 17, 19, 23, 29, 31])
def test_pack_length_and_padding(r):
    u = O.unsolvable_table(r)
    b = O.pack_table_bytes(u)
    assert len(b) == (r * r + 7) // 8
    tail = (r * r) % 8
    if tail:
        assert b[-1] >> tail == 0
    # unpack and compare bit by bit
    bits = [(b[i // 8] >> (i % 8)) & 1 for i in range(r * r)]
    assert bits == [int(x) for x in u.reshape(-1)]


# ---------------------------------------------------------------- Eq. 1.1 closed forms

def test_q11_closed_form():
    """Q_{1,1}(t) = (t - 1)(t + 1)(t^2 + 1)^4."""
    want = [1]
    for f in ([-1, 1], [1, 1], [1, 0, 1], [1, 0, 1], [1, 0, 1], [1, 0, 1]):
        want = _polymul(want, f)
    assert _coeff_list(1, 1) == want


@pytest.mark.parametrize("p", [1, 2, 3, 7, 12345])
def test_q_p0_closed_form(p):
    """Q_{p,0}(t) = t^6 (t - p^2)^2 (t + p^2)^2."""
    want = [0, 0, 0, 0, 0, 0, 1]
    for f in ([-p * p, 1], [-p * p, 1], [p * p, 1], [p * p, 1]):
        want = _polymul(want, f)
    assert _coeff_list(p, 0) == want


@pytest.mark.parametrize("q", [1, 2, 5, 9, 4321])
def test_q_0q_closed_form(q):
    """Q_{0,q}(t) = t^6 (t^4 + 6 q^4 t^2 + q^8)."""
    want = [0] * 6 + [q ** 8, 0, 6 * q ** 4, 0, 1]
    assert _coeff_list(0, q) == want


def test_evenness():
    for p, q in [(2, 3), (5, 7), (100, 3), (65535, 4097)]:
        c = _coeff_list(p, q)
        assert all(c[k] == 0 for k in range(1, 11, 2))
        for t in (1, 2, 17, 1000):
            assert O.q_value(p, q, t) == O.q_value(p, q, -t)


def test_weighted_homogeneity():
    """Q_{lp,lq}(l^2 t) = l^20 Q_pq(t) (exact integers)."""
    g = random.Random(1)
    for _ in range(200):
        p, q, t, lam = (g.randint(0, 10 ** 6), g.randint(0, 10 ** 6),
                        g.randint(-10 ** 9, 10 ** 9), g.randint(1, 1000))
        assert O.q_value(lam * p, lam * q, lam * lam * t) == lam ** 20 * O.q_value(p, q, t)


def test_reflection():
    """t^10 Q_pq(p^2 q^2 / t) = -p^10 q^10 Q_qp(t): coefficient of t^(10-k) on the left
    is c_k(p, q) (pq)^(2k); on the right -(pq)^10 c_(10-k)(q, p)."""
    g = random.Random(2)
    for _ in range(200):
        p, q = g.randint(1, 10 ** 5), g.randint(1, 10 ** 5)
        a, b = _coeff_list(p, q), _coeff_list(q, p)
        for k in range(11):
            assert a[k] * (p * q) ** (2 * k) == -((p * q) ** 10) * b[10 - k]


def test_diagonal_has_root():
    """Q_{k,k}(k^2) = 0: the pairs p = q carry the integer root t = k^2."""
    for k in list(range(1, 60)) + [2 ** 20 - 3, 2 ** 31 + 11]:
        assert O.q_value(k, k, k * k) == 0


def test_sympy_factorisation_consistent():
    """Library cross-check: sympy factors Q_{k,k} with the root t = k^2 and finds Q_pq
    irreducible for small coprime p != q (Conjecture 1.1)."""
    sympy = pytest.importorskip("sympy")
    t = sympy.symbols("t")

    def poly(p, q):
        return sum(c * t ** k for k, c in O.q_coefficients(p, q).items())

    for k in (1, 2, 3):
        _, fl = sympy.factor_list(poly(k, k))
        assert any(sympy.degree(f, t) == 1 and f.subs(t, k * k) == 0 for f, _ in fl)
    for p, q in [(2, 1), (3, 2), (5, 3), (7, 4)]:
        _, fl = sympy.factor_list(poly(p, q))
        assert len(fl) == 1 and fl[0][1] == 1 and sympy.degree(fl[0][0], t) == 10


# ---------------------------------------------------------------- Definition 1.1 / Eq. 2.3

@pytest.mark.parametrize("r", [2, 3, 5, 7, 11, 13])
def test_table_vs_pure_python_definition(r):
    """The numpy table equals Definition 1.1 evaluated pair by pair in pure Python."""
    u = O.unsolvable_table(r)
    for a in range(r):
        for b in range(r):
            assert u[a, b] == (0 if O.is_solvable(a, b, r) else 1)


@pytest.mark.parametrize("r", W.first_odd_primes(24))
def test_structural_zeros_and_symmetry(r):
    """Row 0 and column 0 vanish (t = 0 is a root when pq = 0 mod r), the diagonals
    p = +-q vanish (t = p^2 is a root), and u_r is symmetric (reflection identity)."""
    u = O.unsolvable_table(r)
    assert not u[0].any() and not u[:, 0].any()
    for a in range(r):
        assert u[a, a] == 0 and u[a, (r - a) % r] == 0
    assert np.array_equal(u, u.T)


@pytest.mark.parametrize("r", W.first_odd_primes(24))
def test_reduced_matches_full(r):
    """u_r(a, b) = v_r(a / b) for b != 0 (weighted homogeneity), u_r(a, 0) = 0."""
    assert np.array_equal(O.full_from_reduced(r, O.reduced_table(r)), O.unsolvable_table(r))


@pytest.mark.slow
@pytest.mark.parametrize("r", [r for r in W.first_odd_primes(64) if r > 97])
def test_reduced_matches_full_to_313(r):
    assert np.array_equal(O.full_from_reduced(r, O.reduced_table(r)), O.unsolvable_table(r))


def test_unsolvable_counts_brute_force():
    """Number of unsolvable k (pairs (k, 1)) for r = 11..41, by pure-Python brute force."""
    for r in [11, 13, 17, 19, 23, 29, 31, 37, 41]:
        brute = sum(0 if O.is_solvable(k, 1, r) else 1 for k in range(r))
        assert O.unsolvable_count(r) == brute


# Number of k in [0, r) with v_r(k) = u_r(k, 1) = 1 for the first 24 odd primes.  The values
# for r = 11..41 are the survey's independent scratch computation; all 24 were recomputed
# by sympy's polynomial factorisation over GF(r) (a linear factor of Q_{k,1}(t) mod r means
# a root), a method that shares nothing with the oracle's evaluation at every t~.
UNSOLVABLE_K = {3: 0, 5: 0, 7: 0, 11: 8, 13: 4, 17: 12, 19: 12, 23: 16, 29: 20, 31: 16, 37: 24,
                41: 28, 43: 24, 47: 24, 53: 40, 59: 32, 61: 36, 67: 28, 71: 40, 73: 56, 79: 32,
                83: 48, 89: 44, 97: 64}

# Those counts ranked by hand: decreasing count / r (density) and count / (r + 1) (rate),
# ties to the smaller r.  For these 24 primes both rankings agree.
ORDER_24 = [73, 53, 11, 17, 23, 29, 41, 97, 37, 19, 61, 83, 71, 43, 59, 31, 47, 89, 67, 79, 13, 3, 5, 7]

# The 1 <= q < p <= 200 triangle with the first 24 odd primes in ascending order (the
# paper's order, section 2): the survey's independent scratch computation of the pair
# total, the survivors and each prime's first-rejecter count (every prime not listed: 0).
C1_PAIRS = 12231
C1_COUNTS = {11: 8153, 13: 1164, 17: 1940, 19: 612, 23: 255, 29: 75, 31: 19, 37: 8, 41: 3, 43: 2}


def test_unsolvable_counts_literal():
    """Definition 1.1 at (k, 1) for every k: the oracle's counts equal the literals."""
    for r, want in UNSOLVABLE_K.items():
        assert O.unsolvable_count(r) == want, r


@pytest.mark.parametrize("r", [43, 53, 73, 97])
def test_unsolvable_literals_by_factorisation(r):
    """The literals themselves, recomputed here by factoring Q_{k,1}(t) over GF(r) with
    sympy (a root mod r is a linear factor; the zero polynomial is solvable)."""
    sp = pytest.importorskip("sympy")
    t = sp.symbols("t")
    n = 0
    for k in range(r):
        c = O.q_coefficients(k, 1)
        poly = sp.Poly(sum(v * t ** e for e, v in c.items()), t, modulus=r)
        solv = poly.is_zero or any(f.degree() == 1 for f, _ in poly.factor_list()[1])
        n += 0 if solv else 1
    assert n == UNSOLVABLE_K[r]


@pytest.mark.parametrize("mode", [True, "rate"])
def test_effective_order_literal(mode):
    """The density and rate orders of the first 24 odd primes equal the hand ranking."""
    primes = W.first_odd_primes(24)
    T = O.Tables(primes, mode, full_limit=0)
    assert [primes[i] for i in T.order] == ORDER_24


@pytest.mark.parametrize("pairwise", [False, True])
def test_c1_literal_counts(pairwise):
    """Section 2 sieve, section 5 loop: C1 in ascending order against the literal pair
    total, survivors and first-rejecter counts.  A wrong first rejecter, an off-by-one at
    q < p or a leaked diagonal pair changes one of them."""
    primes = W.first_odd_primes(24)
    res = O.run(primes, [W.triangle(200)], pairwise=pairwise)["ranges"][0]
    assert res["n_pairs"] == C1_PAIRS
    assert res["survivors"] == [] and res["roots"] == []
    assert res["counts"] == [C1_COUNTS.get(r, 0) for r in primes]


def test_c1_literal_counts_by_totient():
    """The C1 pair total is sum_{p=2..200} phi(p), a closed count."""
    assert int(_phi_sum(200)[2:].sum()) == C1_PAIRS


def test_effective_order_by_density():
    primes = W.first_odd_primes(40)
    cnt = [O.unsolvable_count(r) for r in primes]
    order = O.effective_order(primes, cnt, True)
    assert sorted(order) == list(range(len(primes)))
    for a, b in zip(order, order[1:]):
        fa, fb = cnt[a] / primes[a], cnt[b] / primes[b]
        assert fa > fb or (fa == fb and primes[a] < primes[b])
    assert O.effective_order(primes, cnt, False) == list(range(len(primes)))
    rate = O.effective_order(primes, cnt, "rate")
    for a, b in zip(rate, rate[1:]):
        fa, fb = cnt[a] / (primes[a] + 1), cnt[b] / (primes[b] + 1)
        assert fa > fb or (fa == fb and primes[a] < primes[b])


def test_rejection_rate_matches_coprime_pairs():
    """The rate count/(r + 1) is the fraction of coprime pairs a prime rejects: counted
    by brute force over all coprime pairs of a large box, prime by prime."""
    pairs = [(p, q) for p in range(1, 400) for q in range(1, 400) if p != q and math.gcd(p, q) == 1]
    for r in (11, 13, 17, 19, 23):
        T = O.Tables([r])
        rej = sum(T.bit(0, p, q) for p, q in pairs)
        assert abs(rej / len(pairs) - O.unsolvable_count(r) / (r + 1)) < 0.01


# ---------------------------------------------------------------- sieve and totals

def _phi_sum(n):
    phi = np.arange(n + 1, dtype=np.int64)
    for i in range(2, n + 1):
        if phi[i] == i:
            phi[i::i] -= phi[i::i] // i
    return phi


def test_triangle_pair_count_is_totient_sum():
    """#{1 <= q < p <= N, gcd = 1} = sum_{p=2..N} phi(p)."""
    phi = _phi_sum(1 << 14)
    for n in (200, 1000):
        rng = W.triangle(n)
        assert sum(len(O.row_pairs(p, rng)) for p in range(2, n + 1)) == int(phi[2:n + 1].sum())
    assert int(phi[2:(1 << 14) + 1].sum()) == 81599337


def test_pairs_vectorised_vs_pure_python():
    g = random.Random(3)
    for _ in range(20):
        p_lo, q_lo = g.randint(1, 300), g.randint(1, 300)
        rng = W.rect(p_lo, p_lo + g.randint(0, 40), q_lo, q_lo + g.randint(0, 40),
                      q_lt_p=g.random() < 0.5, allow_diagonal=g.random() < 0.5)
        a = [(p, int(q)) for p in range(rng["p_lo"], rng["p_hi"] + 1) for q in O.row_pairs(p, rng)]
        assert a == list(O.pairs_in_range(rng))


@pytest.mark.parametrize("by_density", [False, True])
def test_sieve_vectorised_vs_pairwise(by_density):
    """The row-vectorised sieve equals the pair-by-pair loop of section 5."""
    primes = W.first_odd_primes(24)
    T = O.Tables(primes, by_density)
    for rng in [W.triangle(120), W.rect(300, 340, 1, 700), W.rect(1, 60, 1, 60, allow_diagonal=True)]:
        a = O.sieve_range(T, rng)
        b = O.sieve_range_pairwise(T, rng)
        assert a == b
        n_pairs, counts, surv = a
        assert sum(counts) + len(surv) == n_pairs


def test_sieve_reduced_lookup_vs_full():
    """The reduced-table lookup path gives the same sieve as full tables."""
    primes = W.first_odd_primes(24)
    A = O.Tables(primes)
    B = O.Tables(primes, full_limit=0)
    rng = W.rect(1000, 1040, 1, 2000)
    assert O.sieve_range(A, rng) == O.sieve_range(B, rng)


def test_weak_sieves():
    """With primes 3, 5, 7 (all-zero tables) every pair survives; every count is 0."""
    rng = W.triangle(40)
    res = O.run([3, 5, 7], [rng])["ranges"][0]
    assert res["counts"] == [0, 0, 0]
    assert len(res["survivors"]) == res["n_pairs"]
    assert res["roots"] == []


def test_sieve_soundness_on_diagonal():
    """A pair with an integer root is never rejected: (k, k) passes every table and its
    root k^2 is reported."""
    primes = W.first_odd_primes(24)
    res = O.run(primes, [W.rect(1, 50, 1, 50, allow_diagonal=True)])["ranges"][0]
    assert [(p, q) for (p, q) in res["survivors"] if p == q] == [(k, k) for k in range(1, 51)]
    assert res["roots"] == [(k, k, k * k) for k in range(1, 51)]


# ---------------------------------------------------------------- roots

def test_root_bound_holds():
    """Every positive real root of R(u) = Q(sqrt u) lies below root_bound_u (numpy's
    companion-matrix roots as the independent routine) and R(u) > 0 beyond it."""
    g = random.Random(4)
    for _ in range(200):
        p, q = g.randint(1, 3000), g.randint(1, 3000)
        c = O.q_coefficients(p, q)
        U = O.root_bound_u(p, q)
        roots = np.roots([float(c[k]) for k in (10, 8, 6, 4, 2, 0)])
        pos = [z.real for z in roots if abs(z.imag) <= 1e-9 * abs(z) and z.real > 0]
        assert all(u <= U * (1 + 1e-9) for u in pos)
        for u in (U + 1, 2 * U, 10 * U + 7):
            assert sum(c[2 * j] * u ** j for j in range(6)) > 0


def test_roots_divisor_method_vs_scan():
    """Rational-root-theorem search equals a brute-force t scan up to the root bound."""
    for p in range(1, 9):
        for q in range(1, 9):
            assert O.integer_roots(p, q) == O.integer_roots_scan(p, q), (p, q)


def test_roots_of_scaled_pairs():
    """Roots scale with the pair: (l, l) has exactly t = l^2 (from Q_{1,1})."""
    for lam in (1, 2, 6, 30, 210, 97 * 89):
        assert O.integer_roots(lam, lam) == [lam * lam]


def test_no_coprime_roots_small():
    """Conjecture 1.1 in the small: no coprime p != q <= 24 has an integer root."""
    for p in range(1, 25):
        for q in range(1, 25):
            if p != q and math.gcd(p, q) == 1:
                assert O.integer_roots(p, q) == []


# ---------------------------------------------------------------- section 6

@pytest.mark.slow
def test_paper_region_statistics():
    """Section 6: no pair of the scanned region passes the 96 primes 11..541, and the
    deepest rejecting prime is at most the 29th of the list (137).  Checked on the rows
    152 <= p <= 200 of the segment of Eq. 5.2."""
    primes = W.primes_between(11, 541)
    assert len(primes) == 96 and primes[28] == 137
    T = O.Tables(primes, full_limit=0)
    deepest = -1
    for rng in W.paper_region_rows(152, 200):
        n_pairs, counts, surv = O.sieve_range(T, rng)
        assert surv == []
        nz = [i for i, c in enumerate(counts) if c]
        deepest = max(deepest, max(nz))
    assert deepest <= 28


def test_ceil_root_exact():
    """The integer k-th root used by the root bound is exact on huge integers."""
    from oracle.cuboid_oracle import _ceil_root
    g = random.Random(5)
    for _ in range(3000):
        x = g.randint(1, 10 ** g.randint(1, 250))
        k = g.randint(1, 5)
        y = _ceil_root(x, k)
        assert y ** k >= x and (y - 1) ** k < x
    for k in (2, 3, 5):
        for b in (1, 2, 10 ** 40 + 1):
            assert _ceil_root(b ** k, k) == b


# ---------------------------------------------------------------- region of Theorem 1.2

def _smallest_q(pred):
    q = 1
    while not pred(q):
        q += 1
    return q


def test_region_bounds_follow_eq_5_1_and_5_2():
    """Eq. 5.1 (p <= 151: p/59 <= q) and Eq. 5.2 (p >= 152: cbrt(p/9) <= q) are the two
    cases of the min() of Eq. 1.2; found here by brute force with exact rationals (the
    cube root compared by cubing), independently of the oracle's integer bounds."""
    from fractions import Fraction as F
    for p in list(range(1, 1200)) + [5000, 12345, 154000, 72796055]:
        linear_is_min = F(p, 59) ** 3 <= F(p, 9)
        assert linear_is_min == (p <= 151)
        if p <= 151:
            lo = _smallest_q(lambda q: F(q) >= F(p, 59))
        else:
            lo = _smallest_q(lambda q: F(q) ** 3 >= F(p, 9))
        assert O.region_q_bounds(p) == (lo, 59 * p)


def test_region_start_and_stop_examples():
    """Section 5: the search starts at (152, 3), whose q obeys Eq. 5.2 and is the first
    such q; the printed stop point (112618, 5691455) lies inside its row's segment; p_max
    = 72796055 is the last p with 59 p below 2^32."""
    assert O.region_q_bounds(152)[0] == 3
    lo, hi = O.region_q_bounds(112618)
    assert lo <= 5691455 <= hi
    assert 59 * 72796055 < 2 ** 32 <= 59 * 72796056


def test_region_pair_count_brute_force():
    """The Moebius count of coprime pairs equals enumeration on small row blocks."""
    for a, b in [(1, 60), (140, 165), (997, 1003)]:
        brute = sum(len(O.row_pairs(r["p_lo"], r)) for r in O.region_rows(a, b))
        assert O.region_pair_count(a, b) == brute


def test_region_pair_count_section6():
    """Section 6 counts about sum_{p <= 154000} 59 p = 699626543000 lattice points; the
    coprime pairs among them are close to 6/pi^2 of that."""
    n_lattice = sum(59 * p for p in range(1, 154001))
    assert n_lattice == 699626543000
    exact = sum(hi - lo + 1 for lo, hi in map(O.region_q_bounds, range(1, 154001)))
    assert abs(exact - n_lattice) / n_lattice < 1e-4
    coprime = O.region_pair_count(1, 154000)
    assert abs(coprime / exact - 6 / math.pi ** 2) < 1e-3


def test_region_scan_matches_pairwise():
    """The region scan (numpy rows) equals the one-pair-at-a-time sieve over the same
    rows, from a mid-row start, with survivors (few primes)."""
    T = O.Tables([3, 5, 7, 11, 13], full_limit=0)
    got = O.region_scan(T, 20, 26, q_from=40)
    counts = [0] * 5
    surv, pairs = [], 0
    for rng in O.region_rows(20, 26, 40):
        k, c, s = O.sieve_range_pairwise(T, rng)
        pairs += k
        counts = [x + y for x, y in zip(counts, c)]
        surv += s
    assert (got["pairs"], got["counts"], got["survivors"]) == (pairs, counts, surv)
    assert surv and got["depth"] == 5 and got["r_max"] == T.primes[T.order[-1]]
    assert O.region_rows(150, 152, 40)[0]["q_lo"] == 40
    assert [r["q_lo"] for r in O.region_rows(150, 152, 40)[1:]] == [3, 3]


def test_deepest_prime():
    """Depth is the position of the last nonzero count in the effective order."""
    T = O.Tables([11, 13, 17, 19], full_limit=0)
    assert O.deepest_prime(T, [5, 0, 2, 0], 0) == (3, 17)
    assert O.deepest_prime(T, [0, 0, 0, 0], 0) == (0, 0)
    assert O.deepest_prime(T, [1, 0, 0, 0], 3) == (4, 19)


# ---------------------------------------------------------------- table files (section 2)

def test_paper_files_layout():
    """The bit tables file starts with the printed u_11 bytes of Eq. 2.6; records are
    8 bytes {short prime; pad; unsigned int offset} and offsets are running sums of
    ceil(r^2/8); reading the files back gives the tables."""
    import struct
    primes = [11, 13, 17, 5]
    blob, recs = O.paper_table_files(primes)
    for row in _read_rows("u11_bytes_eq2_6.txt"):          # the bytes printed in Eq. 2.6
        idx, bits = row.split()
        assert blob[int(idx)] == int(bits, 2)
    sizes = [(r * r + 7) // 8 for r in primes]
    assert len(blob) == sum(sizes) and len(recs) == 8 * len(primes)
    offs = [0, sizes[0], sizes[0] + sizes[1], sizes[0] + sizes[1] + sizes[2]]
    for k, r in enumerate(primes):
        rec = recs[8 * k:8 * k + 8]
        assert rec[2:4] == b"\0\0"
        assert struct.unpack("<h", rec[:2])[0] == r and struct.unpack("<I", rec[4:])[0] == offs[k]
    back = O.read_paper_table_files(blob, recs)
    assert [r for r, _ in back] == primes
    for r, u in back:
        assert (u == O.unsolvable_table(r)).all()


def test_eq_2_7_limits():
    """Eq. 2.7: the tables of the primes from 11 on fit 32-bit offsets up to the prime
    just below 9697 and no further; 100 primes from 11 (to 569) need under 1.5 MB."""
    import sympy
    total, last_ok = 0, None
    for r in sympy.primerange(11, 20000):
        total += r * r / 8
        if total >= 2 ** 32:
            assert r == 9697 and last_ok < 9697
            break
        last_ok = r
    first100 = list(sympy.primerange(11, 600))[:100]
    assert first100[-1] == 569
    assert sum((r * r + 7) // 8 for r in first100) < 1.5 * 2 ** 20


# ---------------------------------------------------------------- Theorem 1.1

def test_theorem_1_1_threshold_by_quadratic():
    """Above max(p^2, pq, q^2), (p^2 + t)(pq + t) > 2 t^2 is t^2 - (p^2 + pq) t - p^3 q < 0,
    i.e. t below the positive root x* = ((p^2 + pq) + sqrt((p^2 + pq)^2 + 4 p^3 q)) / 2;
    the largest such integer t is found with an integer square root and the check flips
    exactly there."""
    g = random.Random(11)
    for _ in range(400):
        p, q = g.randint(1, 10 ** 6), g.randint(1, 10 ** 6)
        b, c = p * p + p * q, p ** 3 * q
        disc = b * b + 4 * c
        def below_root(t):                          # t < x*  <=>  2t - b < sqrt(disc)
            return 2 * t - b < 0 or (2 * t - b) ** 2 < disc
        t_star = (b + math.isqrt(disc)) // 2
        while not below_root(t_star):
            t_star -= 1
        while below_root(t_star + 1):
            t_star += 1
        lo = max(p * p, p * q, q * q)
        for t in (t_star - 1, t_star, t_star + 1, t_star + 2, lo, lo + 1):
            if t <= 0:
                continue
            want = t > lo and t <= t_star
            assert O.theorem_1_1_holds(p, q, t) == want, (p, q, t)


def test_theorem_1_1_small_window():
    """p = 2, q = 1: the window is 5 <= t <= 7 (x* = 3 + sqrt(17) = 7.12)."""
    assert [t for t in range(1, 20) if O.theorem_1_1_holds(2, 1, t)] == [5, 6, 7]


def test_diagonal_roots_are_not_cuboids():
    """The roots t = k^2 of the pairs p = q sit on the boundary t = p^2 (Theorem 1.1
    asks for t > p^2), so they never give a cuboid."""
    for k in (1, 2, 7, 1000, 2 ** 31 + 11):
        assert not O.theorem_1_1_holds(k, k, k * k)


# ---------------------------------------------------------------- 64-bit ranges (beyond section 6's p_max)

def test_coprime_count_brute_force():
    """The Moebius count of the q prime to p in [q_lo, q_hi] equals the gcd count."""
    g = random.Random(11)
    for _ in range(300):
        p = g.randrange(1, 20000)
        a = g.randrange(1, 5000)
        b = a + g.randrange(-3, 700)
        assert O.coprime_count(p, a, b) == sum(1 for q in range(a, b + 1) if math.gcd(p, q) == 1)


def test_coprime_count_periodic_in_q():
    """Shifting q by a multiple of p keeps every gcd(p, q): the counts of [a, b] and
    [a + k p, b + k p] agree, at q near 2^39 too (exact integers, no 64-bit bound)."""
    for p in (30, 9699690, 72796057, 4294967291):
        for k in (1, 2 ** 39 // p):
            assert O.coprime_count(p, 1000, 9000) == O.coprime_count(p, 1000 + k * p, 9000 + k * p)


def test_sieve_vectorised_vs_pairwise_above_2_32():
    """Rows of p beyond the paper's 32-bit limit with q above 2^32 (and rows of q with p
    near 2^39): the numpy sieve (int64 residues) equals the pure-Python-int pairwise
    sieve, so no 64-bit intermediate overflows."""
    primes = W.primes_between(11, 41)
    T = O.Tables(primes)
    for rng in [W.rect(72796056, 72796058, 2 ** 32 - 150, 2 ** 32 + 150),
                W.rect(2 ** 39 - 40, 2 ** 39 + 40, 1, 6),
                W.rect(2 ** 40 - 30, 2 ** 40 - 1, 2 ** 32 - 4, 2 ** 32 - 1)]:
        assert O.sieve_range(T, rng) == O.sieve_range_pairwise(T, rng)


def test_sieve_outcome_depends_on_residues_only():
    """Section 2: a coprime pair's first rejecting prime depends only on (p mod r, q mod r)
    for the listed primes.  With L the product of the primes, (p, q) and (p, q + k L)
    meet the same first rejecter whenever both are coprime, at q beyond 2^39."""
    primes = [11, 13, 17, 19]
    T = O.Tables(primes)
    L = 11 * 13 * 17 * 19
    k = (2 ** 39) // L
    for p in (72796057, 2 ** 31 + 11):
        for q in range(5000, 5400):
            q2 = q + k * L
            if math.gcd(p, q) != 1 or math.gcd(p, q2) != 1:
                continue
            first = [next((i for i in T.order if T.bit(i, p, x)), None) for x in (q, q2)]
            assert first[0] == first[1]


def test_diagonal_root_near_2_40():
    """Q_{k,k}(k^2) = 0 at k near 2^40, and for a prime k the divisor search finds
    exactly that root (the exact root test of 64-bit ranges meets t near 2^80)."""
    for k in (2 ** 39 + 1, 2 ** 40 - 87):
        assert O.q_value(k, k, k * k) == 0
    k = 2 ** 40 - 87
    assert _is_prime_mr(k)
    assert O.integer_roots(k, k) == [k * k]


def _is_prime_mr(n):
    """Miller-Rabin with the first twelve primes as bases (exact below 3.3e24)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for b in small:
        if n % b == 0:
            return n == b
    d, s = n - 1, 0
    while d % 2 == 0:
        d, s = d // 2, s + 1
    for b in small:
        x = pow(b, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True
