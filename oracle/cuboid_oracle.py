"""Oracle for the modulo-primes cuboid sieve -- TEST INFRASTRUCTURE ONLY.

Paper: R. R. Gallyamov, I. R. Kadyrov, D. D. Kashelevskiy, N. G. Kutlugallyamov,
R. A. Sharipov, "A fast modulo primes algorithm for searching perfect cuboids and its
implementation" (arXiv:1601.00636).

This is a plain, slow, obviously-correct CPU restatement of what the GPU library
computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code, constants or helpers with the CUDA
library and never imports it.  Integers are Python built-in arbitrary-precision ints
(numpy int64 only where every intermediate is < 2**44, i.e. residues modulo a table
prime r < 2**13 and their products).

What it computes, in the paper's notation:

* Q_pq(t), Eq. 1.1 (section 1, Conjecture 1.1): coefficients and exact values.
* u_r(p~, q~), Eq. 2.3 with Definition 1.1 of section 2: the unsolvability bit,
  built by trying every t~ in [0, r).
* The byte packing of Eq. 2.6 (row-major index p~ r + q~, least significant bit first).
* The bit sieve of section 2 and the search loop of section 5: for each pair the primes
  are tried in order and the first prime whose bit is 1 rejects the pair.
* Integer roots t > 0 of Q_pq for the pairs that pass every prime, found with the
  rational root theorem (Q is monic and even, so u = t^2 divides the constant term
  -p^10 q^10 and t divides (pq)^5).

Readings where the paper is silent (each is also listed in the design notes):

* Only coprime pairs with p != q are sieved (Conjecture 1.1); the test-only option
  ``allow_diagonal`` adds the pairs p == q whatever their gcd.
* Range bounds are inclusive; ``q_lt_p`` restricts a range to q < p (q <= p with
  ``allow_diagonal``).
* The effective prime order is the caller's order, or the primes sorted by decreasing
  fraction of unsolvable k in the reduced table v_r (count/r), or by the rejection rate
  of a coprime pair (count/(r + 1)); ties: smaller r first.  A pair's count goes to the
  first prime of the effective order that rejects it.
* The reduced table v_r(k) = u_r(k, 1) is obtained by brute force over t~; the identity
  u_r(a, b) = v_r(a b^-1 mod r) for b != 0 and u_r(a, 0) = 0 (weighted homogeneity of
  Eq. 1.1: Q_{lp,lq}(l^2 t) = l^20 Q_pq(t)) is checked against brute-force full tables in
  the tests for every r <= 313 and is used by ``lookup`` only for larger r.
"""
from __future__ import annotations

from fractions import Fraction
from math import gcd, isqrt

import numpy as np

# Primes up to this bound get brute-force full r x r tables (Eq. 2.3 by definition);
# larger primes are looked up through the reduced table (homogeneity identity).
FULL_TABLE_LIMIT = 313


# --------------------------------------------------------------------------------------
# Eq. 1.1: the polynomial Q_pq(t)
# --------------------------------------------------------------------------------------

def q_coefficients(p: int, q: int) -> dict[int, int]:
    """Coefficients {power of t: integer} of Q_pq(t), Eq. 1.1 (section 1).

    Only even powers occur: t^10, t^8, t^6, t^4, t^2, t^0.
    """
    p2 = p * p
    q2 = q * q
    return {
        10: 1,
        8: (2 * q2 + p2) * (3 * q2 - 2 * p2),
        6: q2 ** 4 + 10 * p2 * q2 ** 3 + 4 * p2 ** 2 * q2 ** 2 - 14 * p2 ** 3 * q2 + p2 ** 4,
        4: -p2 * q2 * (q2 ** 4 - 14 * p2 * q2 ** 3 + 4 * p2 ** 2 * q2 ** 2
                       + 10 * p2 ** 3 * q2 + p2 ** 4),
        2: -(p2 ** 3) * (q2 ** 3) * (q2 + 2 * p2) * (3 * p2 - 2 * q2),
        0: -(q2 ** 5) * (p2 ** 5),
    }


def q_value(p: int, q: int, t: int) -> int:
    """Exact value of Q_pq(t), Eq. 1.1."""
    return sum(c * t ** k for k, c in q_coefficients(p, q).items())


def q_value_mod(p: int, q: int, t: int, r: int) -> int:
    """Q_pq(t) mod r, Eq. 2.2 (the quotient equation of section 2)."""
    return q_value(p, q, t) % r


# --------------------------------------------------------------------------------------
# Definition 1.1 / Eq. 2.3: unsolvability bits
# --------------------------------------------------------------------------------------

def is_solvable(a: int, b: int, r: int) -> bool:
    """Definition 1.1 (section 2): (a, b) is solvable mod r iff some t in [0, r) makes
    Q_ab(t) = 0 mod r.  Pure Python; for small r and for cross-checks."""
    return any(q_value(a, b, t) % r == 0 for t in range(r))


def _coeffs_mod_rows(a: int, r: int) -> np.ndarray:
    """Coefficients of Q_{a,b} mod r for every b in [0, r): array [6, r] in order
    t^10, t^8, t^6, t^4, t^2, t^0.  Eq. 1.1 is evaluated on a numpy object array, i.e.
    with exact Python ints element by element, then reduced mod r."""
    b = np.arange(r, dtype=object)
    c = q_coefficients(a, b)
    out = np.zeros((6, r), dtype=np.int64)
    for row, k in enumerate((10, 8, 6, 4, 2, 0)):
        out[row] = (np.asarray(c[k] + 0 * b, dtype=object) % r).astype(np.int64)
    return out


def unsolvable_table(r: int) -> np.ndarray:
    """The full table u_r of Eq. 2.3 as a uint8 array [p~][q~], built by Definition 1.1:
    for each (p~, q~) every t~ in [0, r) is tried (numpy evaluates all t~ at once)."""
    t = np.arange(r, dtype=np.int64)
    u = np.zeros((r, r), dtype=np.uint8)
    for a in range(r):
        c = _coeffs_mod_rows(a, r)                       # [6, r(b)]
        acc = np.ones((r, r), dtype=np.int64)            # [b, t]: value of the t^10 term's coefficient
        for row in range(1, 6):                          # Horner in t^2 over the even powers
            acc = (acc * (t * t % r)[None, :] + c[row][:, None]) % r
        solvable = (acc == 0).any(axis=1)
        u[a] = (~solvable).astype(np.uint8)
    return u


def reduced_table(r: int) -> np.ndarray:
    """v_r(k) = u_r(k, 1) for k in [0, r), uint8, by Definition 1.1 at (k, 1)."""
    t = np.arange(r, dtype=np.int64)
    v = np.zeros(r, dtype=np.uint8)
    for k in range(r):
        c = q_coefficients(k, 1)
        acc = np.ones(r, dtype=np.int64)
        for kk in (8, 6, 4, 2, 0):
            acc = (acc * (t * t % r) + c[kk] % r) % r
        v[k] = 0 if (acc == 0).any() else 1
    return v


def full_from_reduced(r: int, v: np.ndarray) -> np.ndarray:
    """u_r(a, b) = v_r(a b^-1 mod r) for b != 0, u_r(a, 0) = 0 (weighted homogeneity)."""
    u = np.zeros((r, r), dtype=np.uint8)
    for b in range(1, r):
        binv = pow(b, r - 2, r)
        for a in range(r):
            u[a, b] = v[a * binv % r]
    return u


def unsolvable_count(r: int) -> int:
    """Number of k in [0, r) with v_r(k) = 1."""
    return int(reduced_table(r).sum())


def pack_table_bytes(u: np.ndarray) -> bytes:
    """Eq. 2.6: the r x r bits in row-major order (index p~ r + q~), eight per byte, the
    first bit of each group in the least significant position, the last byte padded
    with zero bits; ceil(r^2 / 8) bytes."""
    r = u.shape[0]
    flat = [int(x) for x in u.reshape(-1)]
    out = bytearray((r * r + 7) // 8)
    for i, bit in enumerate(flat):
        if bit:
            out[i // 8] |= 1 << (i % 8)
    return bytes(out)


# --------------------------------------------------------------------------------------
# Tables for a prime list, the effective order and lookups
# --------------------------------------------------------------------------------------

class Tables:
    """Tables for a list of primes: full u_r for r <= FULL_TABLE_LIMIT, reduced v_r for
    every r, and the effective order (indices into the caller's list)."""

    def __init__(self, primes, by_density: bool = False, full_limit: int = FULL_TABLE_LIMIT,
                 reduced=None):
        """``reduced``: the reduced tables ``reduced_table(r)`` of the primes, when they
        were already computed (for instance by worker processes); else built here."""
        self.primes = [int(r) for r in primes]
        self.reduced = ([np.asarray(v, dtype=np.uint8) for v in reduced] if reduced is not None
                        else [reduced_table(r) for r in self.primes])
        self.full = [unsolvable_table(r) if r <= full_limit else None
                     for r in self.primes]
        self.inv = [np.array([0] + [pow(b, r - 2, r) for b in range(1, r)], dtype=np.int64)
                    for r in self.primes]
        self.order = effective_order(self.primes, [int(v.sum()) for v in self.reduced],
                                     by_density)

    def lookup(self, i: int, a: int, b: np.ndarray) -> np.ndarray:
        """u_r(a, b) for prime index i (caller order), a scalar, b an int64 array."""
        r = self.primes[i]
        if self.full[i] is not None:
            return self.full[i][a % r][b % r]
        bb = b % r
        k = (a % r) * self.inv[i][bb] % r
        return np.where(bb == 0, 0, self.reduced[i][k]).astype(np.uint8)

    def bit(self, i: int, a: int, b: int) -> int:
        return int(self.lookup(i, a, np.array([b], dtype=np.int64))[0])


def effective_order(primes, unsolvable_counts, by_density) -> list[int]:
    """The order in which the primes are tried.

    * False / "given": the caller's order (the paper's ascending list, section 2);
    * True / "density": decreasing unsolvable fraction count/r of the reduced table;
    * "rate": decreasing rejection rate count/(r + 1) of a random coprime pair (given
      gcd(p, q) = 1, r divides p with probability 1/(r + 1), likewise q, and otherwise
      p/q mod r is uniform on the r - 1 nonzero residues, count of which are unsolvable).
    Comparisons are exact (fractions); ties go to the smaller r."""
    idx = list(range(len(primes)))
    mode = {False: "given", True: "density"}.get(by_density, by_density)
    if mode == "given":
        return idx
    extra = 1 if mode == "rate" else 0
    if mode not in ("density", "rate"):
        raise ValueError(f"unknown order {by_density!r}")
    return sorted(idx, key=lambda i: (-Fraction(unsolvable_counts[i], primes[i] + extra), primes[i]))


# --------------------------------------------------------------------------------------
# Pairs, sieve and roots (section 2 bit sieve, section 5 search loop)
# --------------------------------------------------------------------------------------

def row_pairs(p: int, rng: dict) -> np.ndarray:
    """The q of row p inside range ``rng`` that are sieved: q in [q_lo, q_hi], q < p
    if q_lt_p (q <= p with allow_diagonal), gcd(p, q) = 1 and q != p, plus q = p when
    allow_diagonal.  Returned ascending as int64."""
    q_lo, q_hi = rng["q_lo"], rng["q_hi"]
    diag = bool(rng.get("allow_diagonal", False))
    if rng.get("q_lt_p", False):
        q_hi = min(q_hi, p if diag else p - 1)
    if q_hi < q_lo:
        return np.zeros(0, dtype=np.int64)
    q = np.arange(q_lo, q_hi + 1, dtype=np.int64)
    keep = (np.gcd(q, p) == 1) & (q != p)
    if diag:
        keep |= (q == p)
    return q[keep]


def pairs_in_range(rng: dict):
    """All sieved pairs (p, q) of a range, in (p, q) order, pure Python."""
    diag = bool(rng.get("allow_diagonal", False))
    for p in range(rng["p_lo"], rng["p_hi"] + 1):
        for q in range(rng["q_lo"], rng["q_hi"] + 1):
            if rng.get("q_lt_p", False) and not (q < p or (diag and q == p)):
                continue
            if p == q:
                if diag:
                    yield (p, q)
                continue
            if gcd(p, q) == 1:
                yield (p, q)


def sieve_range(tables: Tables, rng: dict):
    """Sieve one range (section 2, section 5): every pair tries the primes in the
    effective order; the first prime whose unsolvability bit is 1 gets the pair's count;
    a pair no prime rejects is a survivor.  Rows are vectorised over q with numpy, which
    keeps each pair's prime order.  Returns (n_pairs, counts[caller order], survivors)."""
    n = len(tables.primes)
    counts = [0] * n
    survivors: list[tuple[int, int]] = []
    n_pairs = 0
    for p in range(rng["p_lo"], rng["p_hi"] + 1):
        alive = row_pairs(p, rng)
        n_pairs += int(alive.size)
        for i in tables.order:
            if alive.size == 0:
                break
            rej = tables.lookup(i, p, alive).astype(bool)
            counts[i] += int(rej.sum())
            alive = alive[~rej]
        survivors.extend((p, int(q)) for q in alive)
    return n_pairs, counts, survivors


def sieve_range_pairwise(tables: Tables, rng: dict):
    """The same sieve one pair at a time, pure Python (for small ranges)."""
    n = len(tables.primes)
    counts = [0] * n
    survivors = []
    n_pairs = 0
    for (p, q) in pairs_in_range(rng):
        n_pairs += 1
        for i in tables.order:
            if tables.bit(i, p, q):
                counts[i] += 1
                break
        else:
            survivors.append((p, q))
    return n_pairs, counts, survivors


def _factor(n: int) -> dict[int, int]:
    f: dict[int, int] = {}
    d = 2
    while d * d <= n:
        while n % d == 0:
            f[d] = f.get(d, 0) + 1
            n //= d
        d += 1
    if n > 1:
        f[n] = f.get(n, 0) + 1
    return f


def _ceil_root(x: int, k: int) -> int:
    """Smallest integer y >= 0 with y^k >= x (exact integer Newton iteration)."""
    if x <= 0:
        return 0
    y = 1 << ((x.bit_length() + k - 1) // k)       # y^k >= x
    while True:
        z = ((k - 1) * y + x // y ** (k - 1)) // k
        if z >= y:
            break
        y = z                                        # y = floor(x^(1/k)) on exit
    return y if y ** k >= x else y + 1


def root_bound_u(p: int, q: int) -> int:
    """An integer U such that every positive real root u of R(u) = Q_pq(sqrt(u)) is
    <= U.  R is monic of degree 5 with coefficients a_j (j = 0..4); if u > 0 and
    u^(5-j) > 5 |a_j| for every j, then |sum_j a_j u^j| < u^5 and R(u) > 0.  So
    U = max_j ceil((5 |a_j|)^(1/(5-j)))."""
    c = q_coefficients(p, q)
    a = {0: c[0], 1: c[2], 2: c[4], 3: c[6], 4: c[8]}
    return max(_ceil_root(5 * abs(a[j]), 5 - j) for j in range(5))


def integer_roots(p: int, q: int) -> list[int]:
    """All integer t > 0 with Q_pq(t) = 0, ascending (rational root theorem).

    Q is monic and even, Q(t) = R(t^2); an integer root u = t^2 of the monic R divides
    R(0) = -p^10 q^10, hence t divides (pq)^5.  Every divisor d of (pq)^5 with
    d^2 <= root_bound_u(p, q) is evaluated exactly.  Needs p, q >= 1."""
    if p < 1 or q < 1:
        raise ValueError("integer_roots needs p, q >= 1")
    tmax = isqrt(root_bound_u(p, q))
    fac: dict[int, int] = {}
    for x in (p, q):
        for f, e in _factor(x).items():
            fac[f] = fac.get(f, 0) + 5 * e
    items = sorted(fac.items())
    roots = []

    def walk(i: int, d: int) -> None:
        if i == len(items):
            if q_value(p, q, d) == 0:
                roots.append(d)
            return
        f, e = items[i]
        x = d
        for _ in range(e + 1):
            if x > tmax:
                break
            walk(i + 1, x)
            x *= f

    walk(0, 1)
    return sorted(roots)


def integer_roots_scan(p: int, q: int) -> list[int]:
    """Brute force: every t in [1, isqrt(root_bound_u)] evaluated exactly (tiny p, q)."""
    tmax = isqrt(root_bound_u(p, q))
    return [t for t in range(1, tmax + 1) if q_value(p, q, t) == 0]


# --------------------------------------------------------------------------------------
# Whole runs
# --------------------------------------------------------------------------------------

def run(primes, ranges, by_density: bool = False, tables: Tables | None = None,
        pairwise: bool = False) -> dict:
    """Sieve every range and test the survivors for integer roots.

    Returns {"order": [...], "ranges": [{"n_pairs", "counts", "survivors", "roots"}]}
    with counts in the caller's prime order, survivors as sorted (p, q) and roots as
    sorted (p, q, t)."""
    tables = tables or Tables(primes, by_density)
    out = []
    for rng in ranges:
        n_pairs, counts, surv = (sieve_range_pairwise if pairwise else sieve_range)(tables, rng)
        surv = sorted(surv)
        roots = sorted((p, q, t) for (p, q) in surv for t in integer_roots(p, q))
        out.append({"n_pairs": n_pairs, "counts": counts, "survivors": surv, "roots": roots})
    return {"order": list(tables.order), "ranges": out}


# --------------------------------------------------------------------------------------
# The region of Theorem 1.2 and the search loop of section 5
# --------------------------------------------------------------------------------------

REGION_SLOPE = 59          # the factor 59 of Eq. 1.2 (q <= 59 p and q >= p / 59)
REGION_CUBE_DIVISOR = 9    # the 9 of cbrt(p / 9) in Eq. 1.2


def region_q_bounds(p: int) -> tuple[int, int]:
    """Integer segment [q_lo, q_hi] of row p in the region of Eq. 1.2,
    min(cbrt(p/9), p/59) <= q <= 59 p, for p >= 1.  An integer q >= 1 satisfies
    q >= cbrt(p/9) iff 9 q^3 >= p iff q^3 >= ceil(p/9), and q >= p/59 iff q >= ceil(p/59);
    q is at least one of them iff it is at least the smaller of the two integer bounds."""
    q_cube = _ceil_root(-(-p // REGION_CUBE_DIVISOR), 3)
    q_lin = -(-p // REGION_SLOPE)
    return max(1, min(q_cube, q_lin)), REGION_SLOPE * p


def region_rows(p_from: int, p_to: int, q_from: int = 0) -> list[dict]:
    """One inclusive range per row p_from..p_to over its segment of Eq. 1.2 (row p_from
    from max(q_from, q_lo) on): the rows the search of section 5 walks."""
    out = []
    for p in range(p_from, p_to + 1):
        lo, hi = region_q_bounds(p)
        if p == p_from:
            lo = max(lo, q_from)
        if lo <= hi:
            out.append({"p_lo": p, "p_hi": p, "q_lo": lo, "q_hi": hi})
    return out


def deepest_prime(tables: Tables, counts, n_surv: int) -> tuple[int, int]:
    """(depth, r_max): the 1-based position in the effective order of the last prime that
    rejected some pair (every prime when a pair survived), and that prime; (0, 0) if no
    pair was sieved.  This is the "depth" of section 6 and the r_max of section 5."""
    depth = len(tables.order) if n_surv else 0
    if not n_surv:
        for e, i in enumerate(tables.order):
            if counts[i]:
                depth = e + 1
    return depth, (tables.primes[tables.order[depth - 1]] if depth else 0)


def region_scan(tables: Tables, p_from: int, p_to: int, q_from: int = 0) -> dict:
    """The section 5 search over rows p_from..p_to of the region of Theorem 1.2: each row
    over its segment of Eq. 1.2, sieved with the bit sieve of section 2, survivors tested
    for integer roots.  Returns pairs, counts (caller order), survivors, roots, depth and
    r_max over the whole scan."""
    n = len(tables.primes)
    counts = [0] * n
    n_pairs = 0
    surv: list[tuple[int, int]] = []
    for rng in region_rows(p_from, p_to, q_from):
        k, c, s = sieve_range(tables, rng)
        n_pairs += k
        counts = [a + b for a, b in zip(counts, c)]
        surv.extend(s)
    roots = sorted((p, q, t) for (p, q) in surv for t in integer_roots(p, q))
    depth, r_max = deepest_prime(tables, counts, len(surv))
    return {"pairs": n_pairs, "counts": counts, "survivors": surv, "roots": roots,
            "depth": depth, "r_max": r_max}


def region_pair_count(p_from: int, p_to: int) -> int:
    """Number of coprime pairs p != q in rows p_from..p_to of the region of Eq. 1.2,
    by Moebius inversion over the squarefree divisors d of p: the integers of [lo, hi]
    prime to p number sum_{d | p} mu(d) (floor(hi/d) - floor((lo-1)/d)).  The pair (1, 1)
    is coprime but diagonal and is removed."""
    spf = list(range(p_to + 1))                      # smallest prime factor sieve
    for i in range(2, isqrt(p_to) + 1):
        if spf[i] == i:
            for j in range(i * i, p_to + 1, i):
                if spf[j] == j:
                    spf[j] = i
    total = 0
    for p in range(p_from, p_to + 1):
        lo, hi = region_q_bounds(p)
        rad = []
        m = p
        while m > 1:
            f = spf[m]
            rad.append(f)
            while m % f == 0:
                m //= f
        divs = [(1, 1)]
        for f in rad:
            divs += [(d * f, -s) for (d, s) in divs]
        total += sum(s * (hi // d - (lo - 1) // d) for (d, s) in divs)
        if lo <= p <= hi and p == 1:
            total -= 1
    return total


def coprime_count(p: int, q_lo: int, q_hi: int) -> int:
    """Number of q in [q_lo, q_hi] with gcd(p, q) = 1 (the pairs of row p that are sieved,
    before the p != q rule), by Moebius inversion over the squarefree divisors d of p:
    sum_{d | p} mu(d) (floor(q_hi / d) - floor((q_lo - 1) / d)).  Any size of q."""
    divs = [(1, 1)]
    for f in _factor(p):
        divs += [(d * f, -s) for (d, s) in divs]
    return sum(s * (q_hi // d - (q_lo - 1) // d) for (d, s) in divs) if q_hi >= q_lo else 0


# --------------------------------------------------------------------------------------
# The paper's table files (section 2, section 3)
# --------------------------------------------------------------------------------------

PRIMES_RECORD = "<hxxI"    # C struct {short prime; unsigned int offset;}: 8 bytes, 2 padding


def full_table(r: int) -> np.ndarray:
    """u_r by Definition 1.1 for r <= FULL_TABLE_LIMIT, else from v_r by homogeneity."""
    return unsolvable_table(r) if r <= FULL_TABLE_LIMIT else full_from_reduced(r, reduced_table(r))


def paper_table_files(primes) -> tuple[bytes, bytes]:
    """(bit tables file, primes file) for the primes in the given order: the Eq. 2.6
    bytes of each u_r back to back, and per prime the record (r, byte offset)."""
    import struct
    blob, recs = bytearray(), bytearray()
    for r in primes:
        recs += struct.pack(PRIMES_RECORD, r, len(blob))
        blob += pack_table_bytes(full_table(r))
    return bytes(blob), bytes(recs)


def read_paper_table_files(blob: bytes, recs: bytes) -> list[tuple[int, np.ndarray]]:
    """Inverse of ``paper_table_files``: [(r, u_r as uint8 [p~][q~])] in file order."""
    import struct
    out = []
    size = struct.calcsize(PRIMES_RECORD)
    for k in range(0, len(recs), size):
        r, off = struct.unpack(PRIMES_RECORD, recs[k:k + size])
        nb = (r * r + 7) // 8
        bits = [(blob[off + i // 8] >> (i % 8)) & 1 for i in range(r * r)]
        out.append((r, np.array(bits, dtype=np.uint8).reshape(r, r)))
    return out


# --------------------------------------------------------------------------------------
# Theorem 1.1: which roots would give a perfect cuboid
# --------------------------------------------------------------------------------------

def theorem_1_1_holds(p: int, q: int, t: int) -> bool:
    """The inequalities of Theorem 1.1 on a positive root t of Q_pq: t > p^2, t > p q,
    t > q^2 and (p^2 + t)(p q + t) > 2 t^2 (exact integers).  With a coprime p != q
    such a root is equivalent to a perfect cuboid."""
    return t > p * p and t > p * q and t > q * q and (p * p + t) * (p * q + t) > 2 * t * t
