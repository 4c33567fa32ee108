"""Seeded synthetic workloads for the modulo-primes cuboid sieve.

This module only generates inputs: prime lists and (p, q) range descriptors shaped like
the search of the paper (the region scan of its section 5 and the statistics of its
section 6).  It holds none of the method's arithmetic (no polynomial, no table, no sieve)
and is shared by the tests, the benchmark and the oracle.  Ranges are plain dicts with
inclusive bounds::

    {"p_lo": int, "p_hi": int, "q_lo": int, "q_hi": int,
     "q_lt_p": bool, "allow_diagonal": bool}

Workload recipes (all bounds inclusive, every pair coprime with p != q unless the range
asks for the diagonal):

* ``triangle(n_max)``: all pairs 1 <= q < p <= n_max.
* ``c1``: triangle(200) with the first 24 odd primes (3..97).
* ``c2``: triangle(2**14) with the first 64 odd primes (3..313).
* ``c3``: 4096 rectangles, area 2**U(8, 22), log2(width_q) ~ U(0, log2 area), width
  clipped to [1, 2**20 - 1], height_p = ceil(area / width), corners uniform so that
  p_hi, q_hi < 2**20; first 128 odd primes (3..727).
* ``c4``: triangle(2**20) with the first 256 odd primes (3..1621).
* ``c5``: a Poisson stream of range queries, area 2**U(10, 26), p, q < 2**24, first 128
  odd primes.

Seeds default to 20160401 and the generator is numpy's PCG64.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 20160401


def first_odd_primes(n: int) -> list[int]:
    """The first ``n`` odd primes (3, 5, 7, ...), by trial division."""
    out: list[int] = []
    c = 3
    while len(out) < n:
        if all(c % f for f in range(3, math.isqrt(c) + 1, 2)):
            out.append(c)
        c += 2
    return out


def primes_between(lo: int, hi: int) -> list[int]:
    """All primes in [lo, hi], by trial division (used for the paper's 11..541 set)."""
    return [c for c in range(max(lo, 2), hi + 1)
            if c == 2 or (c % 2 and all(c % f for f in range(3, math.isqrt(c) + 1, 2)))]


def rng(seed: int = DEFAULT_SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def rect(p_lo: int, p_hi: int, q_lo: int, q_hi: int, q_lt_p: bool = False,
         allow_diagonal: bool = False) -> dict:
    return {"p_lo": int(p_lo), "p_hi": int(p_hi), "q_lo": int(q_lo), "q_hi": int(q_hi),
            "q_lt_p": bool(q_lt_p), "allow_diagonal": bool(allow_diagonal)}


def triangle(n_max: int) -> dict:
    """All pairs 1 <= q < p <= n_max."""
    return rect(2, n_max, 1, n_max - 1, q_lt_p=True)


def lattice_points(r: dict) -> int:
    """Lattice points of a range's rectangle (its area; a size for scheduling work)."""
    return (r["p_hi"] - r["p_lo"] + 1) * (r["q_hi"] - r["q_lo"] + 1)


def c1() -> dict:
    return {"name": "c1_triangle200_24primes", "primes": first_odd_primes(24),
            "ranges": [triangle(200)]}


def c2() -> dict:
    return {"name": "c2_triangle16384_64primes", "primes": first_odd_primes(64),
            "ranges": [triangle(1 << 14)]}


def batched_rectangles(n: int = 4096, seed: int = DEFAULT_SEED, log2_area=(8.0, 22.0),
                       limit: int = 1 << 20) -> list[dict]:
    """Rectangles with log-uniform area and log-uniform aspect, corners uniform."""
    g = rng(seed)
    la = g.uniform(log2_area[0], log2_area[1], size=n)
    lw = g.uniform(0.0, 1.0, size=n) * la
    out = []
    for i in range(n):
        area = 2.0 ** la[i]
        w = int(min(max(round(2.0 ** lw[i]), 1), limit - 1))
        h = int(min(max(math.ceil(area / w), 1), limit - 1))
        p_lo = int(g.integers(1, limit - h + 1))
        q_lo = int(g.integers(1, limit - w + 1))
        out.append(rect(p_lo, p_lo + h - 1, q_lo, q_lo + w - 1))
    return out


def c3(n: int = 4096, seed: int = DEFAULT_SEED) -> dict:
    return {"name": "c3_4096rects_p2^20_128primes", "primes": first_odd_primes(128),
            "ranges": batched_rectangles(n, seed)}


def c4() -> dict:
    return {"name": "c4_triangle2^20_256primes", "primes": first_odd_primes(256),
            "ranges": [triangle(1 << 20)]}


def sampled_rows(n_max: int, k: int, seed: int = DEFAULT_SEED) -> list[dict]:
    """k distinct full rows p (2 <= p <= n_max) of a triangle, each as its own range."""
    g = rng(seed)
    ps = sorted(int(x) for x in g.choice(np.arange(2, n_max + 1), size=k, replace=False))
    return [rect(p, p, 1, p - 1, q_lt_p=True) for p in ps]


def poisson_queries(rate: float, n: int, seed: int = DEFAULT_SEED, log2_area=(10.0, 26.0),
                    limit: int = 1 << 24) -> list[dict]:
    """A Poisson stream of range queries: each has an arrival time ``t`` (seconds)."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    rects = batched_rectangles(n, seed + 1, log2_area, limit)
    for i, r in enumerate(rects):
        r["t"] = float(t[i])
    return rects


def c5(rate: float = 1e3, n: int = 10000, seed: int = DEFAULT_SEED) -> dict:
    return {"name": f"c5_serving_rate{rate:g}_128primes", "primes": first_odd_primes(128),
            "ranges": poisson_queries(rate, n, seed)}


def paper_region_rows(p_lo: int, p_hi: int) -> list[dict]:
    """Rows of the region of Theorem 1.2 for p >= 152 (the segment of Eq. 5.2):
    ceil(cbrt(p/9)) <= q <= 59 p, one range per row."""
    out = []
    for p in range(p_lo, p_hi + 1):
        q_lo = 1
        while q_lo ** 3 * 9 < p:
            q_lo += 1
        out.append(rect(p, p, q_lo, 59 * p))
    return out
