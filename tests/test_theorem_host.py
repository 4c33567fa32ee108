"""Theorem 1.1 on roots, host side of the library (no GPU) against the oracle, on the
thresholds of each inequality and on 128-bit t."""
import random

import oracle as O


def test_theorem11_flags_match_oracle():
    import paper_1601_00636_gb300 as cb
    g = random.Random(3)
    roots = []
    for _ in range(3000):
        p, q = g.randint(1, 2 ** 32 - 1), g.randint(1, 2 ** 32 - 1)
        lo = max(p * p, p * q, q * q)
        b, c = p * p + p * q, p ** 3 * q
        x = (b + int((b * b + 4 * c) ** 0.5)) // 2          # near the quadratic's threshold
        for t in (lo - 1, lo, lo + 1, x - 2, x - 1, x, x + 1, x + 2, g.randint(1, 2 ** 128 - 1)):
            if 0 < t < 2 ** 128:
                roots.append((p, q, t))
    for k in (1, 5, 2 ** 32 - 1):
        roots.append((k, k, k * k))
    roots += [(2, 1, t) for t in range(1, 12)] + [(1, 2, 0)]
    got = cb.cuboid_theorem11_flags(roots)
    want = [O.theorem_1_1_holds(p, q, t) for p, q, t in roots]
    assert got == want
    assert any(want) and not all(want)
    assert cb.cuboid_theorem11_flags([]) == []
