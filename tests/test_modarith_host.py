"""The root test's 62-bit modular arithmetic, compiled for the host from the same source,
against Python's exact integers (CPU only): Montgomery products, the reduction of a 64-bit
word, Garner's mixed-radix sign, and the moduli themselves."""
import random

import pytest

sympy = pytest.importorskip("sympy")


@pytest.fixture(scope="module")
def cb():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_1601_00636_gb300 as cb
    return cb


EDGE = [0, 1, 2, (1 << 61) - 1, 1 << 61, (1 << 62) - 1, 1 << 62, (1 << 63) - 1, 1 << 63, (1 << 64) - 1]


def test_moduli_are_the_14_largest_primes_below_2_62(cb):
    mods = cb.cuboid_probe_modarith(3, 0)
    want, m = [], 1 << 62
    for _ in range(14):
        m = sympy.prevprime(m)
        want.append(m)
    assert mods == want
    assert all((1 << 61) < x < (1 << 62) for x in mods)


@pytest.mark.parametrize("device", [False])
def test_products_and_reductions(cb, device):
    mods = cb.cuboid_probe_modarith(3, 0)
    g = random.Random(62)
    for j, m in enumerate(mods):
        a = EDGE + [m - 1, m, m + 1, 2 * m - 1, 4 * m, 8 * m - 1] + [g.getrandbits(64) for _ in range(400)]
        b = list(reversed(a))
        a = [x % (1 << 64) for x in a]
        b = [x % (1 << 64) for x in b]
        assert cb.cuboid_probe_modarith(0, j, a, b, device=device) == [x * y % m for x, y in zip(a, b)]
        assert cb.cuboid_probe_modarith(1, j, a, device=device) == [x % m for x in a]


def _sign_cases(mods, K, g, count):
    P = 1
    for m in mods[:K]:
        P *= m
    half = (P - 1) // 2
    xs = [0, 1, -1, half, -half, half - 1, -half + 1] + [g.randrange(-half, half + 1) for _ in range(count)]
    xs += [g.choice([-1, 1]) * g.getrandbits(g.randrange(1, P.bit_length())) % (half + 1) for _ in range(count)]
    flat = []
    for x in xs:
        flat += [x % m for m in mods[:K]]
    want = [0 if x == 0 else (1 if x > 0 else (1 << 64) - 1) for x in xs]
    return flat, want


@pytest.mark.parametrize("K", [1, 2, 4, 6, 8, 12, 14])
def test_garner_sign(cb, K):
    """The sign of an integer below half the moduli's product from its residues."""
    mods = cb.cuboid_probe_modarith(3, 0)
    flat, want = _sign_cases(mods, K, random.Random(K), 300)
    assert cb.cuboid_probe_modarith(2, K, flat) == want
