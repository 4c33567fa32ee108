"""The arithmetic helpers on the GPU against exact references: the sieve's residue routine
against the % operator for every 32-bit n and every modulus the sieve uses it with (the
256 table primes of the largest benchmark list, the largest table prime, and factor-sized
moduli up to 2^32 - 5), and the root test's 62-bit modular arithmetic against Python's
integers."""
import random

import pytest

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


def test_mod_min_every_uint32_for_every_table_prime(cb):
    mods = [2] + W.first_odd_primes(256) + [9689]
    assert cb.cuboid_probe_mod_min(mods) == [0] * len(mods)


def test_mod_min_factor_sized_moduli(cb):
    """Row factors reach 2^32 - 5 (the largest 32-bit prime); reciprocal 1 above 2^31."""
    mods = [65521, 65537, 1000003, (1 << 31) - 1, (1 << 31) + 11, 3221225473, (1 << 32) - 5, 4294967295]
    assert cb.cuboid_probe_mod_min(mods) == [0] * len(mods)


def test_modarith_on_device_matches_python(cb):
    from test_modarith_host import EDGE, _sign_cases
    mods = cb.cuboid_probe_modarith(3, 0)
    g = random.Random(103)
    for j, m in enumerate(mods):
        a = [x % (1 << 64) for x in EDGE + [m - 1, m, m + 1, 8 * m - 1] + [g.getrandbits(64) for _ in range(2000)]]
        b = list(reversed(a))
        assert cb.cuboid_probe_modarith(0, j, a, b, device=True) == [x * y % m for x, y in zip(a, b)]
        assert cb.cuboid_probe_modarith(1, j, a, device=True) == [x % m for x in a]
    for K in (1, 3, 4, 8, 12, 14):
        flat, want = _sign_cases(mods, K, random.Random(K + 50), 1000)
        assert cb.cuboid_probe_modarith(2, K, flat, device=True) == want
