"""The allocation-free sieve entry point against the regular one.

cuboid_sieve_noalloc exists for callers that may not allocate device memory at the
moment they sieve (latency-bound loops, where cudaMalloc and cudaFree synchronise the
device; hosts that lend the library a fixed pool; processes at their memory limit).
All of its working memory is one static device array shared by every call, so this test
runs it twice in a row on the same inputs and checks each call, output by output,
against cuboid_sieve_batch: counts, pair totals, survivors and roots must be identical
(integer results, so the tolerance is zero).  The file name makes pytest collect it last.
"""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1601_00636_gb300 as cb
    torch.cuda.set_device(0)
    return cb, torch, torch.cuda.current_stream()


def _expected(cb, t, n_primes, ranges, stream):
    res = cb.cuboid_sieve_batch(t, ranges, stream)
    try:
        assert cb.cuboid_result_wait(res) == cb.OK
        return [cb.cuboid_result_get(res, i, n_primes) for i in range(len(ranges))]
    finally:
        cb.cuboid_result_free(res)


def _noalloc(cb, torch, t, n_primes, order, ranges, stream, surv_cap=1 << 17, root_cap=1 << 10):
    n = len(ranges)
    arr = cb.ranges_array(ranges)
    d_ranges = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).cuda()
    counts = torch.full((n * n_primes,), -1, dtype=torch.int64, device="cuda")   # stale contents
    npairs = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    surv = torch.zeros(surv_cap, dtype=torch.int64, device="cuda")
    surv_rng = torch.zeros(surv_cap, dtype=torch.int32, device="cuda")
    roots = torch.zeros(root_cap * 3, dtype=torch.int64, device="cuda")          # 24-byte records
    root_rng = torch.zeros(root_cap, dtype=torch.int32, device="cuda")
    totals = torch.full((3,), -1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    st = cb.cuboid_sieve_noalloc(t, d_ranges.data_ptr(), n, counts.data_ptr(), npairs.data_ptr(),
                                 surv.data_ptr(), surv_rng.data_ptr(), surv_cap, roots.data_ptr(),
                                 root_rng.data_ptr(), root_cap, totals.data_ptr(), stream)
    assert st == cb.OK
    torch.cuda.synchronize()
    n_surv, n_roots, status = (int(x) for x in totals.cpu())
    assert status == 0 and n_surv <= surv_cap and n_roots <= root_cap
    counts = counts.cpu().view(n, n_primes).tolist()
    out = []
    sv = surv.cpu().tolist()[:n_surv]
    sr = surv_rng.cpu().tolist()[:n_surv]
    rv = roots.cpu().view(-1, 3).tolist()[:n_roots]
    rr = root_rng.cpu().tolist()[:n_roots]
    for k in range(n):
        caller = [0] * n_primes
        for e, i in enumerate(order):
            caller[i] = counts[k][e]
        s = sorted(((x >> 32) & 0xFFFFFFFF, x & 0xFFFFFFFF) for x, r in zip(sv, sr) if r == k)
        roots_k = sorted((rec[0] & 0xFFFFFFFF, (rec[0] >> 32) & 0xFFFFFFFF,
                          ((rec[2] & 0xFFFFFFFFFFFFFFFF) << 64) | (rec[1] & 0xFFFFFFFFFFFFFFFF))
                         for rec, r in zip(rv, rr) if r == k)
        out.append({"n_pairs": int(npairs[k]), "counts": caller, "survivors": s, "roots": roots_k})
    return out


def test_noalloc_matches_regular_entry_point_twice(env):
    cb, torch, stream = env
    primes = [13, 17, 19]
    ranges = [W.triangle(300), W.rect(1, 120, 1, 120, allow_diagonal=True), W.rect(5000, 5100, 1, 3000),
              W.rect(700, 760, 10, 4000)]
    t = cb.cuboid_tables_build(primes, cb.ORDER_BY_DENSITY, stream)
    try:
        order = cb.cuboid_tables_order(t)
        want = _expected(cb, t, len(primes), ranges, stream)
        assert any(w["survivors"] for w in want) and any(w["roots"] for w in want)
        for _ in range(2):
            got = _noalloc(cb, torch, t, len(primes), order, ranges, stream)
            for g, w in zip(got, want):
                assert g["n_pairs"] == w["n_pairs"]
                assert g["counts"] == w["counts"]
                assert g["survivors"] == [tuple(x) for x in w["survivors"]]
                assert g["roots"] == [tuple(x) for x in w["roots"]]
    finally:
        cb.cuboid_tables_free(t)


def test_noalloc_rejects_too_many_ranges(env):
    cb, torch, stream = env
    t = cb.cuboid_tables_build([11], 0, stream)
    try:
        n = cb.NOALLOC_MAX_RANGES + 1
        st = cb.cuboid_sieve_noalloc(t, 1, n, 1, 1, 0, 0, 0, 0, 0, 0, 1, stream)
        assert st == cb.ETOOLARGE
    finally:
        cb.cuboid_tables_free(t)


def test_noalloc_at_full_capacity(env):
    """Exactly CUBOID_NOALLOC_MAX_RANGES uneven one-row ranges: the plan fills the last
    slot of the fixed array and the plan's prefix sum runs over more than 1024 ranges."""
    import random
    cb, torch, stream = env
    primes = W.first_odd_primes(8)
    g = random.Random(20160401)
    ranges = []
    for _ in range(cb.NOALLOC_MAX_RANGES):
        p = g.randint(2, 1 << 20)
        lo = g.randint(1, 1 << 20)
        ranges.append(W.rect(p, p, lo, lo + g.choice([0, 1, 63, 64, 200, 1000, 5000])))
    t = cb.cuboid_tables_build(primes, cb.ORDER_BY_RATE, stream)
    try:
        order = cb.cuboid_tables_order(t)
        want = _expected(cb, t, len(primes), ranges, stream)
        for _ in range(2):
            got = _noalloc(cb, torch, t, len(primes), order, ranges, stream)
            assert [g_["n_pairs"] for g_ in got] == [w["n_pairs"] for w in want]
            assert [g_["counts"] for g_ in got] == [w["counts"] for w in want]
            assert [g_["survivors"] for g_ in got] == [[tuple(x) for x in w["survivors"]] for w in want]
            assert [g_["roots"] for g_ in got] == [[tuple(x) for x in w["roots"]] for w in want]
    finally:
        cb.cuboid_tables_free(t)
