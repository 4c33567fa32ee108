"""Serving loop (continuous batching) and autotuner on the GPU.

* Every query's result is the same served in a mix as served alone, and equals the
  oracle's stored result.
* Admission control refuses queries beyond the slot limit (EBUSY) and admits them later.
* Status codes: bad ranges, unknown tickets, busy tables, bounded shutdown.
* The autotuner returns a shape under which the results stay identical.
"""
import json
import os
import time

import pytest

import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1601_00636_gb300 as cb
    torch.cuda.set_device(0)
    return cb, torch.cuda.current_stream()


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(GOLDEN, "c5_small_queries.json")) as f:
        return json.load(f)


def _wait(cb, srv, tickets, n_primes, timeout=60.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for tk in tickets:
            if tk in out:
                continue
            res = cb.cuboid_server_poll(srv, tk)
            if res is not None:
                st = cb.cuboid_result_wait(res)
                out[tk] = (st, cb.cuboid_result_get(res, 0, n_primes))
                cb.cuboid_result_free(res)
        assert time.time() - t0 < timeout, "server did not finish in time"
        time.sleep(0.0005)
    return [out[tk] for tk in tickets]


def _same(got, want):
    assert got["n_pairs"] == want["n_pairs"]
    assert got["counts"] == want["counts"]
    assert [tuple(x) for x in got["survivors"]] == [tuple(x) for x in want["survivors"]]
    assert [tuple(x) for x in got["roots"]] == [tuple(x) for x in want["roots"]]


def test_served_mix_equals_alone_and_oracle(env, golden):
    cb, stream = env
    primes = golden["primes"]
    t = cb.cuboid_tables_build(primes, 0, stream)
    srv = cb.cuboid_server_create(t, 0, 256)
    try:
        mix = [cb.cuboid_server_submit(srv, q) for q in golden["ranges"]]
        assert all(tk is not None for tk in mix)
        got_mix = _wait(cb, srv, mix, len(primes))
        got_alone = []
        for q in golden["ranges"]:
            tk = cb.cuboid_server_submit(srv, q)
            got_alone.append(_wait(cb, srv, [tk], len(primes))[0])
        for (st1, a), (st2, b), want in zip(got_mix, got_alone, golden["results"]):
            assert st1 == st2 == cb.OK
            _same(a, want)
            _same(b, want)
        stats = cb.cuboid_server_stats(srv)
        assert stats["admitted"] == stats["finished"] == 2 * len(golden["ranges"])
        assert stats["in_flight"] == 0 and stats["batches"] >= 2
    finally:
        assert cb.cuboid_server_destroy(srv, 60000) == cb.OK
        cb.cuboid_tables_free(t)


def test_admission_refuses_beyond_slots(env, golden):
    cb, stream = env
    primes = golden["primes"]
    t = cb.cuboid_tables_build(primes, 0, stream)
    srv = cb.cuboid_server_create(t, 0, 4)
    try:
        big = W.rect(1, 1 << 16, 1, 1 << 16)     # ~3e9 pairs: keeps the slots busy for a while
        tickets, refused = [], 0
        for _ in range(12):
            tk = cb.cuboid_server_submit(srv, big)
            if tk is None:
                refused += 1
            else:
                tickets.append(tk)
        assert refused > 0 and len(tickets) <= 4
        res = _wait(cb, srv, tickets, len(primes))
        first = res[0][1]
        for st, r in res:
            assert st == cb.OK and r["counts"] == first["counts"]
        assert cb.cuboid_server_stats(srv)["refused"] == refused
        tk = cb.cuboid_server_submit(srv, big)    # slots free again
        assert tk is not None
        _wait(cb, srv, [tk], len(primes))
    finally:
        assert cb.cuboid_server_destroy(srv, 60000) == cb.OK
        cb.cuboid_tables_free(t)


def test_server_status_codes(env):
    cb, stream = env
    t = cb.cuboid_tables_build(W.first_odd_primes(24), 0, stream)
    srv = cb.cuboid_server_create(t, 0, 16)
    try:
        with pytest.raises(cb.CuboidError) as e:
            cb.cuboid_server_submit(srv, W.rect(5, 4, 1, 2))
        assert e.value.status == cb.ERANGE
        with pytest.raises(cb.CuboidError) as e:
            cb.cuboid_server_poll(srv, 987654321)
        assert e.value.status == cb.EINVAL
        assert cb.cuboid_tables_free(t) == cb.EBUSY
        # a long query keeps the server busy: a zero-wait shutdown reports ETIMEOUT
        tk = cb.cuboid_server_submit(srv, W.rect(2, 1 << 18, 1, (1 << 18) - 1, q_lt_p=True))
        assert tk is not None
        assert cb.cuboid_server_destroy(srv, 0) == cb.ETIMEOUT
        _wait(cb, srv, [tk], 24)
    finally:
        assert cb.cuboid_server_destroy(srv, 60000) == cb.OK
    assert cb.cuboid_tables_free(t) == cb.OK


def test_autotune_keeps_results(env, tmp_path):
    cb, stream = env
    g = json.load(open(os.path.join(GOLDEN, "c3_small_rects.json")))
    t = cb.cuboid_tables_build(g["primes"], 0, stream)
    try:
        cache = str(tmp_path / "tune.txt")
        tune, ms = cb.cuboid_autotune(t, g["ranges"], cb.MODE_BATCHED, stream, cache)
        assert ms > 0 and tune["block_threads"] in (256, 512)
        assert cb.cuboid_tables_get_tuning(t) == tune
        tune2, ms2 = cb.cuboid_autotune(t, g["ranges"], cb.MODE_BATCHED, stream, cache)   # cache hit
        assert tune2 == tune and abs(ms2 - ms) < 1e-3
        res = cb.cuboid_sieve_batch(t, g["ranges"], stream)
        assert cb.cuboid_result_wait(res) == cb.OK
        for i, want in enumerate(g["results"]):
            _same(cb.cuboid_result_get(res, i, len(g["primes"])), want)
        cb.cuboid_result_free(res)
    finally:
        cb.cuboid_tables_free(t)
