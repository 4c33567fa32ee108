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
        assert ms > 0 and tune["block_threads"] in (256, 320, 512, 640)
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


def test_overflowing_query_does_not_fail_its_batch(env):
    """With the weak table of 13, most pairs survive.  Four queries of ~39k survivors keep
    the server's streams busy while 6 queries of ~34k survivors, 12 small ones and one of
    ~108k survivors queue up and are batched together: the batch's survivor buffer (2^16
    records) overflows.  Every query whose records did not all fit runs again alone; the
    others keep their results.  Each result equals the query sieved alone (with a large
    buffer), except the one that overflows even alone: EOVERFLOW, with exact pair total
    and counts."""
    cb, stream = env
    t = cb.cuboid_tables_build([13], 0, stream)
    srv = cb.cuboid_server_create(t, 0, 256)
    try:
        occupy = [W.rect(1000 + 400 * i, 1299 + 400 * i, 5000, 5299) for i in range(4)]
        medium = [W.rect(2000 + 300 * i, 2279 + 300 * i, 7000, 7279) for i in range(6)]
        small = [W.rect(100 + 20 * i, 109 + 20 * i, 1000, 1099) for i in range(12)]
        big = W.rect(10000, 10499, 20000, 20499)
        queries = occupy + medium[:3] + small[:6] + [big] + medium[3:] + small[6:]
        tickets = [cb.cuboid_server_submit(srv, q) for q in queries]
        assert all(tk is not None for tk in tickets)
        results = _wait(cb, srv, tickets, 1)
        for q, (st, got) in zip(queries, results):
            r = cb.cuboid_sieve(t, q["p_lo"], q["p_hi"], q["q_lo"], q["q_hi"], 0, stream)
            assert cb.cuboid_result_wait(r) == cb.OK
            want = cb.cuboid_result_get(r, 0, 1)
            cb.cuboid_result_free(r)
            if q is big:
                assert st == cb.EOVERFLOW
                assert got["n_pairs"] == want["n_pairs"] and got["counts"] == want["counts"]
                assert len(want["survivors"]) > 1 << 16
            else:
                assert st == cb.OK, q
                _same(got, want)
        stats = cb.cuboid_server_stats(srv)
        assert stats["retried"] >= 1
        assert stats["finished"] == stats["admitted"] == len(queries)
    finally:
        assert cb.cuboid_server_destroy(srv, 60000) == cb.OK
        cb.cuboid_tables_free(t)


def test_replay_matches_polled_results(env, golden):
    """The native load replay: every query finishes, its latency is positive, its pair
    total is the stored oracle result's, and its result stays available to poll."""
    cb, stream = env
    primes = golden["primes"]
    t = cb.cuboid_tables_build(primes, 0, stream)
    srv = cb.cuboid_server_create(t, 0, 256)
    try:
        qs = golden["ranges"]
        r = cb.cuboid_server_replay(srv, qs, [1e-4 * i for i in range(len(qs))], 60000)
        assert all(st == cb.OK for st in r["status"]) and all(x > 0 for x in r["latency_s"])
        assert r["npairs"] == [w["n_pairs"] for w in golden["results"]]
        assert r["wall_s"] >= 1e-4 * (len(qs) - 1)
        for tk, want in zip(r["tickets"], golden["results"]):
            res = cb.cuboid_server_poll(srv, tk)
            assert res is not None and cb.cuboid_result_wait(res) == cb.OK
            _same(cb.cuboid_result_get(res, 0, len(primes)), want)
            cb.cuboid_result_free(res)
        with pytest.raises(Exception):
            cb.cuboid_server_replay(srv, qs[:2], [1.0, 0.5], 1000)  # arrival times must not decrease
    finally:
        assert cb.cuboid_server_destroy(srv, 60000) == cb.OK
        cb.cuboid_tables_free(t)


def test_served_full_size_queries_vs_oracle(env):
    """The 24 full-size serving queries (areas up to 2^26, p, q < 2^24) submitted together
    to the server: each result equals the oracle's stored result."""
    import gzip
    cb, stream = env
    with gzip.open(os.path.join(GOLDEN, "c5_full_queries.json.gz"), "rt") as f:
        g = json.load(f)
    n = len(g["primes"])
    t = cb.cuboid_tables_build(g["primes"], cb.ORDER_BY_RATE, stream)
    srv = cb.cuboid_server_create(t, 0, 256)
    try:
        tickets = [cb.cuboid_server_submit(srv, q) for q in g["ranges"]]
        got = _wait(cb, srv, tickets, n)
        for (st, a), want in zip(got, g["results"]):
            c = [0] * n
            for i, v in want["counts_nz"]:
                c[i] = v
            assert st == cb.OK
            _same(a, {"n_pairs": want["n_pairs"], "counts": c, "survivors": want["survivors"],
                      "roots": want["roots"]})
    finally:
        assert cb.cuboid_server_destroy(srv, 60000) == cb.OK
        cb.cuboid_tables_free(t)
