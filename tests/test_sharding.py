"""Sharding of ranges across ranks (CPU): the shards from cuboid_shard_range partition a
range, carry balanced lattice-point loads, and -- sieved by separate gloo ranks and merged
with one reduction of counts and a gather of survivor lists -- reproduce the whole
range's result."""
import os
import random
import socket

import pytest

import workloads as W


@pytest.fixture(scope="module")
def cb():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_1601_00636_gb300 as cb
    return cb


def _points(r):
    """Lattice points of a range by brute force (before coprimality)."""
    n = 0
    diag = r.get("allow_diagonal", False)
    for p in range(r["p_lo"], r["p_hi"] + 1):
        hi = r["q_hi"]
        if r.get("q_lt_p"):
            hi = min(hi, p if diag else p - 1)
        n += max(0, hi - r["q_lo"] + 1)
    return n


def _cells(r):
    diag = r.get("allow_diagonal", False)
    out = set()
    for p in range(r["p_lo"], r["p_hi"] + 1):
        hi = r["q_hi"]
        if r.get("q_lt_p"):
            hi = min(hi, p if diag else p - 1)
        for q in range(r["q_lo"], hi + 1):
            out.add((p, q))
    return out


RANGES = [W.triangle(300), W.rect(1, 200, 1, 150, q_lt_p=True, allow_diagonal=True),
          W.rect(10, 400, 5, 30), W.rect(7, 9, 1, 500), W.rect(100, 100, 1, 10), W.triangle(3),
          W.rect(50, 120, 60, 300, q_lt_p=True)]


@pytest.mark.parametrize("rng", RANGES)
@pytest.mark.parametrize("k", [1, 2, 3, 7, 16])
def test_shards_partition_and_balance(cb, rng, k):
    whole = _cells(rng)
    seen = set()
    loads = []
    for i in range(k):
        s, pts = cb.cuboid_shard_range(rng, k, i)
        if s is None:
            loads.append(0)
            continue
        c = _cells(s)
        assert not (c & seen)
        seen |= c
        assert pts == len(c) == _points(s)
        loads.append(pts)
    assert seen == whole
    longest_row = max(rng["q_hi"] - rng["q_lo"] + 1, rng["p_hi"] - rng["p_lo"] + 1)
    assert max(loads) - min(loads) <= 2 * longest_row + 1


def test_shard_errors(cb):
    import ctypes
    r = cb.range_from_dict(W.triangle(10))
    out = cb.cuboid_range()
    assert cb._lib.cuboid_shard_range(ctypes.byref(r), 0, 0, ctypes.byref(out), None) == cb.EINVAL
    assert cb._lib.cuboid_shard_range(ctypes.byref(r), 2, 2, ctypes.byref(out), None) == cb.EINVAL
    bad = cb.make_range(5, 4, 1, 2)
    assert cb._lib.cuboid_shard_range(ctypes.byref(bad), 2, 0, ctypes.byref(out), None) == cb.ERANGE


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, rng, primes, q):
    import torch
    import torch.distributed as dist

    import oracle as O
    import paper_1601_00636_gb300 as cb
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shard, _ = cb.cuboid_shard_range(rng, world, rank)
        if shard is None:
            n_pairs, counts, surv = 0, [0] * len(primes), []
        else:
            n_pairs, counts, surv = O.sieve_range(O.Tables(primes), shard)
        t = torch.tensor([n_pairs] + counts, dtype=torch.int64)
        dist.all_reduce(t)                      # the one reduction: counts and pair totals
        gathered = [None] * world
        dist.all_gather_object(gathered, surv)  # survivor lists are concatenated
        if rank == 0:
            q.put((t.tolist(), sorted(s for part in gathered for s in part)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("rng,primes", [(W.triangle(240), W.first_odd_primes(24)),
                                        (W.rect(1, 60, 1, 60, allow_diagonal=True), [13, 17])])
def test_two_gloo_ranks_merge_to_the_whole(cb, rng, primes):
    import torch.multiprocessing as mp

    import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, rng, primes, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    n_pairs, counts, surv = O.sieve_range(O.Tables(primes), rng)
    assert got[0] == [n_pairs] + counts
    assert got[1] == sorted(surv)
