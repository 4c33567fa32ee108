"""GPU: the paper's table files (section 2) through the C ABI.

Export must write byte for byte the files the oracle writes (Eq. 2.6 packing, 8-byte
{short prime; unsigned int offset} records); import must make the file's bits the
device tables, so that sieving with imported tables equals the oracle, and the checked
import must refuse a file whose bits differ from the definition.
"""
import hashlib
import json
import os

import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def cb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1601_00636_gb300 as cb
    torch.cuda.set_device(0)
    return cb


def _export(cb, t, tmp_path):
    bits, prim = str(tmp_path / "Cuboid_pq_bit_tables.bin"), str(tmp_path / "Cuboid_primes.bin")
    n = cb.cuboid_tables_export(t, bits, prim)
    return n, open(bits, "rb").read(), open(prim, "rb").read()


@pytest.mark.parametrize("flags", ["reduced", "full"])
def test_export_paper_primes_matches_golden(cb, tmp_path, flags):
    """The 96 primes 11..541 of section 2: both files hash to the oracle's."""
    g = json.load(open(os.path.join(GOLDEN, "paper_files_11_541.json")))
    fl = cb.BUILD_FULL if flags == "full" else cb.BUILD_REDUCED
    t = cb.cuboid_tables_build(g["primes"], fl)
    try:
        n, blob, recs = _export(cb, t, tmp_path)
    finally:
        cb.cuboid_tables_free(t)
    assert n == len(blob) == g["bit_tables_bytes"] and len(recs) == g["primes_bytes"]
    assert hashlib.sha256(blob).hexdigest() == g["bit_tables_sha256"]
    assert hashlib.sha256(recs).hexdigest() == g["primes_sha256"]


def test_export_small_list_bytes(cb, tmp_path):
    primes = [11, 13, 5, 2, 3, 7, 97, 31]
    t = cb.cuboid_tables_build(primes, cb.ORDER_BY_RATE)
    try:
        _, blob, recs = _export(cb, t, tmp_path)
    finally:
        cb.cuboid_tables_free(t)
    assert (blob, recs) == O.paper_table_files(primes)       # caller order, whatever the sieve order


@pytest.mark.parametrize("order", ["given", "rate"])
def test_import_oracle_files_then_sieve(cb, tmp_path, order):
    """Files written by the oracle, imported (checked), sieve the 200-triangle exactly as
    the oracle does; the loader reports the primes file's size."""
    primes = W.first_odd_primes(24)
    blob, recs = O.paper_table_files(primes)
    (tmp_path / "b.bin").write_bytes(blob)
    (tmp_path / "p.bin").write_bytes(recs)
    fl = (cb.ORDER_BY_RATE if order == "rate" else cb.ORDER_AS_GIVEN) | cb.IMPORT_CHECK
    t, nbytes = cb.cuboid_tables_import(str(tmp_path / "b.bin"), str(tmp_path / "p.bin"), fl)
    try:
        assert nbytes == len(recs) == 8 * 24
        n, _, flags = cb.cuboid_tables_info(t)
        assert n == 24 and flags & cb.TABLES_IMPORTED
        T = O.Tables(primes, by_density={"given": False, "rate": "rate"}[order])
        assert cb.cuboid_tables_order(t) == list(T.order)
        for i, r in enumerate(primes):
            assert cb.cuboid_tables_copy_reduced(t, i, r) == bytes(O.reduced_table(r))
        rng = {"p_lo": 1, "p_hi": 200, "q_lo": 1, "q_hi": 200, "q_lt_p": True}
        want = O.run(primes, [rng], tables=T)["ranges"][0]
        res = cb.cuboid_sieve(t, 1, 200, 1, 200, cb.Q_LT_P)
        try:
            cb.cuboid_result_wait(res)
            got = cb.cuboid_result_get(res, 0, 24)
        finally:
            cb.cuboid_result_free(res)
        assert got["n_pairs"] == want["n_pairs"] and got["counts"] == want["counts"]
        assert sorted(got["survivors"]) == want["survivors"] and sorted(got["roots"]) == want["roots"]
    finally:
        cb.cuboid_tables_free(t)


def test_import_uses_the_files_bits(cb, tmp_path):
    """A file with one flipped bit: the unchecked import carries the flipped bit into the
    device tables (export gives the file back unchanged), the checked one gives EVERIFY."""
    primes = [11, 13, 17]
    blob, recs = O.paper_table_files(primes)
    bad = bytearray(blob)
    off13 = (11 * 11 + 7) // 8
    bad[off13 + 3] ^= 0x10
    (tmp_path / "b.bin").write_bytes(bytes(bad))
    (tmp_path / "p.bin").write_bytes(recs)
    st, _ = cb.cuboid_tables_import_status(str(tmp_path / "b.bin"), str(tmp_path / "p.bin"), cb.IMPORT_CHECK)
    assert st == cb.EVERIFY
    t, _ = cb.cuboid_tables_import(str(tmp_path / "b.bin"), str(tmp_path / "p.bin"))
    try:
        d = tmp_path / "out"
        d.mkdir()
        _, blob2, recs2 = _export(cb, t, d)
        assert blob2 == bytes(bad) and recs2 == recs
    finally:
        cb.cuboid_tables_free(t)


def test_export_import_round_trip_paper_primes(cb, tmp_path):
    """Export the section 2 primes, import them back (checked): the region scan of rows
    152..400 gives the same counts with both tables."""
    primes = W.primes_between(11, 541)
    t = cb.cuboid_tables_build(primes, cb.ORDER_AS_GIVEN)
    try:
        _export(cb, t, tmp_path)
        t2, nbytes = cb.cuboid_tables_import(str(tmp_path / "Cuboid_pq_bit_tables.bin"),
                                             str(tmp_path / "Cuboid_primes.bin"), cb.IMPORT_CHECK)
        try:
            assert nbytes == 8 * 96
            a = cb.cuboid_region_scan(t, 152, 400)
            b = cb.cuboid_region_scan(t2, 152, 400)
            assert a[0] == b[0] == 0 and a[1] == b[1] and a[2] == b[2]
        finally:
            cb.cuboid_tables_free(t2)
    finally:
        cb.cuboid_tables_free(t)
