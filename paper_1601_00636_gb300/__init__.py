"""Python binding of libcuboid (the C ABI declared in include/cuboid.h).

Argument marshalling only: every step of the sieve and of the root test runs in the
library's CUDA kernels.  Function names are those of the C ABI.  Importing this package
loads ``libcuboid.so`` built in-tree (``paper_1601_00636_gb300/build.py`` or
``__graft_entry__.build()``) and raises ImportError when it is missing: there is no
CPU fallback.

Streams are passed as ``None`` (legacy default stream), an int handle, or any object
with a ``cuda_stream`` attribute (e.g. ``torch.cuda.Stream``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# CUBOID_DEBUG=1 loads the debug build (index checks in the kernels; build.py --debug)
DEBUG = os.environ.get("CUBOID_DEBUG", "") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "libcuboid_debug.so" if DEBUG else "libcuboid.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1601_00636_gb300/build.py "
                      "or __graft_entry__.build(); there is no CPU fallback")
_lib = C.CDLL(LIB_PATH)

# ------------------------------------------------------------------ constants (cuboid.h)
OK, EBUSY, ERANGE, EPMAX, EQLOW, EQHIGH, ENOTABLES, EINVAL, ENOMEM = 0, 1, 2, 3, 4, 5, 6, 7, 8
ETIMEOUT, ECUDA, EOVERFLOW, EAGAIN, EVERIFY, ETOOLARGE, EINDEX = 9, 10, 11, 12, 13, 14, 15
NOALLOC_MAX_RANGES = 4096
STATUS_NAMES = {0: "OK", 1: "EBUSY", 2: "ERANGE", 3: "EPMAX", 4: "EQLOW", 5: "EQHIGH", 6: "ENOTABLES", 7: "EINVAL", 8: "ENOMEM",
                9: "ETIMEOUT", 10: "ECUDA", 11: "EOVERFLOW", 12: "EAGAIN", 13: "EVERIFY", 14: "ETOOLARGE",
                15: "EINDEX"}

ORDER_AS_GIVEN, ORDER_BY_DENSITY, ORDER_BY_RATE = 0x0, 0x1, 0x4
BUILD_REDUCED, BUILD_FULL = 0x0, 0x2
TABLES_IMPORTED, IMPORT_CHECK = 0x10, 0x8
Q_LT_P, ALLOW_DIAGONAL, ROWS_P, ROWS_Q = 0x1, 0x2, 0x4, 0x8
MODE_PLAIN, MODE_BATCHED, MODE_COUNT_STEPS, MODE_TIME_SIEVE = 0x0, 0x1, 0x100, 0x200
MODE_STAGE_TIMEOUT = 0x400


class CuboidError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")
        self.status = status


def _check(st: int, where: str) -> int:
    if st != OK:
        raise CuboidError(st, where)
    return st


class cuboid_range(C.Structure):
    _fields_ = [("p_lo", C.c_uint32), ("p_hi", C.c_uint32), ("q_lo", C.c_uint32),
                ("q_hi", C.c_uint32), ("flags", C.c_uint32), ("reserved", C.c_uint32)]


class cuboid_root(C.Structure):
    _fields_ = [("p", C.c_uint32), ("q", C.c_uint32), ("t_lo", C.c_uint64), ("t_hi", C.c_uint64)]


class cuboid_range_wide(C.Structure):
    _fields_ = [("p_lo", C.c_uint64), ("p_hi", C.c_uint64), ("q_lo", C.c_uint64),
                ("q_hi", C.c_uint64), ("flags", C.c_uint32), ("reserved", C.c_uint32)]


class cuboid_root_wide(C.Structure):
    _fields_ = [("p", C.c_uint64), ("q", C.c_uint64), ("t_lo", C.c_uint64), ("t_hi", C.c_uint64)]


class cuboid_region_report_wide(C.Structure):
    _fields_ = [("p", C.c_uint64), ("q", C.c_uint64), ("r_max", C.c_uint32), ("depth", C.c_uint32),
                ("pairs", C.c_uint64), ("n_surv", C.c_uint64), ("n_roots", C.c_uint64)]


class cuboid_tuning(C.Structure):
    _fields_ = [("block_threads", C.c_uint32), ("ctas_per_sm", C.c_uint32),
                ("smem_primes", C.c_uint32), ("tiles_per_warp", C.c_uint32),
                ("hot_primes", C.c_uint32), ("row_lanes", C.c_uint32)]


class cuboid_stats(C.Structure):
    _fields_ = [("words", C.c_uint64), ("word_steps", C.c_uint64), ("warp_steps", C.c_uint64),
                ("tiles", C.c_uint64)]


class cuboid_search_report(C.Structure):
    _fields_ = [("p", C.c_uint32), ("q", C.c_uint32), ("r_max", C.c_uint32), ("depth", C.c_uint32),
                ("pairs", C.c_uint64), ("n_surv", C.c_uint64), ("n_roots", C.c_uint64)]


_P = C.c_void_p
_u32, _u64 = C.c_uint32, C.c_uint64
_SIGS = {
    "cuboid_tables_build": (C.c_int, [C.POINTER(_u32), _u32, _u32, _P, C.POINTER(_P)]),
    "cuboid_tables_info": (C.c_int, [_P, C.POINTER(_u32), C.POINTER(_u64), C.POINTER(_u32)]),
    "cuboid_tables_order": (C.c_int, [_P, C.POINTER(_u32)]),
    "cuboid_tables_copy_bits": (C.c_int, [_P, _u32, C.POINTER(C.c_uint8), C.c_size_t, C.POINTER(C.c_size_t)]),
    "cuboid_tables_copy_reduced": (C.c_int, [_P, _u32, C.POINTER(C.c_uint8), C.c_size_t]),
    "cuboid_tables_export": (C.c_int, [_P, C.c_char_p, C.c_char_p, C.POINTER(_u64)]),
    "cuboid_tables_import": (C.c_int, [C.c_char_p, C.c_char_p, _u32, _P, C.POINTER(_P), C.POINTER(_u64)]),
    "cuboid_tables_set_tuning": (C.c_int, [_P, C.POINTER(cuboid_tuning)]),
    "cuboid_tables_get_tuning": (C.c_int, [_P, C.POINTER(cuboid_tuning)]),
    "cuboid_tables_free": (C.c_int, [_P]),
    "cuboid_autotune": (C.c_int, [_P, C.POINTER(cuboid_range), _u32, _u32, _P, C.c_char_p,
                                  C.POINTER(cuboid_tuning), C.POINTER(C.c_float)]),
    "cuboid_result_create": (C.c_int, [_P, _u32, _u64, _u64, C.POINTER(_P)]),
    "cuboid_sieve": (C.c_int, [_P, _u32, _u32, _u32, _u32, _u32, _P, C.POINTER(_P)]),
    "cuboid_sieve_batch": (C.c_int, [_P, C.POINTER(cuboid_range), _u32, _P, C.POINTER(_P)]),
    "cuboid_sieve_into": (C.c_int, [_P, C.POINTER(cuboid_range), _u32, _u32, _P]),
    "cuboid_sieve_device": (C.c_int, [_P, _P, _u32, _u32, _P]),
    "cuboid_result_download": (C.c_int, [_P, _P]),
    "cuboid_result_wait": (C.c_int, [_P]),
    "cuboid_result_get": (C.c_int, [_P, _u32, C.POINTER(_u64), C.POINTER(_u64), C.POINTER(_u64),
                                    C.POINTER(C.POINTER(_u64)), C.POINTER(_u64),
                                    C.POINTER(C.POINTER(cuboid_root))]),
    "cuboid_result_sieve_ms": (C.c_int, [_P, C.POINTER(C.c_float), C.POINTER(_u32)]),
    "cuboid_result_stats": (C.c_int, [_P, C.POINTER(cuboid_stats)]),
    "cuboid_result_free": (C.c_int, [_P]),
    "cuboid_sieve_noalloc": (C.c_int, [_P, _P, _u32, _P, _P, _P, _P, _u64, _P, _P, _u64, _P, _P]),
    "cuboid_region_qmin": (_u32, [_u32]),
    "cuboid_region_scan": (C.c_int, [_P, _u32, _u32, _u32, _P, C.POINTER(_u64), C.POINTER(_u64), _u64,
                                     C.POINTER(cuboid_root), _u64, C.POINTER(cuboid_search_report)]),
    "cuboid_search_start": (C.c_int, [_P, _u32, _u32, C.POINTER(_P)]),
    "cuboid_search_current": (C.c_int, [_P, C.POINTER(_u32), C.POINTER(_u32)]),
    "cuboid_search_stop": (C.c_int, [_P, C.POINTER(cuboid_search_report), C.POINTER(_u64)]),
    "cuboid_search_report_write": (C.c_int, [C.POINTER(cuboid_search_report), C.c_char_p]),
    "cuboid_theorem11_flags": (C.c_int, [C.POINTER(cuboid_root), _u64, C.POINTER(C.c_uint8)]),
    "cuboid_shard_range": (C.c_int, [C.POINTER(cuboid_range), _u32, _u32, C.POINTER(cuboid_range),
                                     C.POINTER(_u64)]),
    "cuboid_verify_pairs": (C.c_int, [C.POINTER(_u32), C.POINTER(_u32), _u32, _P, C.POINTER(cuboid_root),
                                      _u64, C.POINTER(_u64)]),
    "cuboid_wide_pieces": (C.c_int, [C.POINTER(cuboid_range_wide), C.POINTER(cuboid_range), C.POINTER(_u64), _u32,
                                     C.POINTER(_u32)]),
    "cuboid_sieve_wide": (C.c_int, [_P, C.POINTER(cuboid_range_wide), _u32, _P, C.POINTER(_P)]),
    "cuboid_result_get_wide": (C.c_int, [_P, _u32, C.POINTER(_u64), C.POINTER(_u64), C.POINTER(_u64),
                                         C.POINTER(C.POINTER(_u64)), C.POINTER(_u64),
                                         C.POINTER(C.POINTER(cuboid_root_wide))]),
    "cuboid_verify_pairs_wide": (C.c_int, [C.POINTER(_u64), C.POINTER(_u64), _u32, _P,
                                           C.POINTER(cuboid_root_wide), _u64, C.POINTER(_u64)]),
    "cuboid_theorem11_flags_wide": (C.c_int, [C.POINTER(cuboid_root_wide), _u64, C.POINTER(C.c_uint8)]),
    "cuboid_region_scan_wide": (C.c_int, [_P, _u64, _u64, _u64, _P, C.POINTER(_u64), C.POINTER(_u64), _u64,
                                          C.POINTER(cuboid_root_wide), _u64, C.POINTER(cuboid_region_report_wide)]),
    "cuboid_server_create": (C.c_int, [_P, _u64, _u32, C.POINTER(_P)]),
    "cuboid_server_submit": (C.c_int, [_P, C.POINTER(cuboid_range), C.POINTER(_u64)]),
    "cuboid_server_poll": (C.c_int, [_P, _u64, C.POINTER(_P)]),
    "cuboid_server_stats": (C.c_int, [_P, C.POINTER(_u64), C.POINTER(_u64), C.POINTER(_u64),
                                      C.POINTER(_u64), C.POINTER(_u64), C.POINTER(_u64)]),
    "cuboid_server_replay": (C.c_int, [_P, C.c_void_p, C.POINTER(C.c_double), _u32, _u32, C.POINTER(_u64),
                                       C.POINTER(C.c_double), C.POINTER(_u64), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_double), C.POINTER(_u64)]),
    "cuboid_server_destroy": (C.c_int, [_P, _u32]),
    "cuboid_probe_int_issue": (C.c_int, [_u32, _u32, _u32, _u32, _P, _P]),
    "cuboid_probe_mod_min": (C.c_int, [C.POINTER(_u32), _u32, C.POINTER(_u64), _P]),
    "cuboid_probe_modarith": (C.c_int, [_u32, _u32, C.POINTER(_u64), C.POINTER(_u64), _u32, C.POINTER(_u64),
                                        C.c_int]),
    "cuboid_device_sms": (C.c_int, [C.POINTER(_u32)]),
    "cuboid_version": (C.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(getattr(s, "cuda_stream"))


def make_range(p_lo, p_hi, q_lo, q_hi, flags=0) -> cuboid_range:
    return cuboid_range(p_lo, p_hi, q_lo, q_hi, flags, 0)


def range_from_dict(d: dict) -> cuboid_range:
    """A workload range dict (workloads module) as a cuboid_range."""
    fl = (Q_LT_P if d.get("q_lt_p") else 0) | (ALLOW_DIAGONAL if d.get("allow_diagonal") else 0)
    fl |= int(d.get("flags", 0))
    return make_range(d["p_lo"], d["p_hi"], d["q_lo"], d["q_hi"], fl)


def _ranges_array(ranges):
    arr = (cuboid_range * len(ranges))()
    for i, r in enumerate(ranges):
        arr[i] = r if isinstance(r, cuboid_range) else range_from_dict(r)
    return arr


# ------------------------------------------------------------------ tables

def cuboid_tables_build(primes, flags: int = 0, stream=None) -> int:
    n = len(primes)
    arr = (_u32 * n)(*[int(x) for x in primes])
    out = _P()
    _check(_lib.cuboid_tables_build(arr, n, flags, _stream(stream), C.byref(out)), "cuboid_tables_build")
    return out.value


def cuboid_tables_info(t):
    n, b, f = _u32(), _u64(), _u32()
    _check(_lib.cuboid_tables_info(t, C.byref(n), C.byref(b), C.byref(f)), "cuboid_tables_info")
    return n.value, b.value, f.value


def cuboid_tables_order(t) -> list[int]:
    n = cuboid_tables_info(t)[0]
    arr = (_u32 * n)()
    _check(_lib.cuboid_tables_order(t, arr), "cuboid_tables_order")
    return list(arr)


def cuboid_tables_copy_bits(t, prime_idx: int) -> bytes:
    need = C.c_size_t()
    st = _lib.cuboid_tables_copy_bits(t, prime_idx, None, 0, C.byref(need))
    if st not in (OK, EOVERFLOW, EINVAL):
        _check(st, "cuboid_tables_copy_bits")
    buf = (C.c_uint8 * max(need.value, 1))()
    _check(_lib.cuboid_tables_copy_bits(t, prime_idx, buf, need.value, C.byref(need)), "cuboid_tables_copy_bits")
    return bytes(buf[:need.value])


def cuboid_tables_copy_reduced(t, prime_idx: int, r: int) -> bytes:
    buf = (C.c_uint8 * r)()
    _check(_lib.cuboid_tables_copy_reduced(t, prime_idx, buf, r), "cuboid_tables_copy_reduced")
    return bytes(buf)


def cuboid_tables_export(t, bit_tables_path: str, primes_path: str) -> int:
    """Write the paper's two table files; returns the bit tables file's size in bytes."""
    n = _u64()
    _check(_lib.cuboid_tables_export(t, bit_tables_path.encode(), primes_path.encode(), C.byref(n)),
           "cuboid_tables_export")
    return n.value


def cuboid_tables_import(bit_tables_path: str, primes_path: str, flags: int = 0, stream=None):
    """Tables from the paper's two files; returns (handle, bytes of the primes file)."""
    out, n = _P(), _u64()
    _check(_lib.cuboid_tables_import(bit_tables_path.encode(), primes_path.encode(), flags, _stream(stream),
                                     C.byref(out), C.byref(n)), "cuboid_tables_import")
    return out.value, n.value


def cuboid_tables_import_status(bit_tables_path: str, primes_path: str, flags: int = 0, stream=None):
    """As cuboid_tables_import, returning (status, handle or None) instead of raising."""
    out, n = _P(), _u64()
    st = _lib.cuboid_tables_import(bit_tables_path.encode(), primes_path.encode(), flags, _stream(stream),
                                   C.byref(out), C.byref(n))
    return st, (out.value if st == OK else None)


def cuboid_tables_set_tuning(t, block_threads=0, ctas_per_sm=0, smem_primes=0, tiles_per_warp=0, hot_primes=0,
                             row_lanes=0):
    tu = cuboid_tuning(block_threads, ctas_per_sm, smem_primes, tiles_per_warp, hot_primes, row_lanes)
    _check(_lib.cuboid_tables_set_tuning(t, C.byref(tu)), "cuboid_tables_set_tuning")


def cuboid_tables_get_tuning(t) -> dict:
    tu = cuboid_tuning()
    _check(_lib.cuboid_tables_get_tuning(t, C.byref(tu)), "cuboid_tables_get_tuning")
    return {k: getattr(tu, k) for k, _ in cuboid_tuning._fields_}


def cuboid_autotune(t, ranges, mode=MODE_BATCHED, stream=None, cache_path=None):
    """Pick the fastest kernel shape for these ranges; returns (tuning dict, ms)."""
    arr = _ranges_array(ranges)
    tu = cuboid_tuning()
    ms = C.c_float()
    cp = cache_path.encode() if cache_path else None
    _check(_lib.cuboid_autotune(t, arr, len(arr), mode, _stream(stream), cp, C.byref(tu), C.byref(ms)),
           "cuboid_autotune")
    return {k: getattr(tu, k) for k, _ in cuboid_tuning._fields_}, ms.value


def cuboid_tables_free(t) -> int:
    return _lib.cuboid_tables_free(t)


# ------------------------------------------------------------------ sieving

def cuboid_result_create(t, max_ranges: int, surv_cap: int = 0, root_cap: int = 0) -> int:
    out = _P()
    _check(_lib.cuboid_result_create(t, max_ranges, surv_cap, root_cap, C.byref(out)), "cuboid_result_create")
    return out.value


def cuboid_sieve(t, p_lo, p_hi, q_lo, q_hi, flags=0, stream=None) -> int:
    out = _P()
    _check(_lib.cuboid_sieve(t, p_lo, p_hi, q_lo, q_hi, flags, _stream(stream), C.byref(out)), "cuboid_sieve")
    return out.value


def cuboid_sieve_batch(t, ranges, stream=None) -> int:
    arr = _ranges_array(ranges)
    out = _P()
    _check(_lib.cuboid_sieve_batch(t, arr, len(ranges), _stream(stream), C.byref(out)), "cuboid_sieve_batch")
    return out.value


def cuboid_sieve_into(res, ranges, mode=MODE_PLAIN, stream=None, arr=None) -> None:
    """``arr`` may be a prebuilt ctypes array of cuboid_range (see ``ranges_array``)."""
    arr = arr if arr is not None else _ranges_array(ranges)
    _check(_lib.cuboid_sieve_into(res, arr, len(arr), mode, _stream(stream)), "cuboid_sieve_into")


def ranges_array(ranges):
    return _ranges_array(ranges)


def cuboid_sieve_device(res, ranges_dev_ptr: int, n: int, mode=MODE_PLAIN, stream=None) -> None:
    _check(_lib.cuboid_sieve_device(res, ranges_dev_ptr, n, mode, _stream(stream)), "cuboid_sieve_device")


def cuboid_result_download(res, stream=None) -> None:
    _check(_lib.cuboid_result_download(res, _stream(stream)), "cuboid_result_download")


def cuboid_result_wait(res) -> int:
    """Returns OK, EOVERFLOW, ERANGE, EVERIFY or ETIMEOUT; raises on other errors."""
    st = _lib.cuboid_result_wait(res)
    if st not in (OK, EOVERFLOW, ERANGE, EVERIFY, ETIMEOUT):
        _check(st, "cuboid_result_wait")
    return st


_GET_BUFS = threading.local()  # per thread: output buffers of cuboid_result_get, by n_primes


def _get_bufs(n_primes: int):
    cache = getattr(_GET_BUFS, "by_n", None)
    if cache is None:
        cache = _GET_BUFS.by_n = {}
    b = cache.get(n_primes)
    if b is None:
        npairs, ns, nr = _u64(), _u64(), _u64()
        counts = (_u64 * n_primes)()
        sp, rp = C.POINTER(_u64)(), C.POINTER(cuboid_root)()
        b = cache[n_primes] = (npairs, counts, ns, sp, nr, rp,
                               (C.byref(npairs), counts, C.byref(ns), C.byref(sp), C.byref(nr), C.byref(rp)))
    return b


def cuboid_result_get(res, range_idx: int, n_primes: int) -> dict:
    npairs, counts, ns, sp, nr, rp, args = _get_bufs(n_primes)
    _check(_lib.cuboid_result_get(res, range_idx, *args), "cuboid_result_get")
    surv = [(int(sp[i]) >> 32, int(sp[i]) & 0xFFFFFFFF) for i in range(ns.value)]
    roots = [(rp[i].p, rp[i].q, (int(rp[i].t_hi) << 64) | int(rp[i].t_lo)) for i in range(nr.value)]
    cuboids = [rt for rt, f in zip(roots, cuboid_theorem11_flags(roots)) if f] if roots else []
    return {"n_pairs": npairs.value, "counts": counts[:], "survivors": surv, "roots": roots,
            "cuboids": cuboids}


def cuboid_result_sieve_ms(res):
    """(milliseconds, launches) of the sieve kernels of the last timed run."""
    ms, n = C.c_float(), _u32()
    _check(_lib.cuboid_result_sieve_ms(res, C.byref(ms), C.byref(n)), "cuboid_result_sieve_ms")
    return ms.value, n.value


def cuboid_result_stats(res) -> dict:
    s = cuboid_stats()
    _check(_lib.cuboid_result_stats(res, C.byref(s)), "cuboid_result_stats")
    return {k: getattr(s, k) for k, _ in cuboid_stats._fields_}


def cuboid_result_free(res) -> int:
    return _lib.cuboid_result_free(res)


def cuboid_sieve_noalloc(t, ranges_dev_ptr: int, n: int, counts_dev_ptr: int, npairs_dev_ptr: int,
                         surv_dev_ptr: int, surv_range_dev_ptr: int, surv_cap: int, roots_dev_ptr: int,
                         root_range_dev_ptr: int, root_cap: int, totals_dev_ptr: int, stream=None) -> int:
    """The allocation-free sieve: every buffer is a device pointer owned by the caller.
    Returns the status code (ETOOLARGE for too many ranges) instead of raising."""
    return _lib.cuboid_sieve_noalloc(t, ranges_dev_ptr, n, counts_dev_ptr, npairs_dev_ptr, surv_dev_ptr,
                                     surv_range_dev_ptr, surv_cap, roots_dev_ptr, root_range_dev_ptr,
                                     root_cap, totals_dev_ptr, _stream(stream))


# ------------------------------------------------------------------ region search (section 5)

def _report(rep: cuboid_search_report) -> dict:
    return {k: getattr(rep, k) for k, _ in cuboid_search_report._fields_}


def cuboid_region_qmin(p: int) -> int:
    return int(_lib.cuboid_region_qmin(p))


def cuboid_region_scan(t, p_from: int, p_to: int, q_from: int = 0, stream=None,
                       surv_cap: int = 1 << 16, root_cap: int = 1 << 12):
    """Scan rows p_from..p_to of the region.  Returns (status, report dict, counts in caller
    order, survivor (p, q) list, root (p, q, t) list); status is OK or EOVERFLOW, others raise."""
    n = cuboid_tables_info(t)[0]
    counts = (_u64 * n)()
    surv = (_u64 * max(surv_cap, 1))()
    roots = (cuboid_root * max(root_cap, 1))()
    rep = cuboid_search_report()
    st = _lib.cuboid_region_scan(t, p_from, q_from, p_to, _stream(stream), counts, surv, surv_cap, roots,
                                 root_cap, C.byref(rep))
    if st not in (OK, EOVERFLOW):
        _check(st, "cuboid_region_scan")
    d = _report(rep)
    ns, nr = min(d["n_surv"], surv_cap), min(d["n_roots"], root_cap)
    sv = [(int(surv[i]) >> 32, int(surv[i]) & 0xFFFFFFFF) for i in range(ns)]
    rv = [(roots[i].p, roots[i].q, (int(roots[i].t_hi) << 64) | int(roots[i].t_lo)) for i in range(nr)]
    return st, d, list(counts), sv, rv


def cuboid_search_start(t, p: int, q: int) -> int:
    """Start the asynchronous search (raises CuboidError with the paper's codes 1..6)."""
    out = _P()
    _check(_lib.cuboid_search_start(t, p, q, C.byref(out)), "cuboid_search_start")
    return out.value


def cuboid_search_start_status(t, p: int, q: int):
    """As cuboid_search_start, returning (status, handle or None) instead of raising."""
    out = _P()
    st = _lib.cuboid_search_start(t, p, q, C.byref(out))
    return st, (out.value if st == OK else None)


def cuboid_search_current(s):
    """(first row of the batch being scanned, deepest prime needed within it)."""
    p, r = _u32(), _u32()
    _check(_lib.cuboid_search_current(s, C.byref(p), C.byref(r)), "cuboid_search_current")
    return p.value, r.value


def cuboid_search_stop(s, n_primes: int):
    """Stop and free the search; returns (status of the scan, report dict, counts)."""
    rep = cuboid_search_report()
    counts = (_u64 * n_primes)()
    st = _lib.cuboid_search_stop(s, C.byref(rep), counts)
    return st, _report(rep), list(counts)


def cuboid_search_report_write(rep: dict, path: str) -> None:
    """Append a report (dict from cuboid_search_stop / cuboid_region_scan) to a text file."""
    r = cuboid_search_report(**rep)
    _check(_lib.cuboid_search_report_write(C.byref(r), path.encode()), "cuboid_search_report_write")


def cuboid_theorem11_flags(roots) -> list[bool]:
    """Theorem 1.1 on (p, q, t) roots: True where t would give a perfect cuboid."""
    n = len(roots)
    arr = (cuboid_root * max(n, 1))()
    for i, (p, q, t) in enumerate(roots):
        arr[i] = cuboid_root(p, q, t & ((1 << 64) - 1), t >> 64)
    out = (C.c_uint8 * max(n, 1))()
    _check(_lib.cuboid_theorem11_flags(arr, n, out), "cuboid_theorem11_flags")
    return [bool(out[i]) for i in range(n)]


def cuboid_shard_range(rng, k: int, i: int):
    """Shard i of k of a range (dict or cuboid_range): (range dict or None if empty, points)."""
    r = rng if isinstance(rng, cuboid_range) else range_from_dict(rng)
    out = cuboid_range()
    pts = _u64()
    _check(_lib.cuboid_shard_range(C.byref(r), k, i, C.byref(out), C.byref(pts)), "cuboid_shard_range")
    if out.p_lo > out.p_hi or out.q_lo > out.q_hi:
        return None, 0
    return {"p_lo": out.p_lo, "p_hi": out.p_hi, "q_lo": out.q_lo, "q_hi": out.q_hi,
            "q_lt_p": bool(out.flags & Q_LT_P), "allow_diagonal": bool(out.flags & ALLOW_DIAGONAL),
            "flags": out.flags & (ROWS_P | ROWS_Q)}, pts.value


def cuboid_verify_pairs(ps, qs, stream=None, cap: int | None = None):
    n = len(ps)
    pa = (_u32 * n)(*ps)
    qa = (_u32 * n)(*qs)
    cap = cap if cap is not None else 5 * n + 5
    out = (cuboid_root * cap)()
    nr = _u64()
    _check(_lib.cuboid_verify_pairs(pa, qa, n, _stream(stream), out, cap, C.byref(nr)), "cuboid_verify_pairs")
    return [(out[i].p, out[i].q, (int(out[i].t_hi) << 64) | int(out[i].t_lo)) for i in range(nr.value)]


# ------------------------------------------------------------------ 64-bit ranges

WIDE_LIMIT = 1 << 40


def wide_range(d: dict) -> cuboid_range_wide:
    """A cuboid_range_wide from a range dict (p_lo, p_hi, q_lo, q_hi, q_lt_p,
    allow_diagonal, flags)."""
    fl = (Q_LT_P if d.get("q_lt_p") else 0) | (ALLOW_DIAGONAL if d.get("allow_diagonal") else 0) | d.get("flags", 0)
    return cuboid_range_wide(d["p_lo"], d["p_hi"], d["q_lo"], d["q_hi"], fl, d.get("reserved", 0))


def cuboid_wide_pieces(rng: dict):
    """The pieces of a 64-bit range: [(piece dict with relative bounds and flags, p base, q base)]."""
    r = wide_range(rng)
    n = _u32()
    st = _lib.cuboid_wide_pieces(C.byref(r), None, None, 0, C.byref(n))
    if st not in (OK, EOVERFLOW):
        _check(st, "cuboid_wide_pieces")
    cap = max(n.value, 1)
    pcs = (cuboid_range * cap)()
    bases = (_u64 * (2 * cap))()
    _check(_lib.cuboid_wide_pieces(C.byref(r), pcs, bases, cap, C.byref(n)), "cuboid_wide_pieces")
    return [({"p_lo": pcs[i].p_lo, "p_hi": pcs[i].p_hi, "q_lo": pcs[i].q_lo, "q_hi": pcs[i].q_hi,
              "flags": pcs[i].flags}, int(bases[2 * i]), int(bases[2 * i + 1])) for i in range(n.value)]


def cuboid_sieve_wide(t, ranges, stream=None) -> int:
    """Sieve 64-bit ranges (dicts); returns the result handle (wait, then cuboid_result_get_wide)."""
    arr = (cuboid_range_wide * len(ranges))(*[wide_range(d) for d in ranges])
    out = _P()
    _check(_lib.cuboid_sieve_wide(t, arr, len(ranges), _stream(stream), C.byref(out)), "cuboid_sieve_wide")
    return out.value


def cuboid_result_get_wide(res, range_idx: int, n_primes: int) -> dict:
    npairs, ns, nr = _u64(), _u64(), _u64()
    counts = (_u64 * n_primes)()
    sp, rp = C.POINTER(_u64)(), C.POINTER(cuboid_root_wide)()
    _check(_lib.cuboid_result_get_wide(res, range_idx, C.byref(npairs), counts, C.byref(ns), C.byref(sp),
                                       C.byref(nr), C.byref(rp)), "cuboid_result_get_wide")
    surv = [(int(sp[2 * i]), int(sp[2 * i + 1])) for i in range(ns.value)]
    roots = [(int(rp[i].p), int(rp[i].q), (int(rp[i].t_hi) << 64) | int(rp[i].t_lo)) for i in range(nr.value)]
    cuboids = [rt for rt, f in zip(roots, cuboid_theorem11_flags_wide(roots)) if f] if roots else []
    return {"n_pairs": npairs.value, "counts": counts[:], "survivors": surv, "roots": roots,
            "cuboids": cuboids}


def cuboid_verify_pairs_wide(ps, qs, stream=None, cap: int | None = None):
    n = len(ps)
    pa = (_u64 * max(n, 1))(*ps)
    qa = (_u64 * max(n, 1))(*qs)
    cap = cap if cap is not None else 5 * n + 5
    out = (cuboid_root_wide * cap)()
    nr = _u64()
    _check(_lib.cuboid_verify_pairs_wide(pa, qa, n, _stream(stream), out, cap, C.byref(nr)),
           "cuboid_verify_pairs_wide")
    return [(int(out[i].p), int(out[i].q), (int(out[i].t_hi) << 64) | int(out[i].t_lo)) for i in range(nr.value)]


def cuboid_region_scan_wide(t, p_from: int, p_to: int, q_from: int = 0, stream=None,
                            surv_cap: int = 1 << 16, root_cap: int = 1 << 12):
    """Scan rows p_from..p_to (< 2^32) of the region with 64-bit q.  Returns (status, report
    dict, counts in caller order, survivor (p, q) list, root (p, q, t) list); status is OK
    or EOVERFLOW, others raise."""
    n = cuboid_tables_info(t)[0]
    counts = (_u64 * n)()
    surv = (_u64 * max(2 * surv_cap, 2))()
    roots = (cuboid_root_wide * max(root_cap, 1))()
    rep = cuboid_region_report_wide()
    st = _lib.cuboid_region_scan_wide(t, p_from, q_from, p_to, _stream(stream), counts, surv, surv_cap, roots,
                                      root_cap, C.byref(rep))
    if st not in (OK, EOVERFLOW):
        _check(st, "cuboid_region_scan_wide")
    d = {k: getattr(rep, k) for k, _ in cuboid_region_report_wide._fields_}
    ns, nr = min(d["n_surv"], surv_cap), min(d["n_roots"], root_cap)
    sv = [(int(surv[2 * i]), int(surv[2 * i + 1])) for i in range(ns)]
    rv = [(int(roots[i].p), int(roots[i].q), (int(roots[i].t_hi) << 64) | int(roots[i].t_lo)) for i in range(nr)]
    return st, d, list(counts), sv, rv


def cuboid_theorem11_flags_wide(roots) -> list[bool]:
    """Theorem 1.1 on (p, q, t) roots with p, q < 2^40."""
    n = len(roots)
    arr = (cuboid_root_wide * max(n, 1))()
    for i, (p, q, t) in enumerate(roots):
        arr[i] = cuboid_root_wide(p, q, t & ((1 << 64) - 1), t >> 64)
    out = (C.c_uint8 * max(n, 1))()
    _check(_lib.cuboid_theorem11_flags_wide(arr, n, out), "cuboid_theorem11_flags_wide")
    return [bool(out[i]) for i in range(n)]


# ------------------------------------------------------------------ serving

def cuboid_server_create(t, mem_budget: int = 0, max_slots: int = 0) -> int:
    out = _P()
    _check(_lib.cuboid_server_create(t, mem_budget, max_slots, C.byref(out)), "cuboid_server_create")
    return out.value


def cuboid_server_submit(s, rng):
    """Returns the ticket, or None when admission is refused (EBUSY)."""
    r = rng if isinstance(rng, cuboid_range) else range_from_dict(rng)
    tk = _u64()
    st = _lib.cuboid_server_submit(s, C.byref(r), C.byref(tk))
    if st == EBUSY:
        return None
    _check(st, "cuboid_server_submit")
    return tk.value


def cuboid_server_poll(s, ticket: int):
    """Returns a result handle (one range), or None while the query runs (EAGAIN)."""
    out = _P()
    st = _lib.cuboid_server_poll(s, ticket, C.byref(out))
    if st == EAGAIN:
        return None
    _check(st, "cuboid_server_poll")
    return out.value


def cuboid_server_stats(s) -> dict:
    v = [_u64() for _ in range(6)]
    _check(_lib.cuboid_server_stats(s, *[C.byref(x) for x in v]), "cuboid_server_stats")
    return dict(zip(("in_flight", "admitted", "refused", "finished", "batches", "retried"), [x.value for x in v]))


def cuboid_server_replay(s, queries, arrival_s, timeout_ms: int = 600000) -> dict:
    """Submit queries[i] at arrival_s[i] seconds (native loop), wait for all; returns
    tickets, per-query latency (s), pairs and status, the wall time and refused retries.
    The results stay available to cuboid_server_poll."""
    n = len(queries)
    arr = _ranges_array(queries) if n else (cuboid_range * 1)()
    at = (C.c_double * max(n, 1))(*[float(x) for x in arrival_s])
    tk = (_u64 * max(n, 1))()
    lat = (C.c_double * max(n, 1))()
    npairs = (_u64 * max(n, 1))()
    st = (C.c_int32 * max(n, 1))()
    wall, refused = C.c_double(), _u64()
    _check(_lib.cuboid_server_replay(s, arr, at, n, timeout_ms, tk, lat, npairs, st, C.byref(wall),
                                     C.byref(refused)), "cuboid_server_replay")
    return {"tickets": list(tk[:n]), "latency_s": list(lat[:n]), "npairs": list(npairs[:n]),
            "status": list(st[:n]), "wall_s": wall.value, "refused": refused.value}


def cuboid_server_destroy(s, timeout_ms: int = 60000) -> int:
    return _lib.cuboid_server_destroy(s, timeout_ms)


# ------------------------------------------------------------------ measurement

def cuboid_probe_int_issue(kind, blocks, threads, iters, sink_dev_ptr: int, stream=None) -> None:
    _check(_lib.cuboid_probe_int_issue(kind, blocks, threads, iters, sink_dev_ptr, _stream(stream)),
           "cuboid_probe_int_issue")


def cuboid_probe_mod_min(mods, stream=None) -> list[int]:
    """Mismatches of the sieve's residue routine against % over every 32-bit n, per modulus."""
    n = len(mods)
    arr = (_u32 * n)(*[int(x) for x in mods])
    out = (_u64 * n)()
    _check(_lib.cuboid_probe_mod_min(arr, n, out, _stream(stream)), "cuboid_probe_mod_min")
    return list(out)


def cuboid_probe_modarith(op: int, j: int, a=(), b=(), device: bool = False) -> list[int]:
    """The root test's modular arithmetic (see cuboid.h): op 0 a b mod m_j, op 1 a mod m_j,
    op 2 Garner sign of residue vectors of length j (a flattened), op 3 the moduli."""
    n = 14 if op == 3 else (len(a) // j if op == 2 else len(a))
    aa = (_u64 * max(1, len(a)))(*[int(x) for x in a])
    bb = (_u64 * max(1, len(b)))(*[int(x) for x in b])
    out = (_u64 * max(1, n))()
    _check(_lib.cuboid_probe_modarith(op, j, aa, bb, n, out, 1 if device else 0), "cuboid_probe_modarith")
    return list(out[:n])


def cuboid_device_sms() -> int:
    v = _u32()
    _check(_lib.cuboid_device_sms(C.byref(v)), "cuboid_device_sms")
    return v.value


def cuboid_version() -> str:
    return _lib.cuboid_version().decode()
