"""The paper's search loop in C with OpenMP (``paper_loop.c``) -- TEST INFRASTRUCTURE AND
CPU BASELINE ONLY.

The nested loop of section 5 over tables in the byte layout of Eq. 2.6, one row per
OpenMP work item: the timed CPU baseline of the benchmark, parity-checked against the
Python oracle in the tests.  Only ``tests/`` and the CPU legs of ``bench.py`` load it.
The shared object is compiled in place with gcc (``build()``; ``__graft_entry__.build()``
compiles it too) and is rebuilt when the source is newer.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "paper_loop.c")
LIB = os.path.join(HERE, f"libpaperloop_{platform.machine()}.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile paper_loop.c with gcc -O2 -fopenmp (without OpenMP if the compiler has none)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", SRC, "-o", tmp]
    p = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if p.returncode:
        p = subprocess.run(base, capture_output=True, text=True)
    if p.returncode:
        raise RuntimeError("gcc failed for paper_loop.c:\n" + p.stderr)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.pl_tables_build.restype = C.c_void_p
        lib.pl_tables_build.argtypes = [C.POINTER(C.c_uint32), C.c_uint32]
        lib.pl_tables_free.argtypes = [C.c_void_p]
        lib.pl_table_bytes.restype = C.POINTER(C.c_uint8)
        lib.pl_table_bytes.argtypes = [C.c_void_p, C.c_uint32]
        lib.pl_sieve.restype = C.c_int
        lib.pl_sieve.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), C.c_uint32, C.c_uint32, C.c_uint32,
                                 C.c_uint32, C.c_uint32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                 C.POINTER(C.c_uint64), C.c_uint64, C.POINTER(C.c_uint64), C.c_int]
        lib.pl_sieve_many.restype = C.c_int
        lib.pl_sieve_many.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.c_uint32,
                                      C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                      C.POINTER(C.c_uint32), C.c_uint64, C.POINTER(C.c_uint64), C.c_int]
        lib.pl_max_threads.restype = C.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    """Threads the loop uses by default (OpenMP's default: the host's cores)."""
    return int(_load().pl_max_threads())


class PaperLoop:
    """Packed tables of a prime list and the section 5 loop over them."""

    def __init__(self, primes):
        lib = _load()
        self.primes = [int(r) for r in primes]
        arr = (C.c_uint32 * len(self.primes))(*self.primes)
        self._h = lib.pl_tables_build(arr, len(self.primes))
        if not self._h:
            raise ValueError("pl_tables_build refused the prime list")

    def close(self):
        if self._h:
            _load().pl_tables_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def table_bytes(self, i: int) -> bytes:
        """The Eq. 2.6 bytes of the i-th prime's table."""
        r = self.primes[i]
        ptr = _load().pl_table_bytes(self._h, i)
        return bytes(ptr[:(r * r + 7) // 8])

    def sieve(self, order, rng: dict, threads: int = 0, surv_cap: int = 1 << 20):
        """(n_pairs, counts in list order, sorted survivors) of one range; ``order`` is the
        effective order (indices into the prime list).  Ranges with the diagonal are not
        supported."""
        if rng.get("allow_diagonal"):
            raise ValueError("the paper loop sieves p != q only")
        n = len(self.primes)
        order_a = (C.c_uint32 * n)(*order)
        counts = (C.c_uint64 * n)()
        n_pairs, n_surv = C.c_uint64(0), C.c_uint64(0)
        surv = (C.c_uint64 * max(1, surv_cap))()
        st = _load().pl_sieve(self._h, order_a, rng["p_lo"], rng["p_hi"], rng["q_lo"], rng["q_hi"],
                              1 if rng.get("q_lt_p") else 0, counts, C.byref(n_pairs), surv, surv_cap,
                              C.byref(n_surv), int(threads))
        if st:
            raise RuntimeError(f"pl_sieve returned {st}")
        k = min(n_surv.value, surv_cap)
        s = sorted((int(x) >> 32, int(x) & 0xFFFFFFFF) for x in surv[:k])
        return n_pairs.value, [int(c) for c in counts], s

    def sieve_many(self, order, ranges, threads: int = 0, surv_cap: int = 1 << 20):
        """[(n_pairs, counts in list order, sorted survivors)] of many ranges in one call;
        the rows of all ranges are the OpenMP work items."""
        n, k = len(self.primes), len(ranges)
        flat = []
        for rng in ranges:
            if rng.get("allow_diagonal"):
                raise ValueError("the paper loop sieves p != q only")
            flat += [rng["p_lo"], rng["p_hi"], rng["q_lo"], rng["q_hi"], 1 if rng.get("q_lt_p") else 0]
        arr = (C.c_uint32 * len(flat))(*flat)
        order_a = (C.c_uint32 * n)(*order)
        counts = (C.c_uint64 * (n * k))()
        pairs = (C.c_uint64 * k)()
        n_surv = C.c_uint64(0)
        surv = (C.c_uint64 * max(1, surv_cap))()
        surv_rng = (C.c_uint32 * max(1, surv_cap))()
        st = _load().pl_sieve_many(self._h, order_a, arr, k, counts, pairs, surv, surv_rng, surv_cap,
                                   C.byref(n_surv), int(threads))
        if st:
            raise RuntimeError(f"pl_sieve_many returned {st}")
        m = min(n_surv.value, surv_cap)
        per = [[] for _ in range(k)]
        for i in range(m):
            x = int(surv[i])
            per[surv_rng[i]].append((x >> 32, x & 0xFFFFFFFF))
        return [(int(pairs[j]), [int(c) for c in counts[j * n:(j + 1) * n]], sorted(per[j])) for j in range(k)]
