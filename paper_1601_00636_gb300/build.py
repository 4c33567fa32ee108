"""Build libcuboid.so in-tree for sm_103a (nvcc, one -gencode, sources compiled in parallel)."""
from __future__ import annotations

import os
import platform
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build", platform.machine())
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libcuboid.so")
LIB_DEBUG = os.path.join(PKG, "libcuboid_debug.so")
SOURCES = ["tables.cu", "plan.cu", "sieve.cu", "verify.cu", "runtime.cu", "server.cu", "noalloc.cu", "tune.cu", "region.cu", "tablefile.cu", "theorem.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found (set NVCC)")
    return cand


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                   "-I", CSRC, "--expt-relaxed-constexpr", *extra]


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(CSRC, "cuboid_internal.cuh"), os.path.join(INCLUDE, "cuboid.h"),
            os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def _arch_of(path: str) -> str:
    """Machine of an ELF shared object (x86_64 / aarch64), from its header."""
    try:
        with open(path, "rb") as f:
            head = f.read(20)
    except OSError:
        return ""
    mach = int.from_bytes(head[18:20], "little")
    return {62: "x86_64", 183: "aarch64"}.get(mach, str(mach))


def build(verbose: bool = False, ptxas_verbose: bool = False, force: bool = False, debug: bool = False) -> str:
    """Compile every source and link libcuboid.so (debug: libcuboid_debug.so, compiled with
    CUBOID_DEBUG, whose kernels check their table, mask, factor and queue indices and
    report a failed check as CUBOID_EINDEX); returns its path."""
    build_dir = BUILD + ("-debug" if debug else "")
    lib = LIB_DEBUG if debug else LIB
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        if force or ptxas_verbose or _stale(o, s):
            extra = ["-Xptxas", "-v"] if ptxas_verbose else []
            if debug:
                extra.append("-DCUBOID_DEBUG")
            jobs.append([cc, *_flags(extra), "-c", s, "-o", o])

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, p

    relink = bool(jobs) or not os.path.exists(lib) or _arch_of(lib) != platform.machine()
    with ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for cmd, p in ex.map(run, jobs):
            if verbose or ptxas_verbose or p.returncode:
                sys.stderr.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
            if p.returncode:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    if relink:
        objs = [os.path.join(build_dir, s.replace(".cu", ".o")) for s in SOURCES]
        tmp = lib + ".tmp"
        cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
               "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or p.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
        if p.returncode:
            raise RuntimeError("link failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, ptxas_verbose="--ptxas" in sys.argv, force="-f" in sys.argv,
                debug="--debug" in sys.argv))
