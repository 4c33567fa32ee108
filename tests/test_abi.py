"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/*.h
declares (CPU only: no compute calls)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:int|uint32_t|const char\*|void)\s+(cuboid_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    return __graft_entry__._builder().build()


def test_header_declares_functions():
    names = _declared()
    assert {"cuboid_tables_build", "cuboid_sieve", "cuboid_sieve_batch", "cuboid_result_wait",
            "cuboid_server_submit"} <= names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert _declared() <= exported


def test_binding_covers_the_abi(lib_path):
    import paper_1601_00636_gb300 as cb
    assert set(cb.EXPORTED) == _declared()
    assert cb.cuboid_version().startswith("libcuboid")


def test_null_handles_are_rejected(lib_path):
    """Misuse is signalled by status codes, never by a crash (host-only paths)."""
    import paper_1601_00636_gb300 as cb
    lib = cb._lib
    assert lib.cuboid_tables_free(None) == cb.ENOTABLES
    assert lib.cuboid_tables_order(None, None) == cb.ENOTABLES
    assert lib.cuboid_result_free(None) == cb.EINVAL
    assert lib.cuboid_result_wait(None) == cb.EINVAL
    assert lib.cuboid_sieve(None, 1, 2, 1, 2, 0, None, None) == cb.ENOTABLES
    assert lib.cuboid_server_destroy(None, 0) == cb.EINVAL
    assert lib.cuboid_probe_int_issue(5, 1, 32, 1, None, None) == cb.EINVAL
    assert lib.cuboid_probe_int_issue(9, 1, 32, 1, 16, None) == cb.EINVAL
    assert lib.cuboid_sieve_wide(None, None, 0, None, None) == cb.ENOTABLES
    assert lib.cuboid_result_get_wide(None, 0, None, None, None, None, None, None) == cb.EINVAL
    assert lib.cuboid_region_scan_wide(None, 1, 0, 2, None, None, None, 0, None, 0, None) == cb.ENOTABLES
    assert lib.cuboid_verify_pairs_wide(None, None, 0, None, None, 0, None) == cb.EINVAL
    assert lib.cuboid_wide_pieces(None, None, None, 0, None) == cb.EINVAL


_STRUCTS = {
    "cuboid_range": ["p_lo", "p_hi", "q_lo", "q_hi", "flags", "reserved"],
    "cuboid_root": ["p", "q", "t_lo", "t_hi"],
    "cuboid_tuning": ["block_threads", "ctas_per_sm", "smem_primes", "tiles_per_warp", "hot_primes", "row_lanes"],
    "cuboid_stats": ["words", "word_steps", "warp_steps", "tiles"],
    "cuboid_search_report": ["p", "q", "r_max", "depth", "pairs", "n_surv", "n_roots"],
    "cuboid_range_wide": ["p_lo", "p_hi", "q_lo", "q_hi", "flags", "reserved"],
    "cuboid_root_wide": ["p", "q", "t_lo", "t_hi"],
    "cuboid_region_report_wide": ["p", "q", "r_max", "depth", "pairs", "n_surv", "n_roots"],
}


def test_struct_layouts_match_header(tmp_path):
    """Every struct of include/cuboid.h has the same size and field offsets in C (gcc on
    the header) as in the ctypes binding."""
    import paper_1601_00636_gb300 as cb
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cuboid.h"', "int main(void) {"]
    for name, fields in _STRUCTS.items():
        offs = " ".join("%zu" for _ in fields)
        args = ", ".join(f"offsetof({name}, {f})" for f in fields)
        lines.append(f'  printf("{name} %zu {offs}\\n", sizeof({name}), {args});')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for ln in out.splitlines():
        name, size, *offs = ln.split()
        st = getattr(cb, name)
        assert ctypes.sizeof(st) == int(size), name
        assert [getattr(st, f).offset for f in _STRUCTS[name]] == [int(o) for o in offs], name
