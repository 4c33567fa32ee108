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
