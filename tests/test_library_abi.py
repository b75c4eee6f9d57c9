"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every function that include/*.h declares (no compute calls: no GPU here)."""
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(lu_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2202_13995_gb300 import build as B
    B.build()
    from paper_2202_13995_gb300 import lu
    return lu.load()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for must in ("lu_create", "lu_destroy", "lu_factor", "lu_solve", "lu_refine", "lu_fact_free"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2202_13995_gb300 import lu
    out = subprocess.run(["nm", "-D", "--defined-only", lu.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)
    assert set(lu.EXPORTED) <= exported


def test_binding_knows_every_declared_function():
    from paper_2202_13995_gb300 import lu
    assert set(declared_functions()) <= set(lu.EXPORTED) | {n for n in declared_functions() if n.startswith(
        ("lu_batched", "lu_server", "lu_solve_batched"))}


def test_build_tag_and_strerror(lib):
    assert b"sm_103a" in lib.lu_build_tag()
    assert lib.lu_strerror(0) == b"ok"
    assert b"invalid" in lib.lu_strerror(-3)


def test_argument_errors_without_gpu(lib):
    import ctypes as C
    # NULL context / bad arguments are rejected before any CUDA call
    assert lib.lu_factor(None, 4, None, 4, 0, 0, C.byref(C.c_void_p()), None) == -1
    assert lib.lu_solve(None, 1, None, 1) == -1
    assert lib.lu_refine(None, None, 1, None, 1, None, 1, 1, 16.0, 10, None, None) == -1


def test_sm103a_cubin_only():
    # the build targets exactly one architecture
    from paper_2202_13995_gb300 import build as B
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
