"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/*.h declares; host-side argument checks that need no GPU."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

import paper_2608_09647_gb300 as cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    return cg.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cg_create", "cg_spmv", "cg_solve", "cg_destroy", "cg_last_error"):
        assert required in names
    assert names == set(cg.EXPORTS) | (names - set(cg.EXPORTS))


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", cg.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for name in declared_functions():
        assert hasattr(lib, name)


def test_binding_covers_every_export():
    assert declared_functions() == set(cg.EXPORTS)


def test_status_strings(lib):
    assert cg.status_string(0) == "CG_OK"
    assert cg.status_string(-4) == "CG_ERR_TIMEOUT"
    assert cg.status_string(42) == "CG_UNKNOWN_STATUS"


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    out = ctypes.c_void_p(123)
    assert lib.cg_create(-1, None, None, None, ctypes.byref(out)) == cg.CG_ERR_INVALID
    assert out.value is None
    assert b"n out of range" in lib.cg_last_error(None)
    assert lib.cg_create(5, None, None, None, ctypes.byref(out)) == cg.CG_ERR_INVALID
    assert b"rowptr" in lib.cg_last_error(None)
    assert lib.cg_create(5, None, None, None, None) == cg.CG_ERR_INVALID


def test_null_handle_calls_are_rejected(lib):
    assert lib.cg_spmv(None, None, None) == cg.CG_ERR_INVALID
    assert lib.cg_solve(None, None, None, 1e-8, 10, 0, 0, None, None) == cg.CG_ERR_INVALID
    assert lib.cg_set_option(None, 0, 1.0) == cg.CG_ERR_INVALID
    lib.cg_destroy(None)
