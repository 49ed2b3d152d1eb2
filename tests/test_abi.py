"""The C ABI library loads without a GPU and exports every function that
include/stmg.h declares; host-side argument checks (no device calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stmg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(st_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1411_0519_gb300 import stmg
    if not os.path.exists(stmg.library_path()):
        from paper_1411_0519_gb300 import build
        build.build()
    return stmg.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["st_setup", "st_vcycle", "st_solve", "st_adjoint_solve", "st_residual", "st_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_match_header():
    from paper_1411_0519_gb300 import stmg
    assert sorted(stmg.EXPORTS) == declared_functions()


def test_setup_rejects_bad_arguments_before_touching_the_device(lib):
    from paper_1411_0519_gb300 import stmg
    opt = stmg.StOptions()
    lib.st_default_options(ctypes.byref(opt))
    assert opt.nu1 == 2 and opt.nu2 == 2 and opt.omega == 0.5 and opt.coarsest_steps == 1
    h = ctypes.c_void_p()
    bad = [
        (stmg.StMesh(2, 254), 1, 16, 1.0),   # n not 2^k - 1
        (stmg.StMesh(4, 7), 1, 16, 1.0),     # dim > 3
        (stmg.StMesh(1, 2047), 1, 16, 1.0),  # n > 1023
        (stmg.StMesh(2, 7), 1, 12, 1.0),     # N not a power of two
        (stmg.StMesh(2, 7), stmg.ST_MAX_PT + 1, 16, 1.0),   # p_t too large
        (stmg.StMesh(2, 7), 1, 16, -1.0),    # T <= 0
    ]
    for mesh, p, N, T in bad:
        rc = lib.st_setup(ctypes.byref(mesh), p, N, T, ctypes.byref(opt), None, ctypes.byref(h))
        assert rc == stmg.ST_EINVAL
        assert not h.value
    assert lib.st_setup(None, 1, 16, 1.0, None, None, ctypes.byref(h)) == stmg.ST_EINVAL
    assert lib.st_num_levels(None) == 0 and lib.st_ndof(None) == 0
    assert lib.st_residual(None, None, None, None, None) == stmg.ST_EINVAL
