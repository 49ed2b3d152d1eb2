"""The C ABI library loads without a GPU and exports every function that
include/stmg.h and include/stmg_mesh.h declare; host-side argument checks
(no device calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stmg.h")
MESH_HEADER = os.path.join(ROOT, "include", "stmg_mesh.h")


def declared_functions(header=HEADER, prefix="st_"):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(" + prefix + r"[a-z0-9_]+)\s*\(", text)))


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
    names = declared_functions() + declared_functions(MESH_HEADER, "stm_")
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert "stm_setup" in names and "stm_solve" in names


def test_binding_lists_match_header():
    from paper_1411_0519_gb300 import stmg
    assert sorted(stmg.EXPORTS) == declared_functions()
    assert sorted(stmg.MESH_EXPORTS) == declared_functions(MESH_HEADER, "stm_")


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


def test_mesh_setup_rejects_bad_arguments_before_touching_the_device(lib):
    """stm_setup checks the mesh, the discretisation and the options on the host."""
    import numpy as np
    from paper_1411_0519_gb300 import stmg
    verts = np.array([[0, 0], [1, 0], [1, 1], [0, 1], [0.5, 0.5]], dtype=np.float64)
    cells = np.array([[0, 1, 4], [1, 2, 4], [2, 3, 4], [3, 0, 4]], dtype=np.int32)

    def mesh(v, c, dim=2):
        return stmg.SimplexMesh(dim, v.shape[0], v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), c.shape[0],
                                c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    opt = stmg.StOptions()
    lib.st_default_options(ctypes.byref(opt))
    opt.smoother = stmg.ST_SMOOTH_VCYCLE
    h = ctypes.c_void_p()
    good = mesh(verts, cells)
    bad_cells = cells.copy()
    bad_cells[0, 0] = 7
    outside = verts.copy()
    outside[0, 0] = -0.5
    cases = [
        (mesh(verts, bad_cells), 1, 1, 16, 1.0, opt),       # vertex index out of range
        (mesh(outside, cells), 1, 1, 16, 1.0, opt),         # vertex outside the unit square
        (mesh(verts, cells, dim=4), 1, 1, 16, 1.0, opt),    # dim
        (good, 1, 4, 16, 1.0, opt),                         # p_t > 3
        (good, 1, 1, 12, 1.0, opt),                         # N not a power of two
        (good, 1, 1, 16, 0.0, opt),                         # T <= 0
        (good, -1, 1, 16, 1.0, opt),                        # refinements
    ]
    for m, ref, p, N, T, o in cases:
        assert lib.stm_setup(ctypes.byref(m), ref, p, N, T, ctypes.byref(o), None, ctypes.byref(h)) == stmg.ST_EINVAL
        assert not h.value
    for field, val in [("smoother", stmg.ST_SMOOTH_EXACT), ("precision", 7), ("coarsest_steps", 2)]:
        o = stmg.StOptions()
        ctypes.pointer(o)[0] = opt
        setattr(o, field, val)
        assert lib.stm_setup(ctypes.byref(good), 1, 1, 16, 1.0, ctypes.byref(o), None, ctypes.byref(h)) == \
            stmg.ST_EINVAL
    assert lib.stm_setup(None, 1, 1, 16, 1.0, None, None, ctypes.byref(h)) == stmg.ST_EINVAL
    assert lib.stm_num_levels(None) == 0 and lib.stm_ndof(None) == 0
    assert lib.stm_residual(None, None, None, None, None) == stmg.ST_EINVAL
