"""Host logic of the Python binding, without a GPU: argument marshalling
refuses anything but contiguous FP64 device tensors of the right size, and
the options map onto st_options as st_default_options documents them."""
import ctypes

import pytest
import torch


@pytest.fixture(scope="module")
def stmg():
    import os
    from paper_1411_0519_gb300 import stmg as m
    if not os.path.exists(m.library_path()):
        from paper_1411_0519_gb300 import build
        build.build()
    m.load_library()
    return m


def test_marshalling_refuses_host_and_wrong_tensors(stmg):
    assert stmg._ptr(None) is None
    with pytest.raises(TypeError):
        stmg._ptr(torch.zeros(4, dtype=torch.float64), 4, "f")          # host memory
    with pytest.raises(TypeError):
        stmg._ptr(torch.zeros(4, dtype=torch.float32), 4, "f")          # wrong dtype (and host)
    with pytest.raises(TypeError):
        stmg._ptr([0.0] * 4, 4, "f")                                     # not a tensor
    with pytest.raises(TypeError):
        stmg._ptr(torch.zeros(4, 4, dtype=torch.float64).t(), 16, "f")  # not contiguous


def test_options_follow_the_documented_defaults(stmg):
    d = stmg.StOptions()
    stmg.lib().st_default_options(ctypes.byref(d))
    o = stmg.make_options()
    for field, _ in stmg.StOptions._fields_:
        assert getattr(o, field) == getattr(d, field), field
    o = stmg.make_options(precision="mixed", coarsening="semi", smoother="vcycle", gamma=2, coarsest_steps=4)
    assert (o.precision, o.coarsening, o.smoother, o.gamma, o.coarsest_steps) == (
        stmg.ST_MIXED, stmg.ST_SEMI, stmg.ST_SMOOTH_VCYCLE, 2, 4)
    with pytest.raises(KeyError):
        stmg.make_options(precision="fp16")
    with pytest.raises(KeyError):
        stmg.make_options(smoother="gauss-seidel")


def test_kernel_classes_match_the_header(stmg):
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "stmg.h")).read()
    idx = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define ST_K_([A-Z]+)\s+(\d+)", hdr)}
    assert idx["COUNT"] == len(stmg.KERNEL_CLASSES)
    names = {"RESIDUAL": "residual", "DST": "dst", "SMOOTH": "smooth", "RESTRICT": "restrict",
             "PROLONG": "prolong", "NORM": "norm", "VECTOR": "vector", "RHS": "rhs", "SPACEMG": "space_mg"}
    for k, v in names.items():
        assert stmg.KERNEL_CLASSES[idx[k]] == v, k
