"""The library's coarsening plan (st_plan: the hierarchy st_setup builds,
computed on the host without a device) against the oracle's hierarchy rule
(Section 2; Section 4 and the Remark on the critical parameter) and the mu*
values the paper prints."""
import os

import pytest

from oracle import hierarchy
from tests.test_oracle_dg import read_mu_star


@pytest.fixture(scope="module")
def stmg():
    from paper_1411_0519_gb300 import stmg as m
    if not os.path.exists(m.library_path()):
        from paper_1411_0519_gb300 import build
        build.build()
    m.load_library()
    return m


CASES = [
    # (d, n, p_t, N, T, options)
    (2, 255, 1, 1024, 1.0, {}),                                  # heat2d_255: full levels, then semi
    (3, 63, 2, 512, 1.0, {}),                                    # heat3d_63
    (1, 63, 1, 64, 1.0, {}),                                     # heat1d_63
    (2, 127, 45, 64, 64.0, {}),                                  # Example 2 protocol at p_t = 45
    (2, 15, 1, 16, 1.0, {"coarsening": "semi"}),
    (2, 15, 1, 16, 1.0, {"coarsening": "full"}),
    (2, 15, 1, 16, 1.0, {"coarsest_steps": 4}),
    (1, 1023, 0, 256, 1.0, {}),
] + [(2, 511, 1, 2048, mu / 128.0, {}) for mu in (1.0 / 16, 0.25, 1.0, 16.0)]   # heat2d_511 mu sweep


@pytest.mark.parametrize("d,n,p,N,T,opts", CASES)
def test_plan_matches_oracle_hierarchy(stmg, d, n, p, N, T, opts):
    levels, ms = stmg.plan(d, n, p, N, T, **opts)
    ref = hierarchy.build_levels(d, n, p, N, T, coarsening=opts.get("coarsening", "auto"),
                                 coarsest_steps=opts.get("coarsest_steps", 1))
    assert len(levels) == len(ref)
    assert abs(ms - hierarchy.mu_star(p)) <= 1e-12 * ms
    nl = len(levels)
    for L, lv in enumerate(levels):          # library: coarsest first; oracle: finest first
        r = ref[nl - 1 - L]
        assert (lv["N"], lv["n"]) == (r["N"], r["n"])
        assert abs(lv["mu"] - r["mu"]) <= 1e-12 * r["mu"]
        # full: how this level was obtained from the next finer one (-1 on the finest)
        assert lv["full"] == (-1 if L == nl - 1 else int(ref[nl - 2 - L]["full"]))


def test_plan_of_the_benchmark_workload(stmg):
    """heat2d_255: mu_fine = 64 >= mu*, so space and time are coarsened together
    until the spatial grid has one node; then time only, down to one step."""
    levels, _ = stmg.plan(2, 255, 1, 1024, 1.0)
    fulls = [lv["full"] for lv in levels[::-1]][1:]   # finest -> coarsest, skip the finest's -1
    ns = [lv["n"] for lv in levels[::-1]]
    assert ns[:8] == [255, 127, 63, 31, 15, 7, 3, 1]
    assert fulls == [1] * 7 + [0] * (len(fulls) - 7)
    assert levels[0]["N"] == 1 and levels[-1]["N"] == 1024


def test_mu_star_of_the_plan_matches_the_printed_values(stmg, golden_dir):
    printed = read_mu_star(golden_dir)
    for p in range(4):
        _, ms = stmg.plan(1, 7, p, 8, 1.0)
        assert abs(ms - printed[str(p)]) < 1e-9, p
    _, ms = stmg.plan(1, 7, 45, 8, 1.0)
    assert abs(ms - printed["inf"]) < 1e-9    # p_t = 45 is at the limit p_t -> infinity to 10 digits


@pytest.mark.parametrize("args,opts", [
    ((2, 254, 1, 16, 1.0), {}), ((4, 7, 1, 16, 1.0), {}), ((2, 7, 1, 12, 1.0), {}), ((2, 2047, 1, 16, 1.0), {}),
    ((2, 7, 48, 16, 1.0), {}), ((2, 7, 1, 16, -1.0), {}), ((2, 7, 1, 16, 1.0), {"coarsest_steps": 32}),
    ((1, 7, 1, 65536, 1.0), {}),
    ((2, 7, 1, 16, 1.0), {"gamma": 3}), ((2, 7, 4, 16, 1.0), {"smoother": "vcycle"}),
    ((2, 511, 1, 16, 1.0), {"transform": "tensor"}), ((2, 31, 1, 16, 1.0), {"transform": "tensor"}),
])
def test_plan_rejects_what_setup_rejects(stmg, args, opts):
    with pytest.raises(stmg.StmgError) as e:
        stmg.plan(*args, **opts)
    assert e.value.code == stmg.ST_EINVAL


def test_plan_checks_the_array_size(stmg):
    import ctypes
    lib = stmg.lib()
    mesh = stmg.StMesh(2, 255)
    opt = stmg.make_options()
    nlev = ctypes.c_int()
    Ns = (ctypes.c_int * 4)()
    rc = lib.st_plan(ctypes.byref(mesh), 1, 1024, 1.0, ctypes.byref(opt), 4, Ns, None, None, None,
                     ctypes.byref(nlev), None)
    assert rc == stmg.ST_EINVAL and nlev.value == 11


def test_transform_option_values(stmg):
    """auto and fft at every length, tensor for 64 <= n + 1 <= 256; other values are rejected."""
    for n in (31, 63, 255, 511):
        stmg.plan(2, n, 1, 16, 1.0, transform="auto")
        stmg.plan(2, n, 1, 16, 1.0, transform="fft")
    for n in (63, 127, 255):
        stmg.plan(2, n, 1, 16, 1.0, transform="tensor")
    import ctypes
    opt = stmg.make_options()
    opt.transform = 3
    nlev, ms = ctypes.c_int(), ctypes.c_double()
    rc = stmg.lib().st_plan(ctypes.byref(stmg.StMesh(2, 63)), 1, 16, 1.0, ctypes.byref(opt), 0, None, None, None,
                            None, ctypes.byref(nlev), ctypes.byref(ms))
    assert rc == stmg.ST_EINVAL
