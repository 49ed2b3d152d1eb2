"""st_norm2_noalloc, the norm for callers that cannot allocate device memory,
against st_norm2 through the C ABI.  Kept in its own file that pytest
collects last."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1411_0519_gb300 import stmg
    return stmg, stmg.lib()


def test_noalloc_norm_matches_st_norm2_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stmg, lib = _lib()
    solver = stmg.Solver(2, 7, 1, 4, 1.0)          # only for the reference entry point st_norm2
    stream = torch.cuda.current_stream()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    # two calls in a row on different data (the second must not see the first's partials)
    for seed, n in [(0, 3 * (1 << 16) + 12345), (1, 1000)]:
        x = torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, n)).cuda()
        rc = lib.st_norm2_noalloc(ctypes.c_void_p(x.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream))
        assert rc == stmg.ST_OK
        ref = solver.norm2(x)
        got = float(out.item())
        assert abs(got - ref) <= 1e-13 * ref, (got, ref)
    solver.close()


def test_noalloc_norm_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stmg, lib = _lib()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = lib.st_norm2_noalloc(ctypes.c_void_p(x.data_ptr()), stmg.ST_NOALLOC_MAX_ELEMENTS + 1,
                              ctypes.c_void_p(out.data_ptr()), None)
    assert rc == stmg.ST_EINVAL
    assert lib.st_norm2_noalloc(None, 4, ctypes.c_void_p(out.data_ptr()), None) == stmg.ST_EINVAL
