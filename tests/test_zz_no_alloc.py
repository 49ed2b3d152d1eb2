"""st_norm2_noalloc, the norm for callers that cannot allocate device memory,
through the C ABI: against st_norm2 (the entry point that allocates its
workspace in a handle) and against an exactly rounded host sum.  Kept in its
own file that pytest collects last."""
import ctypes
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

CHUNK = 1 << 16   # elements per partial sum of the allocation-free kernel


def _lib():
    from paper_1411_0519_gb300 import stmg
    return stmg, stmg.lib()


def _host_norm(x):
    """||x||_2 from an exactly rounded sum of the squares (math.fsum on the host)."""
    a = np.asarray(x, dtype=np.float64)
    return math.sqrt(math.fsum((a * a).tolist())) if a.size else 0.0


def _call(lib, x, n, out, stream):
    return lib.st_norm2_noalloc(ctypes.c_void_p(x.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_norm_matches_st_norm2_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stmg, lib = _lib()
    solver = stmg.Solver(2, 7, 1, 4, 1.0)          # only for the reference entry point st_norm2
    stream = torch.cuda.current_stream()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    # two calls in a row on different data (the second must not see the first's partials)
    for seed, n in [(0, 3 * CHUNK + 12345), (1, 1000)]:
        x = torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, n)).cuda()
        assert _call(lib, x, n, out, stream) == stmg.ST_OK
        ref = solver.norm2(x)
        got = float(out.item())
        assert abs(got - ref) <= 1e-13 * ref, (got, ref)
    solver.close()


def test_noalloc_norm_chunk_edges_and_stale_partials():
    """n = 0 (one empty partial), exact multiples of the chunk (the last partial
    is full), and a large call followed by a short one (partials beyond the
    short call's count stay stale and must not be read), each against the host."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stmg, lib = _lib()
    stream = torch.cuda.current_stream()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    big = np.random.default_rng(7).uniform(-3, 3, 5 * CHUNK + 17)
    cases = [0, CHUNK, 2 * CHUNK, 5 * CHUNK + 17, 3, CHUNK - 1, CHUNK + 1]
    for n in cases:
        host = big[:n]
        x = torch.from_numpy(host.copy()).cuda() if n else torch.zeros(1, dtype=torch.float64, device="cuda")
        out.fill_(-1.0)
        assert _call(lib, x, n, out, stream) == stmg.ST_OK
        got = float(out.item())
        ref = _host_norm(host)
        assert abs(got - ref) <= 1e-14 * max(ref, 1e-300) or (n == 0 and got == 0.0), (n, got, ref)


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
