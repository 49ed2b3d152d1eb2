"""The sine basis change of the exact block inverse (Section 3.1) through st_transform: the
tensor-core form (exact digit products, ST_DST_TENSOR) and the FFT form (ST_DST_FFT) against
SciPy's DST-I, on random fields with a spread of line scales and on special lines (zeros,
subnormals, magnitudes near the ends of the FP64 range, Inf / NaN)."""
import numpy as np
import pytest
import scipy.fft

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_1411_0519_gb300 import stmg  # noqa: E402

CASES = [(1, 63), (1, 255), (2, 63), (2, 127), (2, 255), (3, 63)]
# normwise error bounds per field: the tensor-core form rounds once per axis pass from exact
# integer sums; an FFT's error grows like eps log2(n + 1) (measured 4.1e-15 at n = 255)
TOL = {"tensor": 2e-15, "fft": 1e-14}


def ref_transform(x, dim, inverse=False):
    """S x along the last dim axes with S_jk = sin(pi j k / (n + 1)); SciPy's DST-I has a factor 2."""
    axes = tuple(range(x.ndim - dim, x.ndim))
    y = scipy.fft.dstn(x, type=1, axes=axes) / 2.0 ** dim
    if inverse:
        y = y * (2.0 / (x.shape[-1] + 1)) ** dim
    return y


def fields(dim, n, slabs, seed):
    """slabs fields of n^dim values, every line along x scaled by its own power of two."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.0, 1.0, (slabs,) + (n,) * dim)
    e = rng.integers(-40, 41, (slabs,) + (n,) * (dim - 1) + (1,))
    return np.ldexp(x, e)


def solver(dim, n, transform, N=4):
    return stmg.Solver(dim, n, 1, N, 1.0, transform=transform)


def rel_field_error(y, ref, dim):
    """max over fields of ||y - ref||_2 / ||ref||_2."""
    ax = tuple(range(1, 1 + dim))
    num = np.sqrt(np.sum((y - ref) ** 2, axis=ax))
    den = np.sqrt(np.sum(ref ** 2, axis=ax))
    return float(np.max(num / np.where(den > 0, den, 1.0)))


@pytest.mark.parametrize("dim,n", CASES)
@pytest.mark.parametrize("transform", ["tensor", "fft"])
def test_transform_matches_scipy(dim, n, transform):
    x = fields(dim, n, 6, 100 * dim + n)
    s = solver(dim, n, transform)
    try:
        xd = torch.from_numpy(x).cuda()
        y = s.transform(xd).cpu().numpy()
        yi = s.transform(xd, inverse=True).cpu().numpy()
    finally:
        s.close()
    # the fields mix line scales over 2^80
    assert rel_field_error(y, ref_transform(x, dim), dim) < TOL[transform]
    assert rel_field_error(yi, ref_transform(x, dim, inverse=True), dim) < TOL[transform]


@pytest.mark.parametrize("dim,n", [(1, 255), (2, 255), (3, 63)])
def test_tensor_equals_fft_and_round_trip(dim, n):
    x = fields(dim, n, 5, 7 + n)
    st, sf = solver(dim, n, "tensor"), solver(dim, n, "fft")
    try:
        xd = torch.from_numpy(x).cuda()
        yt = st.transform(xd)
        yf = sf.transform(xd)
        back = st.transform(yt, inverse=True)
    finally:
        st.close()
        sf.close()
    assert rel_field_error(yt.cpu().numpy(), yf.cpu().numpy(), dim) < TOL["fft"] + TOL["tensor"]
    assert rel_field_error(back.cpu().numpy(), x, dim) < 2 * TOL["tensor"]


def test_tensor_batches_in_place_and_ragged_blocks():
    """300 fields of 255^2: two slab batches of the tensor path, a line count that is not a
    multiple of the 128-line tile; in place (x is y)."""
    dim, n, slabs = 2, 255, 300
    x = fields(dim, n, slabs, 3)
    s = solver(dim, n, "tensor")
    try:
        xd = torch.from_numpy(x).cuda()
        s.transform(xd, out=xd)
        y = xd.cpu().numpy()
    finally:
        s.close()
    assert rel_field_error(y, ref_transform(x, dim), dim) < TOL["tensor"]


def special_lines(n):
    """Rows of n values that stress the digit split: zero, one spike, near-overflow, subnormal,
    smallest subnormals, mixed magnitudes within the line, constant."""
    rng = np.random.default_rng(5)
    rows = [
        np.zeros(n),
        np.where(np.arange(n) == 7, 3.0, 0.0),
        np.ldexp(rng.uniform(-1, 1, n), 1000),
        np.ldexp(rng.uniform(-1, 1, n), -1040),
        np.ldexp(1.0, -1074) * (np.arange(n) + 1.0),
        np.where(np.arange(n) % 2 == 1, np.ldexp(rng.uniform(-1, 1, n), 30), np.ldexp(rng.uniform(-1, 1, n), -30)),
        -np.ones(n),
        np.ldexp(rng.uniform(-1, 1, n), -1000),
    ]
    return np.stack(rows)


def test_tensor_special_lines_1d():
    n = 255
    x = special_lines(n)
    s = solver(1, n, "tensor")
    try:
        y = s.transform(torch.from_numpy(x).cuda()).cpu().numpy()
    finally:
        s.close()
    # exact products in extended precision: y_k = sum_j x_j sin(pi j k / 256), the argument
    # reduced exactly (j k mod 512) and pi in long double
    j = np.arange(1, n + 1)
    pi_l = np.longdouble("3.14159265358979323846264338327950288")
    S = np.sin(pi_l * (np.outer(j, j) % (2 * (n + 1))).astype(np.longdouble) / (n + 1))
    for r in range(x.shape[0]):
        exact = x[r].astype(np.longdouble) @ S
        scale = np.sqrt((n + 1) / 2.0) * np.sqrt(np.sum(x[r].astype(np.longdouble) ** 2))
        if scale == 0:
            assert np.all(y[r] == 0.0)
            continue
        err = np.abs(y[r].astype(np.longdouble) - exact)
        # the FP64 result cannot be finer than the smallest subnormal 2^-1074
        err = np.maximum(err - np.ldexp(np.longdouble(1.0), -1074), 0)
        assert float(np.max(err) / scale) < 1e-15, r
        assert np.all(np.isfinite(y[r]))


def test_tensor_non_finite_lines():
    """A line holding Inf or NaN comes out non-finite (as with the FFT); the others are unaffected."""
    n = 127
    x = fields(1, n, 4, 11)
    x[1, 5] = np.inf
    x[2, 9] = np.nan
    st, sf = solver(1, n, "tensor"), solver(1, n, "fft")
    try:
        yt = st.transform(torch.from_numpy(x).cuda()).cpu().numpy()
        yf = sf.transform(torch.from_numpy(x).cuda()).cpu().numpy()
    finally:
        st.close()
        sf.close()
    for r in (1, 2):
        assert not np.all(np.isfinite(yt[r])) and not np.all(np.isfinite(yf[r]))
    for r in (0, 3):
        assert np.all(np.isfinite(yt[r]))
        ref = ref_transform(x[r:r + 1], 1)
        assert rel_field_error(yt[r:r + 1], ref, 1) < TOL["tensor"]


@pytest.mark.parametrize("dim,n,precision", [(2, 127, "fp64"), (2, 127, "mixed"), (3, 63, "fp64"), (1, 255, "fp64")])
def test_solve_tensor_equals_fft(dim, n, precision):
    """The whole solve with either transform: iteration counts and solutions agree within the
    transforms' rounding as amplified by the solve."""
    N, p_t = 16, 1
    rng = np.random.default_rng(2)
    f = torch.from_numpy(rng.standard_normal((N, p_t + 1) + (n,) * dim)).cuda()
    u0 = torch.from_numpy(rng.standard_normal((n,) * dim)).cuda()
    out = {}
    for tr in ("tensor", "fft"):
        s = stmg.Solver(dim, n, p_t, N, 1.0, precision=precision, transform=tr, rtol=1e-10)
        try:
            u, it, rr = s.solve(f, u0)
            out[tr] = (u.cpu().numpy(), it, rr)
        finally:
            s.close()
    ut, it_t, _ = out["tensor"]
    uf, it_f, _ = out["fft"]
    # FP64: the same iterations; mixed: the FP32 cycles see transforms of different rounding
    assert abs(it_t - it_f) <= (0 if precision == "fp64" else 1)
    assert np.linalg.norm(ut - uf) / np.linalg.norm(uf) < 1e-11


def test_tensor_option_rejected_outside_range():
    with pytest.raises(stmg.StmgError):
        stmg.Solver(2, 511, 1, 4, 1.0, transform="tensor")
