"""Pins of the oracle at high time degree (Example 2 of the paper sweeps
p_t up to 45): the quadrature-assembled time matrices against closed forms
and structure, the multigrid fixed point against a direct solve, and the
iteration counts of the Example 2 protocol in a bounded band."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import dg_time, multigrid, spacetime, transfer


@pytest.mark.parametrize("p", [4, 10, 25, 45])
def test_time_matrices_closed_forms(p):
    """Legendre slab basis: K_tau[k,l] = 1 - 2 [l < k, k - l odd],
    M_tau = tau diag(1 / (2k + 1)), N_tau = st en^T with st_k = (-1)^k, en_k = 1."""
    tau = 0.37
    K, M, Nt = dg_time.time_matrices(p, tau)
    q = p + 1
    k, l = np.meshgrid(np.arange(q), np.arange(q), indexing="ij")
    Kc = 1.0 - 2.0 * ((l < k) & ((k - l) % 2 == 1))
    assert np.abs(K - Kc).max() < 1e-10
    assert np.abs(M - tau * np.diag(1.0 / (2 * np.arange(q) + 1))).max() < 1e-12 * tau
    assert np.abs(Nt - np.outer((-1.0) ** np.arange(q), np.ones(q))).max() < 1e-10


@pytest.mark.parametrize("p", [4, 10, 45])
def test_time_restriction_is_lower_triangular_and_exact_on_polynomials(p):
    """R_s[k, l] (coarse k <- fine l) vanishes for l > k (a coarse P_k restricted
    to half the slab has degree k), and R_s^T maps every coarse polynomial onto
    its restriction exactly."""
    R1, R2 = transfer.time_blocks(p, 1.0)
    assert np.abs(np.triu(R1, 1)).max() < 1e-10 and np.abs(np.triu(R2, 1)).max() < 1e-10
    q = p + 1
    s = np.linspace(-1.0, 1.0, 7)
    from numpy.polynomial import legendre as Lg
    for kc in [0, q // 2, q - 1]:
        coarse = np.zeros(q)
        coarse[kc] = 1.0
        for R, shift in [(R1, -1.0), (R2, 1.0)]:
            fine = R.T @ coarse                        # fine coefficients on that half
            assert np.abs(Lg.legval(s, fine) - Lg.legval((s + shift) / 2.0, coarse)).max() < 1e-9


@pytest.mark.parametrize("d,n,N,p", [(1, 7, 4, 10), (2, 3, 4, 6), (1, 3, 4, 45)])
def test_high_order_fixed_point_equals_direct_solve(d, n, N, p):
    H = multigrid.Hierarchy(d, n, p, N, 1.0)
    disc = H.finest.disc
    f = np.random.default_rng(6).uniform(-1, 1, disc.shape())
    u, it, _ = multigrid.solve(H, f, rtol=1e-13, maxit=80)
    ud = spla.spsolve(spacetime.global_matrix(disc), f.reshape(-1)).reshape(disc.shape())
    assert np.abs(u - ud).max() <= 1e-10 * np.abs(ud).max()


@pytest.mark.parametrize("p", [0, 1, 3, 10, 45])
def test_example2_iteration_counts_bounded(p):
    """Example 2 protocol (tau = 1, f = 0, u^0 ~ U[0, 1], eps = 1e-8) on a small
    Q1 grid: the paper's Table 2 reports 4-7 V-cycles for every p_t; on the
    tensor grid with the exact block inverse the counts stay in 3-9."""
    d, n, N = 2, 7, 16
    H = multigrid.Hierarchy(d, n, p, N, float(N))
    disc = H.finest.disc
    u0 = np.random.default_rng(0).uniform(0.0, 1.0, disc.shape())
    _, it, _ = multigrid.solve(H, np.zeros(disc.shape()), u=u0, rtol=1e-8, maxit=40)
    assert 3 <= it <= 9, it


def _paper_table2():
    import os
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "example2_iterations.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        vals = [int(v) for v in line.split()]
        rows[vals[0]] = vals[1:]
    return [0, 1, 2, 3, 4, 5, 10, 15, 20, 25, 30, 35, 40, 45], rows


def test_example2_iterations_against_the_papers_table():
    """The same protocol on the 15^2 Q1 grid (N = 32, tau = 1) against the
    printed counts of the refined levels (all 7): within one V-cycle for every
    p_t.  The paper's triangles and our tensor grid are different meshes, so
    only the band is compared."""
    degrees, rows = _paper_table2()
    paper = dict(zip(degrees, rows[3]))
    for p in [0, 5, 20, 45]:   # a subset keeps the CPU suite short; the GPU test sweeps all
        ref = paper[p]
        H = multigrid.Hierarchy(2, 15, p, 32, 32.0)
        disc = H.finest.disc
        u0 = np.random.default_rng(0).uniform(0.0, 1.0, disc.shape())
        _, it, _ = multigrid.solve(H, np.zeros(disc.shape()), u=u0, rtol=1e-8, maxit=40)
        assert abs(it - ref) <= 1, (p, it, ref)
