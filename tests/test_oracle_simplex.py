"""Pins of the oracle's P1 spaces on the paper's simplicial meshes (Section 4,
Examples 1 and 2: the unit square in 4 triangles, the unit cube in 12
tetrahedra, refined uniformly) and of the space-time multigrid on them.

Independent of the oracle's quadrature assembly: closed-form mesh counts, the
textbook element mass |T| (1 + delta_ij) / ((d+1)(d+2)), the stiffness from the
geometry of the opposite facets (cotangent formula in 2D, facet normals and
areas in 3D), the vanishing discrete Laplacian of linear functions, the
Galerkin identities of nested conforming spaces (P^T M_f P = M_c,
P^T K_f P = K_c, R L_f P = L_c), the multigrid fixed point against a dense
direct solve, multigrid against forward substitution in time, and the
printed iteration counts of Example 2 within one cycle."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import mesh_multigrid as mm
from oracle import multigrid, simplex


def _family(d, levels):
    init = simplex.unit_square_four_triangles() if d == 2 else simplex.unit_cube_twelve_tetrahedra()
    return simplex.MeshFamily(init, levels)


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_square_mesh_counts(level):
    m = simplex.refined(simplex.unit_square_four_triangles(), level)
    k = 2 ** level
    assert len(m.cells) == 4 * 4 ** level
    assert len(m.verts) == (k + 1) ** 2 + k ** 2
    assert len(m.interior()) == (k - 1) ** 2 + k ** 2
    areas = [0.5 * abs(np.linalg.det(m.verts[c[1:]] - m.verts[c[0]])) for c in m.cells]
    assert abs(sum(areas) - 1.0) < 1e-14 and np.ptp(areas) < 1e-15   # congruent triangles
    assert abs(m.size() - 2.0 ** -level) < 1e-15


@pytest.mark.parametrize("level", [0, 1, 2])
def test_cube_mesh_counts(level):
    m = simplex.refined(simplex.unit_cube_twelve_tetrahedra(), level)
    k = 2 ** level
    assert len(m.cells) == 12 * 8 ** level
    assert len(m.verts) == (k + 1) ** 3 + k ** 3
    assert len(m.interior()) == (k - 1) ** 3 + k ** 3
    vols = [abs(np.linalg.det(m.verts[c[1:]] - m.verts[c[0]])) / 6.0 for c in m.cells]
    assert abs(sum(vols) - 1.0) < 1e-12 and min(vols) > 0


def _closed_form_matrices(mesh):
    """Mass |T| (1 + delta_ij) / ((d+1)(d+2)); stiffness |T| grad l_i . grad l_j with
    grad l_i = -n_i |F_i| / (d |T|), n_i the outward unit normal of the facet F_i
    opposite vertex i (2D: facet = edge, 3D: triangle)."""
    d = mesh.d
    inner = mesh.interior()
    pos = {v: i for i, v in enumerate(inner)}
    n = len(inner)
    M = np.zeros((n, n))
    K = np.zeros((n, n))
    for c in mesh.cells:
        x = mesh.verts[c]
        if d == 2:
            vol = 0.5 * abs((x[1, 0] - x[0, 0]) * (x[2, 1] - x[0, 1]) - (x[2, 0] - x[0, 0]) * (x[1, 1] - x[0, 1]))
        else:
            vol = abs(np.dot(np.cross(x[1] - x[0], x[2] - x[0]), x[3] - x[0])) / 6.0
        g = []
        for i in range(d + 1):
            others = [x[j] for j in range(d + 1) if j != i]
            if d == 2:
                e = others[1] - others[0]
                nrm = np.array([e[1], -e[0]])
                area = np.linalg.norm(e)
            else:
                nrm = np.cross(others[1] - others[0], others[2] - others[0])
                area = 0.5 * np.linalg.norm(nrm)
            nrm = nrm / np.linalg.norm(nrm)
            if np.dot(nrm, x[i] - others[0]) > 0:     # make it point away from vertex i
                nrm = -nrm
            g.append(-nrm * area / (d * vol))
        for a in range(d + 1):
            for b in range(d + 1):
                ia, ib = pos.get(c[a]), pos.get(c[b])
                if ia is None or ib is None:
                    continue
                M[ia, ib] += vol * (1.0 + (a == b)) / ((d + 1) * (d + 2))
                K[ia, ib] += vol * float(g[a] @ g[b])
    return M, K


@pytest.mark.parametrize("d,level", [(2, 0), (2, 1), (2, 2), (3, 0), (3, 1)])
def test_p1_matrices_against_closed_forms(d, level):
    init = simplex.unit_square_four_triangles() if d == 2 else simplex.unit_cube_twelve_tetrahedra()
    m = simplex.refined(init, level)
    M, K = simplex.p1_matrices(m)
    Mc, Kc = _closed_form_matrices(m)
    assert np.abs(M.toarray() - Mc).max() < 1e-15
    assert np.abs(K.toarray() - Kc).max() < 1e-13
    assert np.allclose(M.toarray(), M.toarray().T, atol=0) and np.allclose(K.toarray(), K.toarray().T, atol=1e-15)


@pytest.mark.parametrize("d,level", [(2, 3), (3, 2)])
def test_discrete_laplacian_of_linear_functions_vanishes(d, level):
    """sum_j K_ij g(x_j) = int grad phi_i . grad g = 0 for linear g at every vertex
    whose neighbours are all interior; sum_j M_ij = int phi_i = |supp phi_i| / (d+1)."""
    m = simplex.refined(simplex.unit_square_four_triangles() if d == 2 else simplex.unit_cube_twelve_tetrahedra(),
                        level)
    M, K = simplex.p1_matrices(m)
    inner = m.interior()
    x = m.verts[inner]
    g = 0.3 + x @ np.arange(1.0, d + 1.0)
    touching = set()
    for c in m.cells:
        if np.any(np.any((m.verts[c] == 0.0) | (m.verts[c] == 1.0), axis=1)):
            touching.update(c.tolist())
    away = [i for i, v in enumerate(inner) if v not in touching]
    assert len(away) > 0
    Kg = K @ g
    assert np.abs(Kg[away]).max() < 1e-12
    supp = np.zeros(len(m.verts))
    for c in m.cells:
        vol = abs(np.linalg.det(m.verts[c[1:]] - m.verts[c[0]])) / (2.0 if d == 2 else 6.0)
        supp[c] += vol
    assert np.abs((M @ np.ones(len(inner)))[away] - supp[inner][away] / (d + 1)).max() < 1e-15


@pytest.mark.parametrize("d,levels", [(2, 3), (3, 2)])
def test_prolongation_and_galerkin_identities(d, levels):
    fam = _family(d, levels)
    for l in range(1, levels + 1):
        P = fam.P[l]
        vals = np.unique(np.round(P.data, 14))
        assert set(vals.tolist()) <= {0.5, 1.0}
        fine, coarse = fam.spaces[l], fam.spaces[l - 1]
        assert np.abs((P.T @ fine.Mh @ P - coarse.Mh).toarray()).max() < 1e-15
        assert np.abs((P.T @ fine.Kh @ P - coarse.Kh).toarray()).max() < 1e-12
        # coarse vertices are fine vertices with weight 1
        ones = np.asarray((P == 1.0).sum(axis=0)).ravel()
        assert np.all(ones == 1)


@pytest.mark.parametrize("d,levels,p,N,T,coarsening", [
    (2, 2, 1, 8, 1.0, "full"), (2, 2, 2, 8, 1.0, "semi"), (3, 1, 1, 4, 0.5, "full"), (2, 3, 0, 16, 4.0, "auto")])
def test_space_time_galerkin_identity(d, levels, p, N, T, coarsening):
    """R L_{tau,h} R^T = L_{2 tau, h or H} with the mesh prolongation (nested spaces,
    Section 2: R = P^T), in the oracle's assembled operators."""
    fam = _family(d, levels)
    H = mm.MeshHierarchy(None, levels, p, N, T, coarsening=coarsening, family=fam, smoother="exact")
    for i in range(len(H.levels) - 1):
        f, c = H.levels[i], H.levels[i + 1]
        Lf = _global(f.disc)
        Lc = _global(c.disc)
        G = (f.R @ Lf @ f.R.T).toarray()
        assert np.abs(G - Lc.toarray()).max() < 1e-12 * np.abs(Lc.toarray()).max(), i


def _global(disc):
    N = disc.N
    return (sp.kron(sp.identity(N), disc.A) + sp.kron(sp.diags([np.ones(N - 1)], [-1], shape=(N, N)), disc.B)).tocsc()


@pytest.mark.parametrize("d,levels,p,N,smoother", [
    (2, 2, 1, 4, "vcycle"), (2, 1, 2, 8, "vcycle"), (2, 2, 0, 4, "exact"), (3, 1, 1, 4, "vcycle")])
def test_multigrid_fixed_point_is_the_direct_solution(d, levels, p, N, smoother):
    fam = _family(d, levels)
    H = mm.MeshHierarchy(None, levels, p, N, 1.0, family=fam, smoother=smoother)
    disc = H.finest.disc
    rng = np.random.default_rng(3)
    f = rng.uniform(-1, 1, disc.shape())
    direct = np.linalg.solve(_global(disc).toarray(), f.reshape(-1)).reshape(disc.shape())
    u, it, hist = multigrid.solve(H, f, rtol=1e-13, maxit=80)
    assert hist[-1] <= 1e-13 * hist[0]
    assert np.abs(u - direct).max() <= 1e-11 * np.abs(direct).max()
    fs = multigrid.forward_substitution(H.finest, f)
    assert np.abs(fs - direct).max() <= 1e-12 * np.abs(direct).max()
    lam, _, _ = multigrid.solve(H, f, rtol=1e-13, maxit=80, adjoint=True)
    directT = np.linalg.solve(_global(disc).toarray().T, f.reshape(-1)).reshape(disc.shape())
    assert np.abs(lam - directT).max() <= 1e-11 * np.abs(directT).max()


def test_inexact_block_inverse_is_a_convergent_approximate_inverse():
    """The spatial V-cycle D~^{-1} of the Remark on the V-cycle approximation in
    space satisfies ||I - D~^{-1} A|| < 1 on the mesh family, and its coarse
    operators are the Galerkin products of the finer ones."""
    fam = _family(2, 3)
    for p in (0, 1, 3):
        vc = mm.MeshSpatialVCycle(fam, 3, p, 0.1)
        A = vc.levels[0]["A"].toarray()
        n = A.shape[0]
        E = np.eye(n) - vc.apply(A)
        assert np.linalg.norm(E, 2) < 0.5, p
        for a, b in zip(vc.levels[:-1], vc.levels[1:]):
            G = (a["R"] @ a["A"] @ a["R"].T).toarray()
            assert np.abs(G - b["A"].toarray()).max() < 1e-13 * np.abs(G).max()


def test_coarsening_rule_on_meshes():
    """Section 4's rule with h the longest edge: tau = 1 on the refined square
    gives mu >= mu* on every mesh, so space coarsens first, then time alone."""
    fam = _family(2, 3)
    ps = mm.build_levels(fam, 3, 1, 16, 16.0)
    kinds = [lv["full"] for lv in ps[:-1]]
    assert kinds == [True, True, True, False]
    assert [lv["l"] for lv in ps] == [3, 2, 1, 0, 0]
    ps = mm.build_levels(fam, 3, 1, 16, 1.0 / 64)      # mu = tau / h^2 = 1/1024 / 2^-6 < mu*
    assert ps[0]["full"] is False


def _example2_rows(golden_dir):
    rows = {}
    for line in open(golden_dir + "/example2_iterations.txt"):
        if line.startswith("#") or not line.strip():
            continue
        vals = [int(v) for v in line.split()]
        rows[vals[0]] = vals[1:]
    return rows


@pytest.mark.slow
@pytest.mark.parametrize("space_level", [1, 2])
def test_example2_on_the_paper_mesh_within_one_cycle(space_level, golden_dir):
    """Example 2 (Section 4): the refined 4-triangle mesh, tau = 1, T = N = 1024,
    f = 0, u^0 ~ U[0, 1], the inexact block inverse, eps = 1e-8: V-cycle counts
    within one of the printed table for p_t = 0 ... 3."""
    rows = _example2_rows(golden_dir)
    fam = _family(2, space_level)
    got = []
    for p, ref in zip([0, 1, 2, 3], rows[space_level][:4]):
        N = 1024
        H = mm.MeshHierarchy(None, space_level, p, N, float(N), family=fam)
        disc = H.finest.disc
        u0 = np.random.default_rng(0).uniform(0.0, 1.0, disc.shape())
        _, it, hist = multigrid.solve(H, np.zeros(disc.shape()), u=u0, rtol=1e-8, maxit=40)
        got.append(it)
        assert abs(it - ref) <= 1, (p, it, ref)
    print("Example 2 on the refined 4-triangle mesh, level", space_level, ":", got)


# ---------------------------------------------------------------- planted mistakes
def _p1_with(mesh, quad=None, transpose_grad=False):
    """p1_matrices with a planted mistake: another quadrature rule for the mass,
    or the columns of J^{-1} taken as the gradients."""
    d = mesh.d
    inner = mesh.interior()
    pos = {v: i for i, v in enumerate(inner)}
    lam, wq = quad if quad is not None else simplex._quadrature(d)
    n = len(inner)
    M = np.zeros((n, n))
    K = np.zeros((n, n))
    for c in mesh.cells:
        x = mesh.verts[c]
        J = (x[1:] - x[0]).T
        det = abs(np.linalg.det(J))
        Jinv = np.linalg.inv(J)
        G = Jinv.T if transpose_grad else Jinv
        grads = np.vstack([-G.sum(axis=0), G])
        for a in range(d + 1):
            for b in range(d + 1):
                ia, ib = pos.get(c[a]), pos.get(c[b])
                if ia is None or ib is None:
                    continue
                M[ia, ib] += det * np.sum(wq * lam[:, a] * lam[:, b])
                K[ia, ib] += det * np.sum(wq) * float(grads[a] @ grads[b])
    return M, K


def test_mutations_of_the_assembly_are_caught():
    m = simplex.refined(simplex.unit_square_four_triangles(), 2)
    Mc, Kc = _closed_form_matrices(m)
    centroid = (np.full((1, 3), 1.0 / 3.0), np.array([0.5]))       # exact for degree 1 only
    M1, _ = _p1_with(m, quad=centroid)
    assert np.abs(M1 - Mc).max() > 1e-3
    m3 = simplex.refined(simplex.unit_cube_twelve_tetrahedra(), 1)
    Mc3, Kc3 = _closed_form_matrices(m3)
    _, Kt = _p1_with(m3, transpose_grad=True)
    assert np.abs(Kt - Kc3).max() > 1e-3


def test_mutation_of_the_prolongation_is_caught():
    fam = _family(2, 2)
    P = fam.P[2].tolil()
    P[P == 0.5] = 0.25                                              # quarter weights at edge midpoints
    P = P.tocsr()
    fine, coarse = fam.spaces[2], fam.spaces[1]
    assert np.abs((P.T @ fine.Mh @ P - coarse.Mh).toarray()).max() > 1e-3


@pytest.mark.slow
@pytest.mark.parametrize("space_level", [0, 1])
def test_example1_on_the_paper_mesh_within_one_cycle(space_level, golden_dir):
    """Example 1 (Section 4): the 12-tetrahedron cube refined uniformly, T = 1,
    N = 2^k, p_t = 1, f = 0, u^0 ~ U[0, 1], the inexact block inverse,
    eps = 1e-8: V-cycle counts within one of the printed table for time levels
    0 ... 6."""
    rows = {}
    for line in open(golden_dir + "/example1_iterations.txt"):
        if line.startswith("#") or not line.strip():
            continue
        vals = [int(v) for v in line.split()]
        rows[vals[0]] = vals[1:]
    fam = _family(3, space_level)
    got = []
    for k in range(7):
        H = mm.MeshHierarchy(None, space_level, 1, 2 ** k, 1.0, family=fam)
        disc = H.finest.disc
        u0 = np.random.default_rng(0).uniform(0.0, 1.0, disc.shape())
        _, it, _ = multigrid.solve(H, np.zeros(disc.shape()), u=u0, rtol=1e-8, maxit=40)
        got.append(it)
        assert abs(it - rows[space_level][k]) <= 1, (k, it, rows[space_level][k])
    print("Example 1 on the refined 12-tetrahedron cube, level", space_level, ":", got)
