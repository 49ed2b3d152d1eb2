"""P1 finite elements on uniformly refined simplicial meshes (Section 4,
Examples 1 and 2): the unit square split into 4 triangles and the unit cube
split into 12 tetrahedra, each refined uniformly several times.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper (it prints no mesh):
* the 4 triangles of the unit square share its centre (0.5, 0.5), one per
  side of the square;
* the 12 tetrahedra of the unit cube share its centre, two per face, each face
  split along the diagonal through its corners of even coordinate sum;
* uniform refinement: a triangle is split at its edge midpoints into 4, a
  tetrahedron at its edge midpoints into 8 (4 corner tetrahedra and the inner
  octahedron cut along the diagonal between the midpoints of edges 02 and 13;
  J. Bey's rule);
* the mesh size h of a level is its longest edge (the coarsening rule of
  Section 4 uses mu = tau / h^2);
* homogeneous Dirichlet conditions: the unknowns are the vertices off the
  boundary of the cube, ordered by their coordinates (z, then y, then x).

The mass and stiffness matrices are assembled element by element from their
definitions (Section 1), int phi_i phi_j and int grad phi_i . grad phi_j, with
a quadrature rule exact for quadratics on each simplex and the barycentric
hat functions; the prolongation of the nested spaces evaluates every coarse
hat function at every fine vertex (P[i, j] = phi_j^coarse(x_i^fine)).
"""
import numpy as np
import scipy.sparse as sp


class Mesh:
    """Vertices (nv, d) and simplices (nc, d + 1) of a conforming mesh of (0,1)^d."""

    def __init__(self, verts, cells):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.cells = np.asarray(cells, dtype=np.int64)

    @property
    def d(self):
        return self.verts.shape[1]

    def interior(self):
        """Indices of the vertices off the boundary, ordered by (z, y, x)."""
        v = self.verts
        inside = np.all((v > 0.0) & (v < 1.0), axis=1)
        idx = np.nonzero(inside)[0]
        keys = [v[idx, a] for a in range(self.d)]          # np.lexsort: last key is primary
        return idx[np.lexsort(keys)]

    def edges(self):
        e = set()
        for c in self.cells:
            for a in range(len(c)):
                for b in range(a + 1, len(c)):
                    e.add((min(c[a], c[b]), max(c[a], c[b])))
        return sorted(e)

    def size(self):
        """Longest edge."""
        return max(np.linalg.norm(self.verts[a] - self.verts[b]) for a, b in self.edges())


def unit_square_four_triangles():
    verts = [(0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (0.0, 1.0), (0.5, 0.5)]
    cells = [(0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4)]
    return Mesh(verts, cells)


def unit_cube_twelve_tetrahedra():
    corners = [(x, y, z) for z in (0.0, 1.0) for y in (0.0, 1.0) for x in (0.0, 1.0)]
    verts = corners + [(0.5, 0.5, 0.5)]
    centre = len(corners)
    index = {c: i for i, c in enumerate(corners)}
    cells = []
    for axis in range(3):
        for side in (0.0, 1.0):
            face = [c for c in corners if c[axis] == side]
            even = [c for c in face if int(sum(c)) % 2 == 0]
            odd = [c for c in face if int(sum(c)) % 2 == 1]
            for o in odd:                                   # two triangles sharing the even diagonal
                cells.append((index[even[0]], index[even[1]], index[o], centre))
    return Mesh(verts, cells)


def refine(mesh):
    """One uniform refinement (red refinement of triangles, Bey's rule for tetrahedra)."""
    verts = [tuple(v) for v in mesh.verts]
    mid = {}

    def m(a, b):
        key = (min(a, b), max(a, b))
        if key not in mid:
            mid[key] = len(verts)
            verts.append(tuple(0.5 * (np.asarray(verts[a]) + np.asarray(verts[b]))))
        return mid[key]

    cells = []
    for c in mesh.cells:
        if mesh.d == 2:
            v0, v1, v2 = c
            m01, m12, m02 = m(v0, v1), m(v1, v2), m(v0, v2)
            cells += [(v0, m01, m02), (v1, m12, m01), (v2, m02, m12), (m01, m12, m02)]
        else:
            x0, x1, x2, x3 = c
            x01, x02, x03 = m(x0, x1), m(x0, x2), m(x0, x3)
            x12, x13, x23 = m(x1, x2), m(x1, x3), m(x2, x3)
            cells += [(x0, x01, x02, x03), (x01, x1, x12, x13), (x02, x12, x2, x23), (x03, x13, x23, x3),
                      (x01, x02, x03, x13), (x01, x02, x12, x13), (x02, x03, x13, x23), (x02, x12, x13, x23)]
    return Mesh(np.array(verts), np.array(cells))


def refined(mesh, times):
    for _ in range(times):
        mesh = refine(mesh)
    return mesh


def _quadrature(d):
    """Points (barycentric, (G, d+1)) and weights on the reference simplex (volume
    1/d!), exact for polynomials of degree 2."""
    if d == 2:
        lam = np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]])
        return lam, np.full(3, 1.0 / 6.0)
    a = (5.0 - np.sqrt(5.0)) / 20.0
    b = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
    lam = np.full((4, 4), a)
    np.fill_diagonal(lam, b)
    return lam, np.full(4, 1.0 / 24.0)


def p1_matrices(mesh):
    """(M_h, K_h) on the interior vertices (order of Mesh.interior()), assembled
    element by element by quadrature of the definitions."""
    d = mesh.d
    inner = mesh.interior()
    pos = -np.ones(len(mesh.verts), dtype=np.int64)
    pos[inner] = np.arange(len(inner))
    lam, wq = _quadrature(d)
    rows, cols, mv, kv = [], [], [], []
    for c in mesh.cells:
        x = mesh.verts[c]
        J = (x[1:] - x[0]).T                               # x = x0 + J xi
        det = abs(np.linalg.det(J))
        Jinv = np.linalg.inv(J)
        grads = np.vstack([-Jinv.sum(axis=0), Jinv])       # grad lambda_i as rows
        for a in range(d + 1):
            ia = pos[c[a]]
            if ia < 0:
                continue
            for b in range(d + 1):
                ib = pos[c[b]]
                if ib < 0:
                    continue
                rows.append(ia)
                cols.append(ib)
                mv.append(det * np.sum(wq * lam[:, a] * lam[:, b]))
                kv.append(det * np.sum(wq) * float(grads[a] @ grads[b]))
    n = len(inner)
    M = sp.csr_matrix((mv, (rows, cols)), shape=(n, n))
    K = sp.csr_matrix((kv, (rows, cols)), shape=(n, n))
    M.sum_duplicates()
    K.sum_duplicates()
    return M, K


def prolongation(coarse, fine):
    """P (fine interior x coarse interior): P[i, j] = value of the coarse hat
    function of vertex j at fine vertex i (the embedding of the nested P1
    spaces), found by locating each fine vertex in a coarse simplex."""
    d = coarse.d
    ci, fi = coarse.interior(), fine.interior()
    cpos = -np.ones(len(coarse.verts), dtype=np.int64)
    cpos[ci] = np.arange(len(ci))
    P = sp.lil_matrix((len(fi), len(ci)))
    X = coarse.verts[coarse.cells]                          # (nc, d+1, d)
    Jinv = np.linalg.inv(np.transpose(X[:, 1:] - X[:, :1], (0, 2, 1)))
    for row, v in enumerate(fi):
        p = fine.verts[v]
        xi = np.einsum("cij,cj->ci", Jinv, p - X[:, 0])
        bary = np.hstack([1.0 - xi.sum(axis=1, keepdims=True), xi])
        cell = int(np.argmax(bary.min(axis=1)))
        assert bary[cell].min() >= -1e-12, "fine vertex outside the coarse mesh"
        for a in range(d + 1):
            j = cpos[coarse.cells[cell, a]]
            if j >= 0 and abs(bary[cell, a]) > 1e-14:
                P[row, j] = bary[cell, a]
    return P.tocsr()


class MeshSpace:
    """One spatial level: the mesh, its interior vertices and (M_h, K_h)."""

    def __init__(self, mesh):
        self.mesh = mesh
        self.d = mesh.d
        self.Mh, self.Kh = p1_matrices(mesh)
        self.Nx = self.Mh.shape[0]
        self.h = mesh.size()
        self.nodes = mesh.verts[mesh.interior()]


class MeshFamily:
    """Spatial levels 0 .. refinements of one initial mesh, with the prolongations
    P_l from level l - 1 to level l (P[0] is None)."""

    def __init__(self, initial, refinements):
        meshes = [initial]
        for _ in range(refinements):
            meshes.append(refine(meshes[-1]))
        self.spaces = [MeshSpace(m) for m in meshes]
        self.P = [None] + [prolongation(meshes[i - 1], meshes[i]) for i in range(1, len(meshes))]
