"""Seeded synthetic inputs for the space-time heat-equation solver.

This module generates inputs only: it contains none of the solver's
arithmetic (no assembled matrix, no transfer, no smoother) and is shared by
the tests, the benchmark and the CPU reference.  All values are FP64 NumPy
arrays in the solver's layout u[n][l][z][y][x] (time step, time dof, then
space with x fastest); a load vector is given directly by its entries.

Workloads (unit square / cube, homogeneous Dirichlet, p_t = DG degree):
  heat1d_63      1D, 63 nodes, p_t=1, N=64,  T=1, manufactured solution
                 u = sin(pi x) cos t (load by quadrature in the tests)
  heat2d_255     2D, 255^2 nodes, p_t=1, N=1024, T=1; f ~ U[-1,1] seed 0,
                 u0 = sin(pi x) sin(pi y)
  heat3d_63      3D, 63^3 nodes, p_t=2, N=512, T=1; f = lumped load of a sum
                 of 16 Gaussians (sigma ~ U[0.05, 0.2]) seed 0, u0 = 0
  adjoint2d_127  2D, 127^2 nodes, p_t=1, N=256, T=1; f ~ U[-1,1] seed 1,
                 smooth u0 seed 2, target u_d = low-mode sine series seed 0
  heat2d_511     2D, 511^2 nodes, p_t=1, N=2048, T = mu/128 for
                 mu in {1/16, 1/4, 1, 16}; f ~ U[-1,1] seed 0
  heat2d_255_n256  heat2d_255 cut to its first 256 time steps (profiling)
  example2_p45     Example 2 protocol at the highest degree of its table: 127^2 Q1,
                   p_t = 45, tau = 1 (N = 64, T = 64), f = 0, iterate ~ U[0, 1]
  heat3d_63_n64    heat3d_63 cut to its first 64 time steps (profiling)
"""
import numpy as np

WORKLOADS = {
    "heat1d_63": dict(d=1, n=63, p_t=1, N=64, T=1.0, rtol=1e-10),
    "heat2d_255": dict(d=2, n=255, p_t=1, N=1024, T=1.0, rtol=1e-8),
    "heat3d_63": dict(d=3, n=63, p_t=2, N=512, T=1.0, rtol=1e-8),
    "adjoint2d_127": dict(d=2, n=127, p_t=1, N=256, T=1.0, rtol=1e-10),
    "heat2d_511": dict(d=2, n=511, p_t=1, N=2048, T=1.0 / 128.0, rtol=1e-8),
    # profiling case: the 255^2 mesh and tau of heat2d_255 on 256 time steps
    # (33M unknowns, 266 MB per vector: above L2, a few GB on the device)
    "heat2d_255_n256": dict(d=2, n=255, p_t=1, N=256, T=0.25, rtol=1e-8),
    "example2_p45": dict(d=2, n=127, p_t=45, N=64, T=64.0, rtol=1e-8),
    # profiling case in 3D: the 63^3 mesh and tau of heat3d_63 on 64 time steps
    # (48M unknowns, 384 MB per vector: above L2, a few GB on the device)
    "heat3d_63_n64": dict(d=3, n=63, p_t=2, N=64, T=0.125, rtol=1e-8),
}


def shape(d, n, p_t, N):
    """Solver layout of a space-time vector: (N, q, n, ..., n)."""
    return (N, p_t + 1) + (n,) * d


def nodes(n):
    return np.arange(1, n + 1, dtype=np.float64) / (n + 1.0)


def grid(d, n):
    """Nodal coordinate arrays (x, y, z order), each shaped (n,)*d with x fastest."""
    g = np.meshgrid(*([nodes(n)] * d), indexing="ij")   # slowest axis first
    return g[::-1]


def uniform_load(d, n, p_t, N, seed=0):
    """Load-vector entries i.i.d. U[-1, 1]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=shape(d, n, p_t, N))


def uniform_load_steps(d, n, p_t, N, s0, s1, seed=0):
    """Time steps [s0, s1) of uniform_load(d, n, p_t, N, seed), drawn without the
    others: the generator (one 64-bit draw per FP64 value) is advanced past the
    entries of the first s0 steps."""
    per_step = (p_t + 1) * n ** d
    rng = np.random.default_rng(seed)
    rng.bit_generator.advance(s0 * per_step)
    return rng.uniform(-1.0, 1.0, size=(s1 - s0, p_t + 1) + (n,) * d)


def uniform_iterate(d, n, p_t, N, seed=0):
    """Random initial iterate with entries in [0, 1] (two-grid protocol)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=shape(d, n, p_t, N))


def sine_ic(d, n):
    """Nodal values of prod_a sin(pi x_a)."""
    out = np.ones((n,) * d)
    for c in grid(d, n):
        out = out * np.sin(np.pi * c)
    return out


def smooth_ic(d, n, seed=2, modes=4):
    """Nodal values of a random low-mode sine series."""
    rng = np.random.default_rng(seed)
    coords = grid(d, n)
    out = np.zeros((n,) * d)
    for ks in np.ndindex(*([modes] * d)):
        term = rng.standard_normal() / (1.0 + sum(k * k for k in ks))
        for k, c in zip(ks, coords):
            term = term * np.sin(np.pi * (k + 1) * c)
        out = out + term
    return out


def gaussian_load(d, n, p_t, N, T, seed=0, count=16):
    """Lumped load of g(x) = sum_i a_i exp(-|x - c_i|^2 / (2 s_i^2)),
    a_i ~ U[-1,1], c_i ~ U[0,1]^d, s_i ~ U[0.05, 0.2], time independent:
    entry (n, l=0, j) = tau h^d g(x_j), entries with l >= 1 are zero."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, count)
    c = rng.uniform(0.0, 1.0, (count, d))
    s = rng.uniform(0.05, 0.2, count)
    coords = grid(d, n)
    g = np.zeros((n,) * d)
    for i in range(count):
        r2 = sum((coords[ax] - c[i, ax]) ** 2 for ax in range(d))
        g = g + a[i] * np.exp(-r2 / (2.0 * s[i] ** 2))
    tau = T / N
    h = 1.0 / (n + 1)
    out = np.zeros(shape(d, n, p_t, N))
    out[:, 0] = tau * h ** d * g
    return out


def smooth_target(d, n, p_t, N, T, seed=0, modes=8):
    """Target field u_d: sum_{k,l<=modes} c_kl / (k^2 + l^2) sin(k pi x) sin(l pi y)
    times cos(t) at the slab midpoint in the l = 0 coefficient, c ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    coords = grid(d, n)
    g = np.zeros((n,) * d)
    for ks in np.ndindex(*([modes] * d)):
        kk = [k + 1 for k in ks]
        term = rng.standard_normal() / float(sum(k * k for k in kk))
        for k, c in zip(kk, coords):
            term = term * np.sin(np.pi * k * c)
        g = g + term
    tau = T / N
    tm = (np.arange(N) + 0.5) * tau
    out = np.zeros(shape(d, n, p_t, N))
    out[:, 0] = np.cos(tm)[(slice(None),) + (None,) * d] * g
    return out


def random_directions(shp, count, seed=3):
    """``count`` seeded unit directions of the given shape."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        v = rng.standard_normal(shp)
        out.append(v / np.linalg.norm(v))
    return out
