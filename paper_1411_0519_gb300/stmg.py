"""Python binding of the stmg C ABI (include/stmg.h).

Argument marshalling only: every step of the solver runs in the CUDA library
libstmg.so.  PyTorch provides device memory and the stream.  If the library
has not been built, importing this module raises; there is no CPU fallback.

Space-time vectors are torch.float64 CUDA tensors of shape (N, q, n, ..., n)
(or any contiguous tensor with N q n^d elements) in the layout of the header:
time step, time dof (Legendre degree), then space with x fastest.
"""
import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_PKG, "libstmg.so")

ST_OK, ST_EINVAL, ST_ENOMEM, ST_ENOTCONV, ST_ENAN, ST_ECUDA = range(6)
ST_FP64, ST_MIXED = 0, 1
ST_AUTO, ST_SEMI, ST_FULL = 0, 1, 2
ST_INIT_GIVEN = 1
ST_MAX_PT = 47
ST_SMOOTH_EXACT, ST_SMOOTH_VCYCLE = 0, 1
ST_DST_AUTO, ST_DST_FFT, ST_DST_TENSOR = 0, 1, 2

EXPORTS = [
    "st_default_options", "st_setup", "st_destroy", "st_last_error", "st_ndof", "st_num_levels",
    "st_level_info", "st_residual", "st_vcycle", "st_solve", "st_solve_host", "st_adjoint_solve",
    "st_level_residual",
    "st_level_block_solve", "st_level_smooth", "st_level_restrict", "st_level_prolong",
    "st_coarsest_solve", "st_norm2", "st_profile_start", "st_profile_stop", "st_profile_level", "st_norm2_noalloc",
    "st_plan", "st_transform",
]

MESH_EXPORTS = [
    "stm_setup", "stm_destroy", "stm_last_error", "stm_ndof", "stm_num_levels", "stm_nodes", "stm_level_info",
    "stm_residual", "stm_vcycle", "stm_solve", "stm_adjoint_solve", "stm_level_residual", "stm_level_block_solve",
    "stm_level_smooth", "stm_level_restrict", "stm_level_prolong", "stm_coarsest_solve",
]

ST_NOALLOC_MAX_ELEMENTS = 1 << 30

KERNEL_CLASSES = ["residual", "dst", "smooth", "restrict", "prolong", "norm", "vector", "rhs", "space_mg", "dst_tc"]


class StMesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int)]


class StOptions(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega", ctypes.c_double),
                ("rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("precision", ctypes.c_int),
                ("coarsening", ctypes.c_int), ("coarsest_steps", ctypes.c_int),
                ("inner_cycles", ctypes.c_int), ("max_workspace_bytes", ctypes.c_size_t),
                ("smoother", ctypes.c_int), ("nu_x", ctypes.c_int), ("omega_x", ctypes.c_double),
                ("gamma", ctypes.c_int), ("transform", ctypes.c_int)]


class SimplexMesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nverts", ctypes.c_int), ("verts", ctypes.POINTER(ctypes.c_double)),
                ("ncells", ctypes.c_int), ("cells", ctypes.POINTER(ctypes.c_int))]


class StmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"stmg error {code}: {msg}")
        self.code = code


def library_path():
    return _LIBPATH


def load_library(path=None):
    """Load libstmg.so and declare the C signatures; raises if it is missing."""
    path = path or _LIBPATH
    if not os.path.exists(path):
        raise ImportError(f"stmg CUDA library not built ({path}); run "
                          "`python -m paper_1411_0519_gb300.build` or __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    H = ctypes.c_void_p
    sig = {
        "st_default_options": (None, [ctypes.POINTER(StOptions)]),
        "st_setup": (I, [ctypes.POINTER(StMesh), I, I, D, ctypes.POINTER(StOptions), P, ctypes.POINTER(H)]),
        "st_destroy": (None, [H]),
        "st_last_error": (ctypes.c_char_p, [H]),
        "st_ndof": (ctypes.c_size_t, [H]),
        "st_num_levels": (I, [H]),
        "st_level_info": (I, [H, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I)]),
        "st_plan": (I, [ctypes.POINTER(StMesh), I, I, D, ctypes.POINTER(StOptions), I, ctypes.POINTER(I),
                        ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(I),
                        ctypes.POINTER(D)]),
        "st_residual": (I, [H, P, P, P, P]),
        "st_vcycle": (I, [H, P, P, P]),
        "st_solve": (I, [H, P, P, P, I, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "st_solve_host": (I, [H, P, P, P, I, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "st_adjoint_solve": (I, [H, P, P, P, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "st_level_residual": (I, [H, I, I, P, P, P]),
        "st_level_block_solve": (I, [H, I, I, P, P]),
        "st_level_smooth": (I, [H, I, I, I, P, P]),
        "st_level_restrict": (I, [H, I, P, P]),
        "st_level_prolong": (I, [H, I, P, P]),
        "st_coarsest_solve": (I, [H, I, P, P]),
        "st_norm2": (I, [H, P, ctypes.c_size_t, ctypes.POINTER(D)]),
        "st_transform": (I, [H, I, I, P, P, ctypes.c_size_t]),
        "st_profile_start": (I, [H, I]),
        "st_norm2_noalloc": (I, [P, ctypes.c_size_t, P, P]),
        "st_profile_level": (I, [H, I, I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D),
                                 ctypes.POINTER(D)]),
        "st_profile_stop": (I, [H, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D),
                                ctypes.POINTER(I)]),
    }
    IP = ctypes.POINTER(I)
    DP = ctypes.POINTER(D)
    sig.update({
        "stm_setup": (I, [ctypes.POINTER(SimplexMesh), I, I, I, D, ctypes.POINTER(StOptions), P,
                          ctypes.POINTER(H)]),
        "stm_destroy": (None, [H]),
        "stm_last_error": (ctypes.c_char_p, [H]),
        "stm_ndof": (ctypes.c_size_t, [H]),
        "stm_num_levels": (I, [H]),
        "stm_nodes": (I, [H, I, IP, DP]),
        "stm_level_info": (I, [H, I, IP, IP, DP, IP]),
        "stm_residual": (I, [H, P, P, P, P]),
        "stm_vcycle": (I, [H, P, P, P]),
        "stm_solve": (I, [H, P, P, P, I, IP, DP]),
        "stm_adjoint_solve": (I, [H, P, P, P, IP, DP]),
        "stm_level_residual": (I, [H, I, I, P, P, P]),
        "stm_level_block_solve": (I, [H, I, I, P, P]),
        "stm_level_smooth": (I, [H, I, I, I, P, P]),
        "stm_level_restrict": (I, [H, I, P, P]),
        "stm_level_prolong": (I, [H, I, P, P]),
        "stm_coarsest_solve": (I, [H, I, P, P]),
    })
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _ptr(t, numel=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous torch.float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


_PRECISION = {"fp64": ST_FP64, "mixed": ST_MIXED}
_TRANSFORM = {"auto": ST_DST_AUTO, "fft": ST_DST_FFT, "tensor": ST_DST_TENSOR}
_COARSEN = {"auto": ST_AUTO, "semi": ST_SEMI, "full": ST_FULL}


def make_options(*, nu1=2, nu2=2, omega=0.5, rtol=1e-8, maxit=50, precision="fp64", coarsening="auto",
                 coarsest_steps=1, inner_cycles=1, max_workspace_bytes=0, smoother="exact", nu_x=2,
                 omega_x=2.0 / 3.0, gamma=1, transform="auto"):
    """st_options from keyword arguments (the defaults of st_default_options).
    transform: "auto" (tensor cores for 64 <= n + 1 <= 256, else FFTs), "fft" or "tensor"."""
    opt = StOptions()
    lib().st_default_options(ctypes.byref(opt))
    opt.nu1, opt.nu2, opt.omega, opt.rtol, opt.maxit = nu1, nu2, omega, rtol, maxit
    opt.precision = _PRECISION[precision]
    opt.coarsening = _COARSEN[coarsening]
    opt.coarsest_steps = coarsest_steps
    opt.inner_cycles = inner_cycles
    opt.max_workspace_bytes = max_workspace_bytes
    opt.smoother = {"exact": ST_SMOOTH_EXACT, "vcycle": ST_SMOOTH_VCYCLE}[smoother]
    opt.nu_x = nu_x
    opt.omega_x = omega_x
    opt.gamma = gamma
    opt.transform = _TRANSFORM[transform]
    return opt


def plan(dim, n, p_t, N, T, **options):
    """The hierarchy st_setup would build (st_plan, host only): (levels, mu_star),
    levels coarsest first as dicts N, n, mu, full (as Solver.level_info)."""
    L = lib()
    opt = make_options(**options)
    mesh = StMesh(dim, n)
    nlev = ctypes.c_int()
    ms = ctypes.c_double()
    rc = L.st_plan(ctypes.byref(mesh), p_t, N, float(T), ctypes.byref(opt), 0, None, None, None, None,
                   ctypes.byref(nlev), ctypes.byref(ms))
    if rc != ST_OK:
        raise StmgError(rc, "st_plan: invalid arguments")
    k = nlev.value
    Ns, ns, fs = (ctypes.c_int * k)(), (ctypes.c_int * k)(), (ctypes.c_int * k)()
    mus = (ctypes.c_double * k)()
    rc = L.st_plan(ctypes.byref(mesh), p_t, N, float(T), ctypes.byref(opt), k, Ns, ns, mus, fs, None, None)
    if rc != ST_OK:
        raise StmgError(rc, "st_plan failed")
    return [{"N": Ns[i], "n": ns[i], "mu": mus[i], "full": fs[i]} for i in range(k)], ms.value


class Solver:
    """A space-time hierarchy (st_setup) bound to the current CUDA stream."""

    def __init__(self, dim, n, p_t, N, T, *, nu1=2, nu2=2, omega=0.5, rtol=1e-8, maxit=50,
                 precision="fp64", coarsening="auto", coarsest_steps=1, inner_cycles=1,
                 max_workspace_bytes=0, smoother="exact", nu_x=2, omega_x=2.0 / 3.0, gamma=1, transform="auto",
                 stream=None, device=None):
        L = lib()
        self._lib = L
        self.dim, self.n, self.p_t, self.N, self.T = dim, n, p_t, N, float(T)
        self.q = p_t + 1
        opt = make_options(nu1=nu1, nu2=nu2, omega=omega, rtol=rtol, maxit=maxit, precision=precision,
                           coarsening=coarsening, coarsest_steps=coarsest_steps, inner_cycles=inner_cycles,
                           max_workspace_bytes=max_workspace_bytes, smoother=smoother, nu_x=nu_x,
                           omega_x=omega_x, gamma=gamma, transform=transform)
        self.options = opt
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        mesh = StMesh(dim, n)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = L.st_setup(ctypes.byref(mesh), p_t, N, float(T), ctypes.byref(opt),
                            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != ST_OK:
            raise StmgError(rc, "st_setup failed (see stderr)")
        self._h = h
        self.ndof = int(L.st_ndof(h))
        self.shape = (N, self.q) + (n,) * dim

    def close(self):
        if getattr(self, "_h", None):
            self._lib.st_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != ST_OK and rc not in allow:
            raise StmgError(rc, self._lib.st_last_error(self._h).decode())
        return rc

    # ------------------------------------------------------------ hierarchy
    @property
    def num_levels(self):
        return int(self._lib.st_num_levels(self._h))

    def level_info(self, L):
        Nl, nl, mu, full = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        self._check(self._lib.st_level_info(self._h, L, ctypes.byref(Nl), ctypes.byref(nl),
                                            ctypes.byref(mu), ctypes.byref(full)))
        return {"N": Nl.value, "n": nl.value, "mu": mu.value, "full": full.value}

    def level_shape(self, L):
        i = self.level_info(L)
        return (i["N"], self.q) + (i["n"],) * self.dim

    def level_ndof(self, L):
        i = self.level_info(L)
        return i["N"] * self.q * i["n"] ** self.dim

    def empty(self, L=None):
        shp = self.shape if L is None else self.level_shape(L)
        return torch.empty(shp, dtype=torch.float64, device=self.device)

    # ------------------------------------------------------------ full solver
    def residual(self, f, u, u0=None, out=None):
        out = self.empty() if out is None else out
        nx = self.n ** self.dim
        self._check(self._lib.st_residual(self._h, _ptr(f, self.ndof, "f"), _ptr(u0, nx, "u0"),
                                          _ptr(u, self.ndof, "u"), _ptr(out, self.ndof, "r")))
        return out

    def vcycle(self, u, f, u0=None):
        nx = self.n ** self.dim
        self._check(self._lib.st_vcycle(self._h, _ptr(u, self.ndof, "u"), _ptr(f, self.ndof, "f"),
                                        _ptr(u0, nx, "u0")))
        return u

    def solve(self, f, u0=None, u=None, initial_guess=None, raise_on_failure=True):
        """Solve L u = f + IC(u0).  ``u`` is the output buffer (allocated if None);
        it is used as the initial iterate when ``initial_guess`` is true (default:
        true exactly when ``u`` is given).  Returns (u, iterations, relative residual)."""
        init = (u is not None) if initial_guess is None else bool(initial_guess)
        u = self.empty() if u is None else u
        nx = self.n ** self.dim
        it, rr = ctypes.c_int(), ctypes.c_double()
        rc = self._lib.st_solve(self._h, _ptr(f, self.ndof, "f"), _ptr(u0, nx, "u0"), _ptr(u, self.ndof, "u"),
                                ST_INIT_GIVEN if init else 0, ctypes.byref(it), ctypes.byref(rr))
        self._check(rc, allow=() if raise_on_failure else (ST_ENOTCONV, ST_ENAN))
        self.last_status = rc
        return u, it.value, rr.value

    def solve_host(self, f, u0=None, u=None, initial_guess=False, raise_on_failure=True):
        """st_solve with host (CPU) tensors.  For pinned tensors the library's first
        sine-transform pass reads f from host memory and its last inverse pass writes
        the solution into ``u`` (a CPU tensor, allocated pinned if None); other host
        memory is copied.  Returns (u, iterations, relative residual)."""
        if u is None:
            u = torch.empty(self.shape, dtype=torch.float64).pin_memory()
        nx = self.n ** self.dim
        for name, t, cnt in (("f", f, self.ndof), ("u", u, self.ndof), ("u0", u0, nx)):
            if t is None:
                continue
            if t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != cnt:
                raise ValueError(f"{name}: need a contiguous float64 CPU tensor with {cnt} elements")
        it, rr = ctypes.c_int(), ctypes.c_double()
        rc = self._lib.st_solve_host(self._h, ctypes.c_void_p(f.data_ptr()),
                                     ctypes.c_void_p(u0.data_ptr()) if u0 is not None else None,
                                     ctypes.c_void_p(u.data_ptr()), ST_INIT_GIVEN if initial_guess else 0,
                                     ctypes.byref(it), ctypes.byref(rr))
        self._check(rc, allow=() if raise_on_failure else (ST_ENOTCONV, ST_ENAN))
        self.last_status = rc
        return u, it.value, rr.value

    def adjoint_solve(self, g, lam=None, raise_on_failure=True):
        """Solve L^T lam = g.  Returns (lam, grad_u0, iterations, relative residual)."""
        lam = self.empty() if lam is None else lam
        gu0 = torch.empty((self.n,) * self.dim, dtype=torch.float64, device=self.device)
        it, rr = ctypes.c_int(), ctypes.c_double()
        rc = self._lib.st_adjoint_solve(self._h, _ptr(g, self.ndof, "g"), _ptr(lam, self.ndof, "lambda"),
                                        _ptr(gu0, gu0.numel(), "grad_u0"), ctypes.byref(it), ctypes.byref(rr))
        self._check(rc, allow=() if raise_on_failure else (ST_ENOTCONV, ST_ENAN))
        self.last_status = rc
        return lam, gu0, it.value, rr.value

    def transform(self, x, L=None, inverse=False, out=None):
        """st_transform: the sine basis change S (or S^-1) of the spatial fields in x (FP64, any
        leading shape, n_L^d values per field) on level L (default finest); out may be x."""
        lv = self.num_levels - 1 if L is None else L
        nL = self.level_info(lv)["n"]
        nx = nL ** self.dim
        if x.numel() % nx:
            raise ValueError(f"x has {x.numel()} elements, not a multiple of n_L^d = {nx}")
        if out is None:
            out = torch.empty_like(x)
        self._check(self._lib.st_transform(self._h, lv, 1 if inverse else 0, _ptr(x, x.numel(), "x"),
                                           _ptr(out, x.numel(), "out"), x.numel() // nx))
        return out

    def norm2(self, x):
        out = ctypes.c_double()
        self._check(self._lib.st_norm2(self._h, _ptr(x, None, "x"), x.numel(), ctypes.byref(out)))
        return out.value

    # ------------------------------------------------------------ kernel timing
    def profile_start(self, max_launches=100000):
        self._check(self._lib.st_profile_start(self._h, max_launches))

    def profile_stop(self):
        """{class: dict(launches, ms, bytes, flops)} from CUDA events on the
        solver's stream; bytes / flops are the algorithmic work of those launches."""
        n = len(KERNEL_CLASSES)
        launches = (ctypes.c_int * n)()
        ms = (ctypes.c_double * n)()
        by = (ctypes.c_double * n)()
        fl = (ctypes.c_double * n)()
        dropped = ctypes.c_int()
        self._check(self._lib.st_profile_stop(self._h, launches, ms, by, fl, ctypes.byref(dropped)))
        out = {k: {"launches": launches[i], "ms": ms[i], "bytes": by[i], "flops": fl[i]}
               for i, k in enumerate(KERNEL_CLASSES)}
        out["_dropped"] = dropped.value
        return out

    def profile_level(self, kernel_class, L):
        """dict(launches, ms, bytes, flops) of one kernel class on level L (after profile_stop)."""
        i = KERNEL_CLASSES.index(kernel_class)
        launches, ms, by, fl = ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.st_profile_level(self._h, i, L, ctypes.byref(launches), ctypes.byref(ms),
                                               ctypes.byref(by), ctypes.byref(fl)))
        return {"launches": launches.value, "ms": ms.value, "bytes": by.value, "flops": fl.value}

    # ------------------------------------------------------------ step level
    def level_residual(self, L, f, u, adjoint=False, out=None):
        m = self.level_ndof(L)
        out = self.empty(L) if out is None else out
        self._check(self._lib.st_level_residual(self._h, L, int(adjoint), _ptr(f, m, "f"), _ptr(u, m, "u"),
                                                _ptr(out, m, "r")))
        return out

    def level_block_solve(self, L, r, adjoint=False, out=None):
        m = self.level_ndof(L)
        out = self.empty(L) if out is None else out
        self._check(self._lib.st_level_block_solve(self._h, L, int(adjoint), _ptr(r, m, "r"), _ptr(out, m, "d")))
        return out

    def level_smooth(self, L, f, u, nu=1, adjoint=False):
        m = self.level_ndof(L)
        self._check(self._lib.st_level_smooth(self._h, L, int(adjoint), nu, _ptr(f, m, "f"), _ptr(u, m, "u")))
        return u

    def level_restrict(self, L, r, out=None):
        out = self.empty(L - 1) if out is None else out
        self._check(self._lib.st_level_restrict(self._h, L, _ptr(r, self.level_ndof(L), "r"),
                                                _ptr(out, self.level_ndof(L - 1), "f_coarse")))
        return out

    def level_prolong(self, L, e, u):
        self._check(self._lib.st_level_prolong(self._h, L, _ptr(e, self.level_ndof(L - 1), "e"),
                                               _ptr(u, self.level_ndof(L), "u")))
        return u

    def coarsest_solve(self, f, adjoint=False, out=None):
        out = self.empty(0) if out is None else out
        m = self.level_ndof(0)
        self._check(self._lib.st_coarsest_solve(self._h, int(adjoint), _ptr(f, m, "f"), _ptr(out, m, "u")))
        return out


class MeshSolver:
    """The space-time hierarchy on a uniformly refined simplicial mesh of the unit
    square / cube (stm_setup, include/stmg_mesh.h), bound to the current CUDA
    stream.  verts: (nverts, dim) coordinates, cells: (ncells, dim + 1) vertex
    indices of the initial mesh.  Vectors: torch.float64 CUDA tensors with
    N q Nx elements in the layout (N, q, Nx), Nx interior vertices ordered by
    (z, y, x) (``nodes()``)."""

    def __init__(self, verts, cells, refinements, p_t, N, T, *, nu1=2, nu2=2, omega=0.5, rtol=1e-8, maxit=50,
                 coarsening="auto", max_workspace_bytes=0, nu_x=2, omega_x=2.0 / 3.0, gamma=1, precision="fp64",
                 inner_cycles=1, stream=None, device=None):
        import numpy as np
        L = lib()
        self._lib = L
        v = np.ascontiguousarray(verts, dtype=np.float64)
        c = np.ascontiguousarray(cells, dtype=np.int32)
        self.dim, self.p_t, self.N, self.T = v.shape[1], p_t, N, float(T)
        self.q = p_t + 1
        self.refinements = refinements
        opt = make_options(nu1=nu1, nu2=nu2, omega=omega, rtol=rtol, maxit=maxit, precision=precision,
                           coarsening=coarsening, coarsest_steps=1, inner_cycles=inner_cycles,
                           max_workspace_bytes=max_workspace_bytes, smoother="vcycle", nu_x=nu_x, omega_x=omega_x,
                           gamma=gamma)
        self.options = opt
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        mesh = SimplexMesh(self.dim, v.shape[0], v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), c.shape[0],
                           c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = L.stm_setup(ctypes.byref(mesh), refinements, p_t, N, float(T), ctypes.byref(opt),
                             ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != ST_OK:
            raise StmgError(rc, "stm_setup failed")
        self._h = h
        self.ndof = int(L.stm_ndof(h))
        self.Nx = self.ndof // (N * self.q)
        self.shape = (N, self.q, self.Nx)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.stm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != ST_OK and rc not in allow:
            raise StmgError(rc, self._lib.stm_last_error(self._h).decode())
        return rc

    def nodes(self, space_level=None):
        """(Nx, dim) coordinates of the interior vertices of a refinement level
        (default: the finest) in the unknowns' order."""
        import numpy as np
        lvl = self.refinements if space_level is None else space_level
        cnt = ctypes.c_int()
        self._check(self._lib.stm_nodes(self._h, lvl, ctypes.byref(cnt), None))
        out = np.zeros((cnt.value, self.dim))
        self._check(self._lib.stm_nodes(self._h, lvl, None, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    @property
    def num_levels(self):
        return int(self._lib.stm_num_levels(self._h))

    def level_info(self, L):
        Nl, sl, mu, full = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        self._check(self._lib.stm_level_info(self._h, L, ctypes.byref(Nl), ctypes.byref(sl), ctypes.byref(mu),
                                             ctypes.byref(full)))
        return {"N": Nl.value, "space_level": sl.value, "mu": mu.value, "full": full.value}

    def level_shape(self, L):
        i = self.level_info(L)
        cnt = ctypes.c_int()
        self._check(self._lib.stm_nodes(self._h, i["space_level"], ctypes.byref(cnt), None))
        return (i["N"], self.q, cnt.value)

    def level_ndof(self, L):
        a, b, c = self.level_shape(L)
        return a * b * c

    def empty(self, L=None):
        shp = self.shape if L is None else self.level_shape(L)
        return torch.empty(shp, dtype=torch.float64, device=self.device)

    def residual(self, f, u, u0=None, out=None):
        out = self.empty() if out is None else out
        self._check(self._lib.stm_residual(self._h, _ptr(f, self.ndof, "f"), _ptr(u0, self.Nx, "u0"),
                                           _ptr(u, self.ndof, "u"), _ptr(out, self.ndof, "r")))
        return out

    def vcycle(self, u, f, u0=None):
        self._check(self._lib.stm_vcycle(self._h, _ptr(u, self.ndof, "u"), _ptr(f, self.ndof, "f"),
                                         _ptr(u0, self.Nx, "u0")))
        return u

    def solve(self, f, u0=None, u=None, initial_guess=None, raise_on_failure=True):
        init = (u is not None) if initial_guess is None else bool(initial_guess)
        u = self.empty() if u is None else u
        it, rr = ctypes.c_int(), ctypes.c_double()
        rc = self._lib.stm_solve(self._h, _ptr(f, self.ndof, "f"), _ptr(u0, self.Nx, "u0"), _ptr(u, self.ndof, "u"),
                                 ST_INIT_GIVEN if init else 0, ctypes.byref(it), ctypes.byref(rr))
        self._check(rc, allow=() if raise_on_failure else (ST_ENOTCONV, ST_ENAN))
        self.last_status = rc
        return u, it.value, rr.value

    def adjoint_solve(self, g, lam=None, raise_on_failure=True):
        lam = self.empty() if lam is None else lam
        gu0 = torch.empty(self.Nx, dtype=torch.float64, device=self.device)
        it, rr = ctypes.c_int(), ctypes.c_double()
        rc = self._lib.stm_adjoint_solve(self._h, _ptr(g, self.ndof, "g"), _ptr(lam, self.ndof, "lambda"),
                                         _ptr(gu0, self.Nx, "grad_u0"), ctypes.byref(it), ctypes.byref(rr))
        self._check(rc, allow=() if raise_on_failure else (ST_ENOTCONV, ST_ENAN))
        self.last_status = rc
        return lam, gu0, it.value, rr.value

    def level_residual(self, L, f, u, adjoint=False, out=None):
        m = self.level_ndof(L)
        out = self.empty(L) if out is None else out
        self._check(self._lib.stm_level_residual(self._h, L, int(adjoint), _ptr(f, m, "f"), _ptr(u, m, "u"),
                                                 _ptr(out, m, "r")))
        return out

    def level_block_solve(self, L, r, adjoint=False, out=None):
        m = self.level_ndof(L)
        out = self.empty(L) if out is None else out
        self._check(self._lib.stm_level_block_solve(self._h, L, int(adjoint), _ptr(r, m, "r"), _ptr(out, m, "d")))
        return out

    def level_smooth(self, L, f, u, nu=1, adjoint=False):
        m = self.level_ndof(L)
        self._check(self._lib.stm_level_smooth(self._h, L, int(adjoint), nu, _ptr(f, m, "f"), _ptr(u, m, "u")))
        return u

    def level_restrict(self, L, r, out=None):
        out = self.empty(L - 1) if out is None else out
        self._check(self._lib.stm_level_restrict(self._h, L, _ptr(r, self.level_ndof(L), "r"),
                                                 _ptr(out, self.level_ndof(L - 1), "f_coarse")))
        return out

    def level_prolong(self, L, e, u):
        self._check(self._lib.stm_level_prolong(self._h, L, _ptr(e, self.level_ndof(L - 1), "e"),
                                                _ptr(u, self.level_ndof(L), "u")))
        return u

    def coarsest_solve(self, f, adjoint=False, out=None):
        out = self.empty(0) if out is None else out
        m = self.level_ndof(0)
        self._check(self._lib.stm_coarsest_solve(self._h, int(adjoint), _ptr(f, m, "f"), _ptr(out, m, "u")))
        return out


def norm2_noalloc(x, out=None, stream=None):
    """||x||_2 into a one-element device tensor without any device allocation by
    the library (st_norm2_noalloc); ``out`` must be given by callers that
    cannot allocate either."""
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=x.device)
    stream = torch.cuda.current_stream(x.device) if stream is None else stream
    rc = lib().st_norm2_noalloc(_ptr(x, None, "x"), x.numel(), _ptr(out, 1, "out"),
                                ctypes.c_void_p(stream.cuda_stream))
    if rc != ST_OK:
        raise StmgError(rc, "st_norm2_noalloc failed")
    return out


class SpaceTimeSolve(torch.autograd.Function):
    """u = L^{-1}(f + IC(u0)) with gradients from the adjoint solve:
    dJ/df = lambda, dJ/du0 = M_h sum_k psi_k(t_0^+) lambda_{1,k}, L^T lambda = dJ/du."""

    @staticmethod
    def forward(ctx, f, u0, solver):
        ctx.solver = solver
        u, it, rr = solver.solve(f.contiguous(), u0.contiguous())
        return u

    @staticmethod
    def backward(ctx, grad_u):
        lam, gu0, it, rr = ctx.solver.adjoint_solve(grad_u.contiguous())
        return lam, gu0, None


def solve(f, u0, solver):
    """Differentiable solve of the heat equation's space-time system."""
    return SpaceTimeSolve.apply(f, u0, solver)
