/*
 * stmg -- space-time multigrid for the heat equation on one GPU.
 *
 * Method: Gander & Neumueller, "Analysis of a new space-time parallel
 * multigrid algorithm for parabolic problems" (arXiv:1411.0519).
 *
 * Problem (Section 1, eq. (chap4_modelproblem)): du/dt - Laplace u = f on
 * (0,1)^d x (0,T), d = 1, 2, 3, u = 0 on the boundary, u(.,0) = u0.  Space:
 * P1 (d = 1) / Q1 (d = 2, 3) finite elements on a uniform grid with n = 2^k - 1
 * interior nodes per axis, h = 1/(n+1).  Time: N = 2^m uniform slabs,
 * tau = T/N, discontinuous Galerkin of degree p_t in the Legendre basis
 * psi_k(t) = P_k(2 (t - t_{n-1}) / tau - 1), q = p_t + 1 dofs per slab.
 * The discrete system (chap4_generalLinearSystem) is block lower-bidiagonal:
 *
 *     A u_1 = f_1,  B u_{n-1} + A u_n = f_n,
 *     A = K_tau (x) M_h + M_tau (x) K_h,   B = -N_tau (x) M_h.
 *
 * Vector layout (every pointer below that holds a space-time vector):
 * contiguous FP64, index ((s * q + l) * n^d + j) for time step s = 0..N-1,
 * time dof l = 0..q-1, spatial node j = (z * n + y) * n + x (x fastest).
 * A spatial field (u0_ic, grad_u0) is n^d contiguous FP64 in the same node
 * order.  All vector pointers are DEVICE pointers owned by the caller and
 * must not alias each other unless stated.  Calls are asynchronous on the
 * stream given to st_setup except where a host result is returned (norms,
 * iteration counts), which synchronises that stream.
 *
 * Levels are numbered as in the paper (Section 2): L = 0 is the coarsest
 * (one time step by default), L = st_num_levels() - 1 the finest.
 *
 * Errors: every int-returning call returns ST_OK (0) or one of the ST_E*
 * codes; nothing throws across this interface.  st_last_error() returns a
 * message for the last failure on that handle.  ST_ECUDA leaves the handle
 * usable only for st_destroy.
 */
#ifndef STMG_H
#define STMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ST_OK        0
#define ST_EINVAL    1   /* bad argument: n != 2^k-1, N not a power of 2, p_t out of range, T <= 0, null pointer */
#define ST_ENOMEM    2   /* device allocation failed or exceeds st_options.max_workspace_bytes */
#define ST_ENOTCONV  3   /* maxit reached before rtol, or the residual grew by 1e6 */
#define ST_ENAN      4   /* a residual norm was NaN or Inf */
#define ST_ECUDA     5   /* a CUDA runtime call failed */

#define ST_FP64      0   /* every kernel in FP64 */
#define ST_MIXED     1   /* FP64 outer residual / update / coarsest solve, FP32 V-cycle */

#define ST_AUTO      0   /* the paper's rule (Section 4): full iff mu_L >= mu*_{p_t} */
#define ST_SEMI      1   /* always semi-coarsen in time */
#define ST_FULL      2   /* full space-time coarsening whenever n_L >= 3 */

#define ST_INIT_GIVEN 1  /* st_solve flag: u holds the initial iterate (else u^0 = 0) */

#define ST_SMOOTH_EXACT  0  /* block inverse D^{-1} exact (Section 3.1): one q x q inverse per sine mode */
#define ST_SMOOTH_VCYCLE 1  /* D~^{-1}: one spatial multigrid V-cycle per step (Remark on the V-cycle
                               approximation in space; damped point-block Jacobi, nu_x, omega_x) */

#define ST_DST_AUTO   0  /* sine transforms on the tensor cores where 64 <= n_L + 1 <= 256, else the FFT kernels
                             (FP64, or double-float on the FP32 pipe in the mixed form) */
#define ST_DST_FFT    1  /* FFT-based sine transforms at every length (FP64; double-float in the mixed form) */
#define ST_DST_TENSOR 2  /* tensor-core sine transforms; st_setup fails (ST_EINVAL) unless 64 <= n + 1 <= 256 */

#define ST_MAX_PT    47  /* largest supported DG degree p_t (q <= 48); degrees above 3 use the
                             generic-q kernels and need ST_SMOOTH_EXACT */

typedef struct st_mesh {
  int dim;  /* 1, 2 or 3 */
  int n;    /* interior nodes per axis, 2^k - 1, k >= 1; n <= 1023 with the exact block
               inverse (the sine transform of a line is held in shared memory) */
} st_mesh;

typedef struct st_options {
  int nu1, nu2;          /* pre-/post-smoothing steps (Section 2), default 2, 2 */
  double omega;          /* block-Jacobi damping omega_t (eq. chap4_smoother), default 1/2 (Lemma 21) */
  double rtol;           /* stop when ||r_k|| <= rtol ||r_0|| (Section 2), default 1e-8 */
  int maxit;             /* maximum V-cycles / refinement steps, default 50 */
  int precision;         /* ST_FP64 or ST_MIXED */
  int coarsening;        /* ST_AUTO, ST_SEMI or ST_FULL */
  int coarsest_steps;    /* time steps on the coarsest level, power of 2, default 1 (Section 2) */
  int inner_cycles;      /* ST_MIXED: FP32 V-cycles per FP64 refinement step, default 1 */
  size_t max_workspace_bytes;  /* 0 = unlimited; setup fails with ST_ENOMEM above it */
  int smoother;          /* ST_SMOOTH_EXACT (default) or ST_SMOOTH_VCYCLE */
  int nu_x;              /* ST_SMOOTH_VCYCLE: spatial pre-/post-smoothing steps, default 2 (Section 4) */
  double omega_x;        /* ST_SMOOTH_VCYCLE: spatial Jacobi damping, default 2/3 (Section 4) */
  int gamma;             /* cycle index (Section 2): 1 = V-cycle (default), 2 = W-cycle */
  int transform;         /* ST_DST_AUTO (default), ST_DST_FFT or ST_DST_TENSOR: how the FP64 sine
                            transforms of the exact block inverse (Section 3.1) are computed.  The
                            tensor-core form splits each line into 7-bit digits scaled by the line's
                            largest exponent and sums exact FP16 digit products in FP32 tensor memory;
                            its error is below 2^-50 of sqrt((n+1)/2) ||line||_2, like the FFT's.  It
                            needs a scratch of max(131072, n^(d-1)) (n+1) 16 bytes (at most 537 MB),
                            allocated on first use and counted in max_workspace_bytes. */
} st_options;

typedef struct st_handle st_handle;

/* Fill *opt with the defaults listed above. */
void st_default_options(st_options* opt);

/* Build the space-time hierarchy for the problem of Section 1 and allocate
 * its device workspace.  Coarsening follows Section 4 (mu_L = tau_L / h_L^2
 * against mu* of Remark chap4_remarkCriticalDiscretizationParameter) until
 * N_L = coarsest_steps.  N is a power of 2 up to 32768.  cuda_stream: a cudaStream_t (NULL = default stream)
 * used by every later call on this handle.  On success *out owns the handle.
 * Errors: ST_EINVAL, ST_ENOMEM, ST_ECUDA. */
int st_setup(const st_mesh* mesh, int p_t, int N, double T, const st_options* opt,
             void* cuda_stream, st_handle** out);

/* Free the handle and its device workspace (NULL is ignored). */
void st_destroy(st_handle* h);

/* Message of the last error on this handle ("" if none; static text for NULL). */
const char* st_last_error(const st_handle* h);

/* Number of unknowns N q n^d of the finest level. */
size_t st_ndof(const st_handle* h);

int st_num_levels(const st_handle* h);

/* The coarsening plan st_setup would build, computed on the host only (no
 * device, no handle): the hierarchy of Section 2 with the rule of Section 4
 * (mu_L = tau_L / h_L^2 against mu* of Remark
 * chap4_remarkCriticalDiscretizationParameter, full coarsening when
 * mu_L >= mu* and n_L >= 3 under ST_AUTO) down to coarsest_steps steps.
 * Arrays hold max_levels entries, level 0 = coarsest, with the meaning of
 * st_level_info; any of them, nlev and mu_star may be NULL.  *nlev receives
 * the number of levels, *mu_star the critical value for p_t.
 * Errors: ST_EINVAL for the argument checks of st_setup, or when an array is
 * given and max_levels is below the number of levels (nlev is still set). */
int st_plan(const st_mesh* mesh, int p_t, int N, double T, const st_options* opt, int max_levels,
            int* N_L, int* n_L, double* mu_L, int* full, int* nlev, double* mu_star);

/* Level L (0 = coarsest): time steps, nodes per axis, mu_L = tau_L/h_L^2 and
 * whether level L was obtained from L+1 by full coarsening (1), semi (0), or
 * is the finest (-1).  Any output pointer may be NULL.  Errors: ST_EINVAL. */
int st_level_info(const st_handle* h, int L, int* N_L, int* n_L, double* mu_L, int* full);

/* r = f + IC - L u on the finest level (system chap4_generalLinearSystem),
 * where IC adds psi_k(t_0^+) (M_h u0_ic) to block 1 (the n = 0 term of eq.
 * (equation1)); u0_ic may be NULL (zero initial value).  r may not alias u.
 * Computed on nodes with the stencils of M_h and K_h at every p_t, by kernels
 * that share nothing with the sine-basis cycle (an independent check of a
 * solve's residual). */
int st_residual(st_handle* h, const double* f, const double* u0_ic, const double* u, double* r);

/* One V-cycle (gamma = 1, Section 2) on L u = f + IC for the finest level, in
 * place on u.  With ST_MIXED this is one refinement step: FP64 residual,
 * inner_cycles FP32 V-cycles on the scaled residual, FP64 update.
 * The cycle runs in the basis that diagonalises the spatial matrices along
 * every axis (sine transform, Section 3.1): f, u0_ic and u are transformed on
 * entry and u is transformed back; the iterates are the same as on nodes up to
 * rounding. */
int st_vcycle(st_handle* h, double* u, const double* f, const double* u0_ic);

/* Solve L u = f + IC to ||r|| <= rtol ||r_0|| by repeated V-cycles (Section 2).
 * flags: ST_INIT_GIVEN to start from the given u, else u^0 = 0.  *iters gets
 * the number of cycles, *relres ||r|| / ||r_0|| (either may be NULL).
 * Returns ST_ENOTCONV / ST_ENAN (u then holds the last iterate). */
int st_solve(st_handle* h, const double* f, const double* u0_ic, double* u, int flags,
             int* iters, double* relres);

/* st_solve with HOST buffers f, u0_ic (may be NULL) and u (all N q n^d values,
 * n^d for u0_ic), on the handle's stream; returns when u is in host memory.
 * When f and u are page-locked memory registered with CUDA (e.g. from
 * cudaHostAlloc), the exact block inverse is used and 64 <= n + 1 <= 512, the
 * first sine-transform pass reads f from host memory and the last inverse pass
 * writes u to it over the CPU-GPU interconnect, so no separate copies are
 * made; otherwise the buffers are copied.  A device buffer for u is allocated
 * on the first call and kept by the handle.
 * Errors: as st_solve, and ST_ENOMEM if that buffer cannot be allocated. */
int st_solve_host(st_handle* h, const double* f, const double* u0_ic, double* u, int flags,
                  int* iters, double* relres);

/* Adjoint solve L^T lambda = g (transposed, backward-in-time system) with the
 * same hierarchy and transfers.  grad_u0 (may be NULL) receives
 * M_h sum_k psi_k(t_0^+) lambda_{1,k}, the derivative of a loss with
 * dJ/du = g with respect to u0_ic; lambda itself is dJ/df. */
int st_adjoint_solve(st_handle* h, const double* g, double* lambda, double* grad_u0,
                     int* iters, double* relres);

/* ---- step-level entry points (one step of the cycle on one level) ----
 * adjoint != 0 selects the transposed operator.  Vectors have the level's
 * layout (N_L, q, n_L^d), on nodes.  With ST_SMOOTH_EXACT each call
 * transforms its inputs to the basis of the cycle, runs the same kernels as
 * st_solve and transforms the result back; it uses the level's internal
 * buffers as scratch (calls on one handle must not overlap). */

/* r = f - L_L u (no IC term) or f - L_L^T u. */
int st_level_residual(st_handle* h, int L, int adjoint, const double* f, const double* u, double* r);

/* d = D_L^{-1} r in FP64: the smoother's block inverse -- exact (Section 3.1)
 * with ST_SMOOTH_EXACT, one spatial V-cycle per step with ST_SMOOTH_VCYCLE. */
int st_level_block_solve(st_handle* h, int L, int adjoint, const double* r, double* d);

/* nu damped block-Jacobi steps u <- u + omega D^{-1}(f - L u) (eq. chap4_smoother). */
int st_level_smooth(st_handle* h, int L, int adjoint, int nu, const double* f, double* u);

/* f_c = R r: level L (L >= 1) to level L-1, eqs. (chap4_restrictionTime),
 * (chap4_spaceRestrictionProlongation); semi or full as the hierarchy says. */
int st_level_restrict(st_handle* h, int L, const double* r_fine, double* f_coarse);

/* u_fine += P e_c, P = R^T, level L-1 to level L. */
int st_level_prolong(st_handle* h, int L, const double* e_coarse, double* u_fine);

/* Exact solve on the coarsest level (Section 2): one step via the block
 * inverse, several by forward (adjoint: backward) substitution. */
int st_coarsest_solve(st_handle* h, int adjoint, const double* f, double* u);

/* Change of basis of `slabs` consecutive FP64 spatial fields of level L
 * (layout (slabs, n_L^d)): y = S x, S the unnormalised DST-I
 * y_k = sum_j x_j sin(pi j k / (n_L + 1)) along every axis (inverse = 0), or
 * y = S^{-1} x = (2 / (n_L + 1))^d S x (inverse = 1).  In the sine basis the
 * spatial operators of every step are diagonal (Section 3.1).  x == y is allowed;
 * other overlap is not.  Uses the handle's transform option; synchronises and
 * reports a pending tensor-core time-out.  Errors: ST_EINVAL, ST_ECUDA. */
int st_transform(st_handle* h, int L, int inverse, const double* x, double* y, size_t slabs);

/* ||x||_2 of n FP64 values (deterministic order); synchronises. */
int st_norm2(st_handle* h, const double* x, size_t n, double* out);

/* ---- kernel timing (CUDA events on the handle's stream) ----
 * Kernel classes for st_profile_stop: */
#define ST_K_RESIDUAL   0   /* residual (forward / transposed); for q <= 4 the finest-level
                               residual of the stopping test with its norm in one pass */
#define ST_K_DST        1   /* batched sine transform along one axis */
#define ST_K_SMOOTH     2   /* damped smoothing step (coupling term, q x q block inverse
                               per sine mode, damping) and the coarsest substitution; in
                               FP32 cycles also the first post-smoothing step with the
                               coarse-grid correction */
#define ST_K_RESTRICT   3
#define ST_K_PROLONG    4
#define ST_K_NORM       5   /* both reduction stages of a separate norm */
#define ST_K_VECTOR     6   /* axpy, casts, copies, memsets */
#define ST_K_RHS        7   /* separate smoother right-hand side (no longer launched:
                               fused into ST_K_SMOOTH; the value is kept) */
#define ST_K_SPACEMG    8   /* spatial V-cycle of the inexact block inverse */
#define ST_K_DSTTC      9   /* tensor-core pass of a sine transform along one axis (ST_K_DST then holds
                               its digit-splitting pass); flops = the FP16 digit products executed */
#define ST_K_COUNT      10

/* Record a CUDA event pair around every kernel launched by this handle, for up
 * to max_launches launches (events are created here, not per launch).  Adds a
 * few microseconds of host time per launch.  Errors: ST_EINVAL, ST_ECUDA. */
int st_profile_start(st_handle* h, int max_launches);

/* Synchronise the stream, stop recording and return per class (arrays of
 * ST_K_COUNT entries, any may be NULL) the number of launches, their summed
 * device time in milliseconds, and their algorithmic HBM bytes and
 * floating-point operations (the minimum the computation needs: each input
 * read once, each output written once; formulas in the library source).
 * Launches beyond max_launches are counted but not timed (*dropped). */
int st_profile_stop(st_handle* h, int* launches, double* ms, double* bytes, double* flops, int* dropped);

/* After st_profile_stop: the same four totals for kernel class cls restricted
 * to the launches that worked on level L (0 = coarsest).  Classes without a
 * level (norms, vector operations) report zeros.  Errors: ST_EINVAL (bad
 * class or level, or no timed region recorded yet). */
int st_profile_level(const st_handle* h, int cls, int L, int* launches, double* ms, double* bytes, double* flops);

/* ---- allocation-free norm ----
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory -- an application whose allocator owns the GPU's
 * memory after start-up, or a code path that must not take the implicit
 * device synchronisation of cudaMalloc / cudaFree.  It needs no handle.
 *
 * *out (a DEVICE pointer to one double) = ||x||_2 of n FP64 values at the
 * device pointer x, asynchronously on cuda_stream (NULL = default stream).
 * The sum of squares is deterministic in its own fixed order (one FP64
 * partial per contiguous chunk of 65536 elements, then one block adds the
 * partials in a fixed order); st_norm2 adds in another fixed order, so the two
 * agree to rounding.  It calls no allocator: the partial sums live in a fixed
 * 128 KB device array inside this library, which every GPU that loads the
 * library holds until the process exits.
 *  - n must not exceed ST_NOALLOC_MAX_ELEMENTS (2^30); larger n returns
 *    ST_EINVAL before any device work.  x or out NULL: ST_EINVAL.
 *  - The array is shared by all calls; calls whose kernels can overlap on
 *    the GPU (different streams with no ordering) race on it and give wrong
 *    results.  Each call overwrites every partial it reads, so nothing has to
 *    be cleared between calls.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and caches it; make
 *    that first call before any stream capture.
 *  - A CUDA error already pending on the calling thread makes the call return
 *    ST_ECUDA without launching; the error is not cleared (it stays for the
 *    caller's own check), and the launches' own status is read without
 *    clearing it either.
 * Errors: ST_EINVAL, ST_ECUDA (pending error, address lookup or launch failed). */
#define ST_NOALLOC_MAX_ELEMENTS ((size_t)1 << 30)
int st_norm2_noalloc(const double* x, size_t n, double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* STMG_H */
