/*
 * stmg_mesh -- space-time multigrid for the heat equation on uniformly
 * refined simplicial meshes of the unit square / cube, on one GPU.
 *
 * Method: Gander & Neumueller, arXiv:1411.0519.  Section 4, Examples 1 and 2:
 * P1 conforming elements in space on an initial mesh of (0,1)^d (triangles,
 * d = 2, or tetrahedra, d = 3) refined uniformly `refinements` times, DG of
 * degree p_t in time (Legendre basis as in stmg.h), N uniform time steps on
 * (0, T), the system of Section 1 (chap4_generalLinearSystem):
 *
 *     A u_1 = f_1,  B u_{n-1} + A u_n = f_n,
 *     A = K_tau (x) M_h + M_tau (x) K_h,   B = -N_tau (x) M_h,
 *
 * solved by the space-time V-cycle of Section 2 with the damped block-Jacobi
 * smoother (eq. chap4_smoother) whose block inverse is the paper's practical
 * approximation (Remark on the V-cycle approximation in space, eq.
 * chap4_smootherApprox): one spatial multigrid V-cycle per time step on the
 * meshes of the refinement, damped point-block Jacobi with the q x q node
 * blocks D^x_j = (M_h)_jj K_tau + (K_h)_jj M_tau (nu_x, omega_x of
 * st_options), the nested-space prolongation of the refinement and its
 * transpose, and an exact solve on the initial mesh.  Coarsening (Section 4):
 * full space-time coarsening to the next coarser mesh iff mu_L = tau_L / h_L^2
 * >= mu*_{p_t} and a coarser mesh exists, otherwise semi coarsening in time,
 * down to one time step, which is solved exactly (spatial V-cycles repeated
 * to rounding).  h_L is the longest edge of the level's mesh.
 *
 * Uniform refinement: each edge is split at its midpoint; a triangle gives 4
 * triangles, a tetrahedron 8 (its 4 corner tetrahedra and the inner
 * octahedron cut along the diagonal between the midpoints of its edges 02
 * and 13, for the vertex order of the given cell).
 *
 * Unknowns: the vertices of the refined mesh that lie strictly inside the
 * unit cube (a vertex with a coordinate <= 0 or >= 1 is on the boundary,
 * homogeneous Dirichlet), ordered by their coordinates: z, then y, then x
 * (stm_nodes returns them).  A space-time vector is contiguous FP64, index
 * ((s * q + l) * Nx + j), time step s, time dof l, node j; a spatial field
 * (u0_ic, grad_u0) has Nx entries.  Vector pointers are DEVICE pointers owned
 * by the caller; calls are asynchronous on the handle's stream except where a
 * host result is returned.  Levels: L = 0 coarsest, stm_num_levels() - 1 finest.
 *
 * Precision: ST_FP64, or ST_MIXED: inner_cycles FP32 cycles (every kernel of
 * the cycle in FP32 with FP32 accumulation, the matrices and tables rounded to
 * FP32) on the FP64 residual scaled by its norm, inside FP64 iterative
 * refinement; the outer residual, the update and the coarsest solve stay FP64.
 * The step-level calls below always run in FP64.
 *
 * Limits: p_t <= 3; smoother ST_SMOOTH_VCYCLE (the exact block inverse of a
 * spatial mesh operator is not built); coarsest_steps = 1;
 * q times the interior vertices of the initial mesh at most 1024 (its exact
 * solve is a dense inverse formed at setup, one per space-time level).  Other options as in stmg.h (nu1, nu2,
 * omega, rtol, maxit, coarsening, nu_x, omega_x, gamma, max_workspace_bytes).
 * Errors: ST_OK or an ST_E* code of stmg.h; stm_last_error gives a message.
 */
#ifndef STMG_MESH_H
#define STMG_MESH_H

#include <stddef.h>

#include "stmg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct st_simplex_mesh {
  int dim;              /* 2: triangles, 3: tetrahedra */
  int nverts;           /* vertices of the initial mesh */
  const double* verts;  /* nverts x dim coordinates (host memory), inside [0, 1]^dim */
  int ncells;           /* simplices of the initial mesh */
  const int* cells;     /* ncells x (dim + 1) vertex indices (host memory), a conforming mesh of (0,1)^dim */
} st_simplex_mesh;

typedef struct stm_handle stm_handle;

/* Refine the initial mesh `refinements` times, assemble M_h and K_h of every
 * mesh (Section 1), build the space-time hierarchy (Sections 2, 4) and its
 * device workspace.  The mesh arrays are read during the call only.
 * Errors: ST_EINVAL (dim, counts, indices, p_t > 3, N not a power of 2,
 * T <= 0, unsupported options, too fine an initial mesh), ST_ENOMEM, ST_ECUDA. */
int stm_setup(const st_simplex_mesh* mesh0, int refinements, int p_t, int N, double T, const st_options* opt,
              void* cuda_stream, stm_handle** out);

void stm_destroy(stm_handle* h);
const char* stm_last_error(const stm_handle* h);

/* Unknowns N q Nx of the finest level. */
size_t stm_ndof(const stm_handle* h);

int stm_num_levels(const stm_handle* h);

/* Interior vertices of refinement level `space_level` (0 = the initial mesh,
 * refinements = the finest): their number, and (coords may be NULL) their
 * coordinates in the unknowns' order, Nx x dim values into host memory. */
int stm_nodes(const stm_handle* h, int space_level, int* count, double* coords);

/* Level L: time steps, refinement level of its mesh, mu_L = tau_L / h_L^2 and
 * whether it was obtained from L + 1 by full coarsening (1), semi (0), or is
 * the finest (-1).  Any output may be NULL. */
int stm_level_info(const stm_handle* h, int L, int* N_L, int* space_level, double* mu_L, int* full);

/* r = f + IC - L u on the finest level; IC adds psi_k(t_0^+) (M_h u0_ic) to
 * block 1 (eq. (equation1)); u0_ic may be NULL.  r may not alias u. */
int stm_residual(stm_handle* h, const double* f, const double* u0_ic, const double* u, double* r);

/* One cycle (Section 2, gamma of the options) on L u = f + IC, in place on u;
 * with ST_MIXED one refinement step (FP64 residual, inner_cycles FP32 cycles,
 * FP64 update). */
int stm_vcycle(stm_handle* h, double* u, const double* f, const double* u0_ic);

/* Cycles until ||r|| <= rtol ||r_0|| (Section 2).  flags: ST_INIT_GIVEN to
 * start from u, else u^0 = 0.  Returns ST_ENOTCONV / ST_ENAN as st_solve. */
int stm_solve(stm_handle* h, const double* f, const double* u0_ic, double* u, int flags, int* iters,
              double* relres);

/* L^T lambda = g (backward in time) with the same hierarchy; grad_u0 (may be
 * NULL) = M_h sum_k psi_k(t_0^+) lambda_{1,k}. */
int stm_adjoint_solve(stm_handle* h, const double* g, double* lambda, double* grad_u0, int* iters,
                      double* relres);

/* ---- one step of the cycle on level L (layout (N_L, q, Nx_L)); adjoint != 0
 * selects the transposed operator.  Calls on one handle must not overlap. */
int stm_level_residual(stm_handle* h, int L, int adjoint, const double* f, const double* u, double* r);
/* d = D~_L^{-1} r: one spatial V-cycle per time step (the smoother's block inverse). */
int stm_level_block_solve(stm_handle* h, int L, int adjoint, const double* r, double* d);
/* nu damped steps u <- u + omega D~^{-1} (f - L u) (eq. chap4_smoother). */
int stm_level_smooth(stm_handle* h, int L, int adjoint, int nu, const double* f, double* u);
/* f_c = R r (L >= 1): time blocks of eq. (chap4_restrictionTime) and, for full
 * coarsening, the transpose of the mesh prolongation. */
int stm_level_restrict(stm_handle* h, int L, const double* r_fine, double* f_coarse);
/* u_fine += R^T e_c. */
int stm_level_prolong(stm_handle* h, int L, const double* e_coarse, double* u_fine);
/* Exact solve on the coarsest level (one time step). */
int stm_coarsest_solve(stm_handle* h, int adjoint, const double* f, double* u);

#ifdef __cplusplus
}
#endif

#endif /* STMG_MESH_H */
