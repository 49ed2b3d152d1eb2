// Device kernels of the space-time multigrid on P1 simplicial meshes
// (node basis).  Vector layout: index ((s * Q + l) * Nx + j), time step s,
// time dof l, interior vertex j.  M_h and K_h share one CSR pattern (vertex
// adjacency of the mesh) with two value arrays.
//
// Time matrices (Section 1, Legendre basis) come by value in MTime: K_tau,
// M_tau / tau, the end values psi_k(t_{n-1}^+), psi_k(t_n^-) (N_tau = st en^T)
// and the time restriction blocks R1, R2 of eq. (chap4_restrictionTime).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace stmm {

template <int Q>
struct MTime {
  double K[Q * Q];    // K_tau[k][l], row = test function k
  double Mh[Q];       // M_tau[k][k] / tau
  double st[Q];       // psi_k(t_{n-1}^+)
  double en[Q];       // psi_k(t_n^-)
  double R1[Q * Q];   // coarse k <- fine l, first fine slab
  double R2[Q * Q];   // coarse k <- fine l, second fine slab
};

struct Csr {
  const int* rp;      // Nx + 1 row starts
  const int* ci;      // column (vertex) of every entry
  const double* mv;   // M_h entries
  const double* kv;   // K_h entries
};

// Prolongation of the nested P1 spaces from mesh level l-1 to l: fine vertex j
// is a coarse vertex (p1 = -2: value of coarse p0) or the midpoint of a coarse
// edge (half the value of each endpoint; -1 marks a boundary endpoint).
struct Parents {
  const int* p0;
  const int* p1;
};

// Its transpose, a CSR over the coarse vertices: fine vertex ci[e], weight w[e].
struct Children {
  const int* rp;
  const int* ci;
  const double* w;
};

__device__ __forceinline__ void spmv_mk(const Csr& A, int j, const double* __restrict__ x, double& m, double& k) {
  double sm = 0.0, sk = 0.0;
  const int e1 = A.rp[j + 1];
  for (int e = A.rp[j]; e < e1; ++e) {
    const double v = x[A.ci[e]];
    sm += A.mv[e] * v;
    sk += A.kv[e] * v;
  }
  m = sm;
  k = sk;
}

// (A x)_k for the space-time block A = K_tau (x) M_h + M_tau (x) K_h (or A^T)
// at vertex j of the slab starting at x (the q fields of one time step).
template <int Q, bool ADJ>
__device__ __forceinline__ void apply_A(const Csr& A, int j, int64_t Nx, const double* __restrict__ x, double tau,
                                        const MTime<Q>& tc, double (&ax)[Q]) {
  double mu[Q], ku[Q];
#pragma unroll
  for (int l = 0; l < Q; ++l) spmv_mk(A, j, x + l * Nx, mu[l], ku[l]);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    double acc = tau * tc.Mh[k] * ku[k];
#pragma unroll
    for (int l = 0; l < Q; ++l) acc += (ADJ ? tc.K[l * Q + k] : tc.K[k * Q + l]) * mu[l];
    ax[k] = acc;
  }
}

// ---------------------------------------------------------------------------
// Space-time residual r = f - L u (system chap4_generalLinearSystem), or
// f - L^T u:  forward  r_{s,k} = f_{s,k} - (A u_s)_k + st[k] M_h (sum_l en[l] u_{s-1,l}),
//             adjoint  r_{s,k} = f_{s,k} - (A^T u_s)_k + en[k] M_h (sum_l st[l] u_{s+1,l}).
// One thread per (vertex, step); steps s0 + blockIdx.y.
// ---------------------------------------------------------------------------
template <int Q, bool ADJ>
__global__ void k_mresidual(const double* __restrict__ f, const double* __restrict__ u, double* __restrict__ r,
                            Csr A, int Nx, int N, int s0, double tau, MTime<Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (j >= Nx || s >= N) return;
  const int64_t slab = (int64_t)Q * Nx;
  double ax[Q];
  apply_A<Q, ADJ>(A, j, Nx, u + s * slab, tau, tc, ax);
  double mt = 0.0;
  const int nb = ADJ ? s + 1 : s - 1;
  if (nb >= 0 && nb < N) {
    const double* un = u + nb * slab;
    const int e1 = A.rp[j + 1];
    for (int e = A.rp[j]; e < e1; ++e) {
      const int c = A.ci[e];
      double t = 0.0;
#pragma unroll
      for (int l = 0; l < Q; ++l) t += (ADJ ? tc.st[l] : tc.en[l]) * un[l * (int64_t)Nx + c];
      mt += A.mv[e] * t;
    }
  }
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int64_t idx = s * slab + (int64_t)k * Nx + j;
    r[idx] = f[idx] - ax[k] + (ADJ ? tc.en[k] : tc.st[k]) * mt;
  }
}

// The residual of k_mresidual fused with the first point-block Jacobi sweep of
// the smoother's spatial V-cycle from a zero guess: r as above and, on the
// same mesh, x = omega_x D_j^{-1} r_j (D^{-T} for the adjoint).
template <int Q, bool ADJ>
__global__ void k_mresidual_jacobi0(const double* __restrict__ f, const double* __restrict__ u,
                                    double* __restrict__ r, double* __restrict__ x, Csr A, int Nx, int N, int s0,
                                    double tau, double omega_x, const double* __restrict__ dinv, MTime<Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (j >= Nx || s >= N) return;
  const int64_t slab = (int64_t)Q * Nx;
  double ax[Q];
  apply_A<Q, ADJ>(A, j, Nx, u + s * slab, tau, tc, ax);
  double mt = 0.0;
  const int nb = ADJ ? s + 1 : s - 1;
  if (nb >= 0 && nb < N) {
    const double* un = u + nb * slab;
    const int e1 = A.rp[j + 1];
    for (int e = A.rp[j]; e < e1; ++e) {
      const int c = A.ci[e];
      double t = 0.0;
#pragma unroll
      for (int l = 0; l < Q; ++l) t += (ADJ ? tc.st[l] : tc.en[l]) * un[l * (int64_t)Nx + c];
      mt += A.mv[e] * t;
    }
  }
  double res[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int64_t idx = s * slab + (int64_t)k * Nx + j;
    res[k] = f[idx] - ax[k] + (ADJ ? tc.en[k] : tc.st[k]) * mt;
    r[idx] = res[k];
  }
  const double* D = dinv + (int64_t)j * Q * Q;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < Q; ++l) acc += (ADJ ? D[l * Q + k] : D[k * Q + l]) * res[l];
    x[s * slab + (int64_t)k * Nx + j] = omega_x * acc;
  }
}

// The last point-block Jacobi sweep of the spatial V-cycle fused with the
// damped update of the smoothing step (eq. chap4_smoother):
// u += omega_t (x + omega_x D_j^{-1} (b - A x)_j), without storing the sweep.
template <int Q, bool ADJ>
__global__ void k_mjacobi_update(const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ u,
                                 Csr A, int Nx, int N, int s0, double tau, double omega_x, double omega_t,
                                 const double* __restrict__ dinv, MTime<Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (j >= Nx || s >= N) return;
  const int64_t base = s * (int64_t)Q * Nx + j;
  double ax[Q];
  apply_A<Q, ADJ>(A, j, Nx, x + s * (int64_t)Q * Nx, tau, tc, ax);
  double res[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) res[k] = b[base + (int64_t)k * Nx] - ax[k];
  const double* D = dinv + (int64_t)j * Q * Q;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < Q; ++l) acc += (ADJ ? D[l * Q + k] : D[k * Q + l]) * res[l];
    const double xn = x[base + (int64_t)k * Nx] + omega_x * acc;
    u[base + (int64_t)k * Nx] += omega_t * xn;
  }
}

// Initial value (eq. (equation1), the n = 0 term): g_{0,k} = f_{0,k} + st[k] (M_h u0)_j.
template <int Q>
__global__ void k_madd_ic(const double* __restrict__ f, const double* __restrict__ u0, double* __restrict__ g,
                          Csr A, int Nx, MTime<Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Nx) return;
  double m = 0.0;
  const int e1 = A.rp[j + 1];
  for (int e = A.rp[j]; e < e1; ++e) m += A.mv[e] * u0[A.ci[e]];
#pragma unroll
  for (int k = 0; k < Q; ++k) g[(int64_t)k * Nx + j] = f[(int64_t)k * Nx + j] + tc.st[k] * m;
}

// grad_u0 = M_h sum_k psi_k(t_0^+) lambda_{0,k}.
template <int Q>
__global__ void k_mic_gradient(const double* __restrict__ lam, double* __restrict__ g, Csr A, int Nx, MTime<Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Nx) return;
  double m = 0.0;
  const int e1 = A.rp[j + 1];
  for (int e = A.rp[j]; e < e1; ++e) {
    const int c = A.ci[e];
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < Q; ++k) t += tc.st[k] * lam[(int64_t)k * Nx + c];
    m += A.mv[e] * t;
  }
  g[j] = m;
}

// ---------------------------------------------------------------------------
// Spatial V-cycle of the inexact block inverse, per time step (no coupling
// between steps): the operator is A_tau (or A_tau^T) of the level's tau.
// Damped point-block Jacobi: y = x + omega D_j^{-1} (b - A x)_j, D_j^{-1} tabulated
// per vertex (dinv, Q x Q row-major; the adjoint uses its transpose).  ZERO: x = 0.
// ---------------------------------------------------------------------------
template <int Q, bool ADJ, bool ZERO>
__global__ void k_mjacobi(const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ y,
                          Csr A, int Nx, int N, int s0, double tau, double omega, const double* __restrict__ dinv,
                          MTime<Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (j >= Nx || s >= N) return;
  const int64_t base = s * (int64_t)Q * Nx + j;
  double res[Q];
  if (ZERO) {
#pragma unroll
    for (int k = 0; k < Q; ++k) res[k] = b[base + (int64_t)k * Nx];
  } else {
    double ax[Q];
    apply_A<Q, ADJ>(A, j, Nx, x + s * (int64_t)Q * Nx, tau, tc, ax);
#pragma unroll
    for (int k = 0; k < Q; ++k) res[k] = b[base + (int64_t)k * Nx] - ax[k];
  }
  const double* D = dinv + (int64_t)j * Q * Q;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < Q; ++l) acc += (ADJ ? D[l * Q + k] : D[k * Q + l]) * res[l];
    y[base + (int64_t)k * Nx] = (ZERO ? 0.0 : x[base + (int64_t)k * Nx]) + omega * acc;
  }
}

// r = b - A x per time step.
template <int Q, bool ADJ>
__global__ void k_mspace_residual(const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ r,
                                  Csr A, int Nx, int N, int s0, double tau, MTime<Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (j >= Nx || s >= N) return;
  const int64_t base = s * (int64_t)Q * Nx + j;
  double ax[Q];
  apply_A<Q, ADJ>(A, j, Nx, x + s * (int64_t)Q * Nx, tau, tc, ax);
#pragma unroll
  for (int k = 0; k < Q; ++k) r[base + (int64_t)k * Nx] = b[base + (int64_t)k * Nx] - ax[k];
}

// bc = (I (x) P^T) r per time step: coarse vertex c gathers its fine vertices.
template <int Q>
__global__ void k_mrestrict_space(const double* __restrict__ r, double* __restrict__ bc, Children ch, int Nc, int Nf,
                                  int N, int s0) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (c >= Nc || s >= N) return;
  double acc[Q];
#pragma unroll
  for (int l = 0; l < Q; ++l) acc[l] = 0.0;
  const int e1 = ch.rp[c + 1];
  for (int e = ch.rp[c]; e < e1; ++e) {
    const int jf = ch.ci[e];
    const double w = ch.w[e];
#pragma unroll
    for (int l = 0; l < Q; ++l) acc[l] += w * r[(s * (int64_t)Q + l) * Nf + jf];
  }
#pragma unroll
  for (int l = 0; l < Q; ++l) bc[(s * (int64_t)Q + l) * Nc + c] = acc[l];
}

__device__ __forceinline__ double interp(const Parents& p, int j, const double* __restrict__ xc) {
  const int a = p.p0[j], b = p.p1[j];
  if (b == -2) return a >= 0 ? xc[a] : 0.0;
  return 0.5 * ((a >= 0 ? xc[a] : 0.0) + (b >= 0 ? xc[b] : 0.0));
}

// x += (I (x) P) xc per time step.
template <int Q>
__global__ void k_mprolong_space_add(const double* __restrict__ xc, double* __restrict__ x, Parents par, int Nc,
                                     int Nf, int N, int s0) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (j >= Nf || s >= N) return;
#pragma unroll
  for (int l = 0; l < Q; ++l)
    x[(s * (int64_t)Q + l) * Nf + j] += interp(par, j, xc + (s * (int64_t)Q + l) * Nc);
}

// Exact solve on the initial mesh: y_s = Ainv b_s (or Ainv^T b_s) with the dense
// inverse of the (Q Nx0)-square block A_tau; one thread per (row, step).
__global__ void k_mdense_apply(const double* __restrict__ b, double* __restrict__ y, const double* __restrict__ ainv,
                               int n, int N, int s0, bool adj) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (i >= n || s >= N) return;
  const double* bs = b + (int64_t)s * n;
  double acc = 0.0;
  for (int k = 0; k < n; ++k) acc += (adj ? ainv[(int64_t)k * n + i] : ainv[(int64_t)i * n + k]) * bs[k];
  y[(int64_t)s * n + i] = acc;
}

// ---------------------------------------------------------------------------
// Space-time restriction (eqs. chap4_restrictionTime, Section 2 R = P^T):
// fc[m, k, c] = sum_l R1[k,l] (Rx r)[2m, l, c] + R2[k,l] (Rx r)[2m+1, l, c],
// Rx = identity (semi) or the transposed mesh prolongation (full).
// ---------------------------------------------------------------------------
template <int Q, bool FULL>
__global__ void k_mrestrict(const double* __restrict__ r, double* __restrict__ fc, Children ch, int Nc, int Nf,
                            int Ncs, int m0, MTime<Q> tc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = m0 + blockIdx.y;
  if (c >= Nc || m >= Ncs) return;
  double a[Q], b[Q];
  const double* r0 = r + (2 * (int64_t)m) * Q * Nf;
  const double* r1 = r0 + (int64_t)Q * Nf;
  if (FULL) {
#pragma unroll
    for (int l = 0; l < Q; ++l) a[l] = b[l] = 0.0;
    const int e1 = ch.rp[c + 1];
    for (int e = ch.rp[c]; e < e1; ++e) {
      const int jf = ch.ci[e];
      const double w = ch.w[e];
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        a[l] += w * r0[(int64_t)l * Nf + jf];
        b[l] += w * r1[(int64_t)l * Nf + jf];
      }
    }
  } else {
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      a[l] = r0[(int64_t)l * Nf + c];
      b[l] = r1[(int64_t)l * Nf + c];
    }
  }
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < Q; ++l) acc += tc.R1[k * Q + l] * a[l] + tc.R2[k * Q + l] * b[l];
    fc[((int64_t)m * Q + k) * Nc + c] = acc;
  }
}

// u[2m + sigma, l, j] += sum_k R_sigma[k,l] (Px ec)[m, k, j] (the transpose of k_mrestrict).
template <int Q, bool FULL>
__global__ void k_mprolong(const double* __restrict__ ec, double* __restrict__ u, Parents par, int Nc, int Nf,
                           int Ncs, int m0, MTime<Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = m0 + blockIdx.y;
  if (j >= Nf || m >= Ncs) return;
  double e[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const double* eck = ec + ((int64_t)m * Q + k) * Nc;
    e[k] = FULL ? interp(par, j, eck) : eck[j];
  }
  double* u0 = u + (2 * (int64_t)m) * Q * Nf;
  double* u1 = u0 + (int64_t)Q * Nf;
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    double a = 0.0, b = 0.0;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      a += tc.R1[k * Q + l] * e[k];
      b += tc.R2[k * Q + l] * e[k];
    }
    u0[(int64_t)l * Nf + j] += a;
    u1[(int64_t)l * Nf + j] += b;
  }
}

}  // namespace stmm
