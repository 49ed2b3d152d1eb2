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

template <typename T, int Q>
struct MTime {
  T K[Q * Q];    // K_tau[k][l], row = test function k
  T Mh[Q];       // M_tau[k][k] / tau
  T st[Q];       // psi_k(t_{n-1}^+)
  T en[Q];       // psi_k(t_n^-)
  T R1[Q * Q];   // coarse k <- fine l, first fine slab
  T R2[Q * Q];   // coarse k <- fine l, second fine slab
};

template <typename T>
struct Csr {
  const int* rp;  // Nx + 1 row starts
  const int* ci;  // column (vertex) of every entry
  const T* mv;    // M_h entries
  const T* kv;    // K_h entries
};

// The same rows padded to the longest row W and stored slot-major: entry w of
// row j at [w * Nx + j] (padding: the row's own vertex with zero weights), so a
// warp's loads of one slot are contiguous and all slots of a row can be in
// flight at once.
template <typename T>
struct Ell {
  int W;
  const int* ci;
  const T* mv;
  const T* kv;
};

// Prolongation of the nested P1 spaces from mesh level l-1 to l: fine vertex j
// is a coarse vertex (p1 = -2: value of coarse p0) or the midpoint of a coarse
// edge (half the value of each endpoint; -1 marks a boundary endpoint).
struct Parents {
  const int* p0;
  const int* p1;
};

// Its transpose, a CSR over the coarse vertices: fine vertex ci[e], weight w[e].
template <typename T>
struct Children {
  const int* rp;
  const int* ci;
  const T* w;
};

// Steps per thread of the CSR kernels below: one pass over the CSR row of a
// vertex serves kMSteps consecutive time steps (the row's indices and weights
// are loaded once, and the gathers of the steps are independent).
constexpr int kMSteps = 4;

// (A x_s)_k for the steps s = sb .. sb + kMSteps - 1 (those below N) of vertex j;
// with TRACE also the M_h-weighted neighbouring trace mt[i] of step s (forward:
// sum_l en[l] x_{s-1,l}, adjoint: sum_l st[l] x_{s+1,l}; zero outside 0..N-1).
template <typename T, int Q, bool ADJ, bool TRACE>
__device__ __forceinline__ void apply_A_steps(const Ell<T>& A, int j, int64_t Nx, int N, int sb,
                                              const T* __restrict__ x, T tau, const MTime<T, Q>& tc,
                                              T (&ax)[kMSteps][Q], T (&mt)[kMSteps]) {
  constexpr int TS = kMSteps;
  const int64_t slab = (int64_t)Q * Nx;
  T mu[TS][Q], ku[TS][Q], tr[TS];
#pragma unroll
  for (int i = 0; i < TS; ++i) {
    tr[i] = T(0);
#pragma unroll
    for (int l = 0; l < Q; ++l) mu[i][l] = ku[i][l] = T(0);
  }
#pragma unroll 4
  for (int w = 0; w < A.W; ++w) {
    const int64_t e = (int64_t)w * Nx + j;
    const int c = A.ci[e];
    const T m = A.mv[e], k = A.kv[e];
    const T* xc = x + c;
    if (TRACE) {   // the neighbouring step of the first step of the block
      const int nb = ADJ ? sb + TS : sb - 1;
      if (!ADJ && nb >= 0) {
        T t = T(0);
#pragma unroll
        for (int l = 0; l < Q; ++l) t += tc.en[l] * xc[nb * slab + l * Nx];
        tr[0] += m * t;
      }
      if (ADJ && nb < N) {
        T t = T(0);
#pragma unroll
        for (int l = 0; l < Q; ++l) t += tc.st[l] * xc[nb * slab + l * Nx];
        tr[TS - 1] += m * t;
      }
    }
#pragma unroll
    for (int i = 0; i < TS; ++i) {
      const int s = sb + i;
      if (s >= N) break;
      T v[Q];
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        v[l] = xc[s * slab + l * Nx];
        mu[i][l] += m * v[l];
        ku[i][l] += k * v[l];
      }
      if (TRACE) {   // step s feeds the trace of step s + 1 (forward) or s - 1 (adjoint)
        T t = T(0);
#pragma unroll
        for (int l = 0; l < Q; ++l) t += (ADJ ? tc.st[l] : tc.en[l]) * v[l];
        if (!ADJ && i + 1 < TS) tr[i + 1] += m * t;
        if (ADJ && i >= 1) tr[i - 1] += m * t;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < TS; ++i) {
    mt[i] = tr[i];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      T acc = tau * tc.Mh[k] * ku[i][k];
#pragma unroll
      for (int l = 0; l < Q; ++l) acc += (ADJ ? tc.K[l * Q + k] : tc.K[k * Q + l]) * mu[i][l];
      ax[i][k] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Space-time residual r = f - L u (system chap4_generalLinearSystem), or
// f - L^T u:  forward  r_{s,k} = f_{s,k} - (A u_s)_k + st[k] M_h (sum_l en[l] u_{s-1,l}),
//             adjoint  r_{s,k} = f_{s,k} - (A^T u_s)_k + en[k] M_h (sum_l st[l] u_{s+1,l}).
// One thread per (vertex, step); steps s0 + blockIdx.y.
// ---------------------------------------------------------------------------
template <typename T, int Q, bool ADJ>
__global__ void k_mresidual(const T* __restrict__ f, const T* __restrict__ u, T* __restrict__ r,
                            Ell<T> A, int Nx, int N, int s0, T tau, MTime<T, Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = s0 + blockIdx.y * kMSteps;
  if (j >= Nx || sb >= N) return;
  const int64_t slab = (int64_t)Q * Nx;
  T ax[kMSteps][Q], mt[kMSteps];
  apply_A_steps<T, Q, ADJ, true>(A, j, Nx, N, sb, u, tau, tc, ax, mt);
#pragma unroll
  for (int i = 0; i < kMSteps; ++i) {
    const int s = sb + i;
    if (s >= N) break;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int64_t idx = s * slab + (int64_t)k * Nx + j;
      r[idx] = f[idx] - ax[i][k] + (ADJ ? tc.en[k] : tc.st[k]) * mt[i];
    }
  }
}

// The residual of k_mresidual fused with the first point-block Jacobi sweep of
// the smoother's spatial V-cycle from a zero guess: r as above and, on the
// same mesh, x = omega_x D_j^{-1} r_j (D^{-T} for the adjoint).
template <typename T, int Q, bool ADJ>
__global__ void k_mresidual_jacobi0(const T* __restrict__ f, const T* __restrict__ u,
                                    T* __restrict__ r, T* __restrict__ x, Ell<T> A, int Nx, int N, int s0,
                                    T tau, T omega_x, const T* __restrict__ dinv, MTime<T, Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = s0 + blockIdx.y * kMSteps;
  if (j >= Nx || sb >= N) return;
  const int64_t slab = (int64_t)Q * Nx;
  T ax[kMSteps][Q], mt[kMSteps];
  apply_A_steps<T, Q, ADJ, true>(A, j, Nx, N, sb, u, tau, tc, ax, mt);
  T D[Q * Q];
#pragma unroll
  for (int e = 0; e < Q * Q; ++e) D[e] = dinv[(int64_t)j * Q * Q + e];
#pragma unroll
  for (int i = 0; i < kMSteps; ++i) {
    const int s = sb + i;
    if (s >= N) break;
    T res[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int64_t idx = s * slab + (int64_t)k * Nx + j;
      res[k] = f[idx] - ax[i][k] + (ADJ ? tc.en[k] : tc.st[k]) * mt[i];
      r[idx] = res[k];
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < Q; ++l) acc += (ADJ ? D[l * Q + k] : D[k * Q + l]) * res[l];
      x[s * slab + (int64_t)k * Nx + j] = omega_x * acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Spatial V-cycle of the inexact block inverse, per time step (no coupling
// between steps): the operator is A_tau (or A_tau^T) of the level's tau.
// Damped point-block Jacobi: y = x + omega D_j^{-1} (b - A x)_j, D_j^{-1} tabulated
// per vertex (dinv, Q x Q row-major; the adjoint uses its transpose).  ZERO: x = 0.
// ---------------------------------------------------------------------------
template <typename T, int Q, bool ADJ, bool ZERO>
__global__ void k_mjacobi(const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ y,
                          Ell<T> A, int Nx, int N, int s0, T tau, T omega, const T* __restrict__ dinv,
                          MTime<T, Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = s0 + blockIdx.y * kMSteps;
  if (j >= Nx || sb >= N) return;
  const int64_t slab = (int64_t)Q * Nx;
  T ax[kMSteps][Q], mt[kMSteps];
  if (!ZERO) apply_A_steps<T, Q, ADJ, false>(A, j, Nx, N, sb, x, tau, tc, ax, mt);
  T D[Q * Q];
#pragma unroll
  for (int e = 0; e < Q * Q; ++e) D[e] = dinv[(int64_t)j * Q * Q + e];
#pragma unroll
  for (int i = 0; i < kMSteps; ++i) {
    const int s = sb + i;
    if (s >= N) break;
    const int64_t base = s * slab + j;
    T res[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) res[k] = b[base + (int64_t)k * Nx] - (ZERO ? T(0) : ax[i][k]);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < Q; ++l) acc += (ADJ ? D[l * Q + k] : D[k * Q + l]) * res[l];
      y[base + (int64_t)k * Nx] = (ZERO ? T(0) : x[base + (int64_t)k * Nx]) + omega * acc;
    }
  }
}

// r = b - A x per time step.
template <typename T, int Q, bool ADJ>
__global__ void k_mspace_residual(const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r,
                                  Ell<T> A, int Nx, int N, int s0, T tau, MTime<T, Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = s0 + blockIdx.y * kMSteps;
  if (j >= Nx || sb >= N) return;
  const int64_t slab = (int64_t)Q * Nx;
  T ax[kMSteps][Q], mt[kMSteps];
  apply_A_steps<T, Q, ADJ, false>(A, j, Nx, N, sb, x, tau, tc, ax, mt);
#pragma unroll
  for (int i = 0; i < kMSteps; ++i) {
    const int s = sb + i;
    if (s >= N) break;
    const int64_t base = s * slab + j;
#pragma unroll
    for (int k = 0; k < Q; ++k) r[base + (int64_t)k * Nx] = b[base + (int64_t)k * Nx] - ax[i][k];
  }
}

// The last point-block Jacobi sweep of the spatial V-cycle fused with the
// damped update of the smoothing step (eq. chap4_smoother):
// u += omega_t (x + omega_x D_j^{-1} (b - A x)_j), without storing the sweep.
template <typename T, int Q, bool ADJ>
__global__ void k_mjacobi_update(const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ u,
                                 Ell<T> A, int Nx, int N, int s0, T tau, T omega_x, T omega_t,
                                 const T* __restrict__ dinv, MTime<T, Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = s0 + blockIdx.y * kMSteps;
  if (j >= Nx || sb >= N) return;
  const int64_t slab = (int64_t)Q * Nx;
  T ax[kMSteps][Q], mt[kMSteps];
  apply_A_steps<T, Q, ADJ, false>(A, j, Nx, N, sb, x, tau, tc, ax, mt);
  T D[Q * Q];
#pragma unroll
  for (int e = 0; e < Q * Q; ++e) D[e] = dinv[(int64_t)j * Q * Q + e];
#pragma unroll
  for (int i = 0; i < kMSteps; ++i) {
    const int s = sb + i;
    if (s >= N) break;
    const int64_t base = s * slab + j;
    T res[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) res[k] = b[base + (int64_t)k * Nx] - ax[i][k];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < Q; ++l) acc += (ADJ ? D[l * Q + k] : D[k * Q + l]) * res[l];
      const T xn = x[base + (int64_t)k * Nx] + omega_x * acc;
      u[base + (int64_t)k * Nx] += omega_t * xn;
    }
  }
}

// Initial value (eq. (equation1), the n = 0 term): g_{0,k} = f_{0,k} + st[k] (M_h u0)_j.
template <int Q>
__global__ void k_madd_ic(const double* __restrict__ f, const double* __restrict__ u0, double* __restrict__ g,
                          Csr<double> A, int Nx, MTime<double, Q> tc) {
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
__global__ void k_mic_gradient(const double* __restrict__ lam, double* __restrict__ g, Csr<double> A, int Nx, MTime<double, Q> tc) {
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

// bc = (I (x) P^T) r per time step: coarse vertex c gathers its fine vertices.
template <typename T, int Q>
__global__ void k_mrestrict_space(const T* __restrict__ r, T* __restrict__ bc, Children<T> ch, int Nc, int Nf,
                                  int N, int s0) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (c >= Nc || s >= N) return;
  T acc[Q];
#pragma unroll
  for (int l = 0; l < Q; ++l) acc[l] = T(0);
  const int e1 = ch.rp[c + 1];
  for (int e = ch.rp[c]; e < e1; ++e) {
    const int jf = ch.ci[e];
    const T w = ch.w[e];
#pragma unroll
    for (int l = 0; l < Q; ++l) acc[l] += w * r[(s * (int64_t)Q + l) * Nf + jf];
  }
#pragma unroll
  for (int l = 0; l < Q; ++l) bc[(s * (int64_t)Q + l) * Nc + c] = acc[l];
}

template <typename T>
__device__ __forceinline__ T interp(const Parents& p, int j, const T* __restrict__ xc) {
  const int a = p.p0[j], b = p.p1[j];
  if (b == -2) return a >= 0 ? xc[a] : T(0);
  return T(0.5) * ((a >= 0 ? xc[a] : T(0)) + (b >= 0 ? xc[b] : T(0)));
}

// x += (I (x) P) xc per time step.
template <typename T, int Q>
__global__ void k_mprolong_space_add(const T* __restrict__ xc, T* __restrict__ x, Parents par, int Nc,
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
template <typename T>
__global__ void k_mdense_apply(const T* __restrict__ b, T* __restrict__ y, const T* __restrict__ ainv,
                               int n, int N, int s0, bool adj) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (i >= n || s >= N) return;
  const T* bs = b + (int64_t)s * n;
  T acc = T(0);
  for (int k = 0; k < n; ++k) acc += (adj ? ainv[(int64_t)k * n + i] : ainv[(int64_t)i * n + k]) * bs[k];
  y[(int64_t)s * n + i] = acc;
}

// ---------------------------------------------------------------------------
// Space-time restriction (eqs. chap4_restrictionTime, Section 2 R = P^T):
// fc[m, k, c] = sum_l R1[k,l] (Rx r)[2m, l, c] + R2[k,l] (Rx r)[2m+1, l, c],
// Rx = identity (semi) or the transposed mesh prolongation (full).
// ---------------------------------------------------------------------------
template <typename T, int Q, bool FULL>
__global__ void k_mrestrict(const T* __restrict__ r, T* __restrict__ fc, Children<T> ch, int Nc, int Nf,
                            int Ncs, int m0, MTime<T, Q> tc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = m0 + blockIdx.y;
  if (c >= Nc || m >= Ncs) return;
  T a[Q], b[Q];
  const T* r0 = r + (2 * (int64_t)m) * Q * Nf;
  const T* r1 = r0 + (int64_t)Q * Nf;
  if (FULL) {
#pragma unroll
    for (int l = 0; l < Q; ++l) a[l] = b[l] = T(0);
    const int e1 = ch.rp[c + 1];
    for (int e = ch.rp[c]; e < e1; ++e) {
      const int jf = ch.ci[e];
      const T w = ch.w[e];
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
    T acc = T(0);
#pragma unroll
    for (int l = 0; l < Q; ++l) acc += tc.R1[k * Q + l] * a[l] + tc.R2[k * Q + l] * b[l];
    fc[((int64_t)m * Q + k) * Nc + c] = acc;
  }
}

// u[2m + sigma, l, j] += sum_k R_sigma[k,l] (Px ec)[m, k, j] (the transpose of k_mrestrict).
template <typename T, int Q, bool FULL>
__global__ void k_mprolong(const T* __restrict__ ec, T* __restrict__ u, Parents par, int Nc, int Nf,
                           int Ncs, int m0, MTime<T, Q> tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = m0 + blockIdx.y;
  if (j >= Nf || m >= Ncs) return;
  T e[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const T* eck = ec + ((int64_t)m * Q + k) * Nc;
    e[k] = FULL ? interp(par, j, eck) : eck[j];
  }
  T* u0 = u + (2 * (int64_t)m) * Q * Nf;
  T* u1 = u0 + (int64_t)Q * Nf;
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    T a = T(0), b = T(0);
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
