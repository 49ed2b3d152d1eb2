// Kernels of the V-cycle with the exact block inverse, in the mixed basis:
// sine coefficients along the first D-1 spatial axes, nodes along the last.
//
// The sine vectors diagonalise M_1 and K_1 (Section 3.1), so with
// v^ = S v (S = DST-I along the first D-1 axes, unnormalised) every operator of
// a level acts mode by mode on lines along the last axis:
//   (M_h v)^ [i, p] = alpha_i (M_1 v^_i)[p],
//   (K_h v)^ [i, p] = alpha_i (K_1 v^_i)[p] + beta_i (M_1 v^_i)[p],
// alpha_i = prod_a m(k_a), beta_i = sum_a kappa(k_a) prod_{b != a} m(k_b),
// m(k) = h/3 (2 + cos(k pi / Nf)), kappa(k) = 2/h (1 - cos(k pi / Nf)).
// The full-coarsening transfer pairs fine modes k and Nf - k with coarse mode k:
// for linear interpolation P, P phi^c_k = (1+c_k)/2 phi^f_k - (1-c_k)/2 phi^f_{Nf-k},
// c_k = cos(k pi / Nf), so with R = P^T
//   (R r)^_k = (1+c_k)/2 r^_k - (1-c_k)/2 r^_{Nf-k}            (restriction)
//   (P e)^_k = (1+c_k) e^_k,  (P e)^_{Nf-k} = -(1-c_k) e^_k      (prolongation; S P S^{-1})
// and mode Nf/2 has no coarse counterpart.  The iterates of the V-cycle are
// the images under S of those of the same cycle written on nodes: one forward
// transform of the data and one inverse transform of the result per solve.
//
// Layout: index ((s * Q + l) * Nx + p * nm + i): time step s, time dof l, line
// position p (0..n-1 along the last axis), mode i (0..nm-1, nm = n^(D-1), the
// first transformed axis fastest), Nx = nm * n.  Consecutive threads take
// consecutive modes, so every access along a line is coalesced.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "stmg_kernels.cuh"

namespace stmg {

// Time traces of a step with the Legendre slab basis (Section 1), whose end
// values are psi_k(t_{n-1}^+) = (-1)^k and psi_k(t_n^-) = 1: the coupling of
// step s to s-1 (forward) uses sum_l u_{s-1,l} and enters row k with sign
// (-1)^k; the transposed coupling to s+1 uses sum_l (-1)^l u_{s+1,l} and
// enters every row with sign +1.  Additions only, no multiplies.
template <typename T, int Q, bool ADJ>
__device__ __forceinline__ T step_trace(const T* __restrict__ nb, int64_t Nx, int64_t o) {
  T v = nb[o];
#pragma unroll
  for (int l = 1; l < Q; ++l) {
    const T x = nb[(int64_t)l * Nx + o];
    v = (ADJ && (l & 1)) ? v - x : v + x;
  }
  return v;
}

template <typename T, bool ADJ>
__device__ __forceinline__ T couple(int k, T g, T mt) {
  return (!ADJ && (k & 1)) ? g - mt : g + mt;
}

// Pointer type with or without __restrict__ (kernels whose buffers may alias
// in one use and not in another).
template <typename P, bool RESTRICT>
struct PtrSel {
  typedef P* type;
};
template <typename P>
struct PtrSel<P, true> {
  typedef P* __restrict__ type;
};

// ---------------------------------------------------------------------------
// Residual r^ = f^ - L^ u^ (forward) or f^ - L^T u^ (adjoint) in the mixed basis;
// the operator is that of k_residual with M_h, K_h replaced by their mode-wise
// line forms.  Row k of the block row of step s:
//   sum_l [a K[k,l] M_1 + delta_kl tau Mh[k] (a K_1 + b M_1)] u_{s,l}
// is a three-point stencil per (k, l) with weights w0 (neighbours) and w1
// (centre), tabulated per mode on the host.  The time coupling adds
// (-1)^k a M_1 t, t = sum_l u_{s-1,l} (adjoint: a M_1 sum_l (-1)^l u_{s+1,l});
// at s = 0 of the forward problem t is the transformed initial value u0^ (or 0).
// One thread per (mode, chunk of mres_chunk<T>() line positions, time step); the
// three-point window slides along the chunk in registers.
// ---------------------------------------------------------------------------
// Line positions per thread: FP64 amortises the per-thread table loads over
// more points; FP32 is bound by memory latency and wants more threads.
template <typename T>
__host__ __device__ constexpr int mres_chunk() { return sizeof(T) == 8 ? 16 : 8; }

// Per-mode residual weights (host table, FP64 formed then rounded to T):
// rw[(e) * nm + i] = w0 for e = k*Q + l, rw[(Q*Q + e) * nm + i] = w1,
// rw[(2*Q*Q) * nm + i] = a m0, rw[(2*Q*Q + 1) * nm + i] = a m1 (M_1 weights
// of the coupling term times alpha_i).
template <typename T, int Q, bool ADJ>
__global__ void __launch_bounds__(256) k_mresidual(const T* __restrict__ f, const T* __restrict__ u,
                                                   const T* __restrict__ u0, T* __restrict__ r, int n, int nm,
                                                   int N, int s0, const T* __restrict__ rw) {
  constexpr int QQ = Q * Q;
  constexpr int CH = mres_chunk<T>();
  const int nch = (n + CH - 1) / CH;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (t >= (int64_t)nm * nch || s >= N) return;
  const int i = (int)(t % nm), c = (int)(t / nm);
  const int p0 = c * CH, p1 = min(p0 + CH, n);
  const int64_t Nx = (int64_t)nm * n;
  T w0[QQ], w1[QQ];
#pragma unroll
  for (int e = 0; e < QQ; ++e) {
    w0[e] = rw[(int64_t)e * nm + i];
    w1[e] = rw[(int64_t)(QQ + e) * nm + i];
  }
  const T am0 = rw[(int64_t)(2 * QQ) * nm + i], am1 = rw[(int64_t)(2 * QQ + 1) * nm + i];
  const T* nb = nullptr;
  if (!ADJ && s > 0) nb = u + (int64_t)(s - 1) * Q * Nx;
  if (ADJ && s < N - 1) nb = u + (int64_t)(s + 1) * Q * Nx;
  const bool use_u0 = !ADJ && s == 0 && u0 != nullptr;
  auto trace = [&](int p) -> T {
    if (p < 0 || p >= n) return T(0);
    const int64_t o = (int64_t)p * nm + i;
    if (nb != nullptr) return step_trace<T, Q, ADJ>(nb, Nx, o);
    return use_u0 ? u0[o] : T(0);
  };
  const T* us = u + (int64_t)s * Q * Nx + i;
  T up[Q], uc[Q];
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    up[l] = p0 > 0 ? us[(int64_t)l * Nx + (int64_t)(p0 - 1) * nm] : T(0);
    uc[l] = us[(int64_t)l * Nx + (int64_t)p0 * nm];
  }
  T tp = trace(p0 - 1), tcur = trace(p0);
  for (int p = p0; p < p1; ++p) {
    T un[Q], sg[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      un[l] = (p + 1 < n) ? us[(int64_t)l * Nx + (int64_t)(p + 1) * nm] : T(0);
      sg[l] = up[l] + un[l];
    }
    const T tn = trace(p + 1);
    const T mt = am0 * (tp + tn) + am1 * tcur;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int64_t idx = ((int64_t)s * Q + k) * Nx + (int64_t)p * nm + i;
      T acc = couple<T, ADJ>(k, f[idx], mt);
#pragma unroll
      for (int l = 0; l < Q; ++l) acc -= w0[k * Q + l] * sg[l] + w1[k * Q + l] * uc[l];
      r[idx] = acc;
    }
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      up[l] = uc[l];
      uc[l] = un[l];
    }
    tp = tcur;
    tcur = tn;
  }
}

// ---------------------------------------------------------------------------
// One damped block-Jacobi step with the exact block inverse (eq. chap4_smoother,
// Section 3.1), fused:  out = (1 - w) u + w A^{-1} (f - B u_prev)  per step,
// where the block inverse of the block row removes A u and only the rank-one
// time coupling B = -N_tau (x) M_h is applied; in the mixed basis A^{-1} is one
// block-tridiagonal solve per mode along the last axis:
//   A_i = tridiag(E_i, Dg_i, E_i),
//   Dg_i = a (4h/6) K + tau Mh (a (2/h) + b (4h/6)),  E_i = a (h/6) K + tau Mh (-a/h + b (h/6)),
// K = K_tau (adjoint: K_tau^T), with host FP64 block-LU factors (no pivoting):
// W_0 = Dg, L_p = E W_{p-1}^{-1}, W_p = Dg - L_p E;
//   forward  z_p = g_p - L_p z_{p-1}   (g = f - B u_prev, formed on the fly)
//   backward x_p = W_p^{-1} (z_p - E x_{p+1}).
// DAMP: the host passes the damped tables w W_p^{-1} and E / w, so the backward
// sweep yields y = w x directly and out = y + wc u with wc = 1 - w.  Without
// DAMP the tables are unscaled and out = x; u at step s is then never read, so
// `out` may be `u` itself (forward substitution of the coarsest solve, one
// step per launch).  u == nullptr means a zero iterate (no coupling term, no
// damping term).  f and out must not alias; with DAMP, u and out must not
// either (both are then __restrict__).  z is kept in `out` between the sweeps.  Tables: fac[((p * 2 + w) * Q*Q + e) * nm + i] (w = 0: L_p, w = 1:
// the inverse block), ecoef[e * nm + i], and the coupling weights a m0, a m1
// of the residual table rw.  One thread per (mode, time step in
// [s0, s0 + gridDim.y)).
// ---------------------------------------------------------------------------
template <typename T, int Q, bool ADJ, bool DAMP>
__global__ void __launch_bounds__(128) k_msmooth(const T* __restrict__ f, typename PtrSel<const T, DAMP>::type u,
                                                 const T* __restrict__ u0, typename PtrSel<T, DAMP>::type out,
                                                 int n, int nm, int N, int s0, T wc,
                                                 const T* __restrict__ fac, const T* __restrict__ ecoef,
                                                 const T* __restrict__ rw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (i >= nm || s >= N) return;
  const int64_t Nx = (int64_t)nm * n;
  constexpr int QQ = Q * Q;
  const T am0 = rw[(int64_t)(2 * QQ) * nm + i], am1 = rw[(int64_t)(2 * QQ + 1) * nm + i];
  const T* nb = nullptr;
  if (u != nullptr) {
    if (!ADJ && s > 0) nb = u + (int64_t)(s - 1) * Q * Nx;
    if (ADJ && s < N - 1) nb = u + (int64_t)(s + 1) * Q * Nx;
  }
  const bool use_u0 = !ADJ && s == 0 && u0 != nullptr;
  const bool any = nb != nullptr || use_u0;
  auto trace = [&](int p) -> T {
    if (p >= n) return T(0);
    const int64_t o = (int64_t)p * nm + i;
    if (nb != nullptr) return step_trace<T, Q, ADJ>(nb, Nx, o);
    return u0[o];
  };
  const T* fs = f + (int64_t)s * Q * Nx + i;
  T* os = out + (int64_t)s * Q * Nx + i;
  T z[Q];
  T tp = T(0), tcur = any ? trace(0) : T(0);
#pragma unroll 2
  for (int p = 0; p < n; ++p) {
    T g[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) g[k] = fs[(int64_t)k * Nx + (int64_t)p * nm];
    if (any) {
      const T tn = trace(p + 1);
      const T mt = am0 * (tp + tn) + am1 * tcur;
#pragma unroll
      for (int k = 0; k < Q; ++k) g[k] = couple<T, ADJ>(k, g[k], mt);
      tp = tcur;
      tcur = tn;
    }
    if (p > 0) {
      const T* Lp = fac + (int64_t)(p * 2 + 0) * QQ * nm + i;
#pragma unroll
      for (int k = 0; k < Q; ++k) {
#pragma unroll
        for (int l = 0; l < Q; ++l) g[k] -= Lp[(int64_t)(k * Q + l) * nm] * z[l];
      }
    }
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      z[l] = g[l];
      os[(int64_t)l * Nx + (int64_t)p * nm] = g[l];
    }
  }
  T E[QQ];
#pragma unroll
  for (int e = 0; e < QQ; ++e) E[e] = ecoef[(int64_t)e * nm + i];
  const T* us = (DAMP && u != nullptr) ? u + (int64_t)s * Q * Nx + i : nullptr;
  T xn[Q];
#pragma unroll 2
  for (int p = n - 1; p >= 0; --p) {
    T t[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) t[l] = (p == n - 1) ? z[l] : os[(int64_t)l * Nx + (int64_t)p * nm];
    if (p < n - 1) {
#pragma unroll
      for (int k = 0; k < Q; ++k) {
#pragma unroll
        for (int l = 0; l < Q; ++l) t[k] -= E[k * Q + l] * xn[l];
      }
    }
    const T* Wi = fac + (int64_t)(p * 2 + 1) * QQ * nm + i;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      T acc = Wi[(int64_t)(k * Q) * nm] * t[0];
#pragma unroll
      for (int l = 1; l < Q; ++l) acc += Wi[(int64_t)(k * Q + l) * nm] * t[l];
      xn[k] = acc;
    }
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      T v = xn[l];
      if (us != nullptr) v += wc * us[(int64_t)l * Nx + (int64_t)p * nm];
      os[(int64_t)l * Nx + (int64_t)p * nm] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Full-coarsening restriction in the mixed basis (eqs. chap4_restrictionTime,
// chap4_spaceRestrictionProlongation): along each transformed axis coarse mode
// k takes ra_k r^_k + rb_k r^_{Nf-k} (ra = (1+c)/2, rb = -(1-c)/2), along the
// last axis (1/2)[1 2 1] at fine positions 2P, 2P+1, 2P+2, then the time blocks
//   fc[m, k] = sum_l R1[k,l] (.)[2m, l] + R2[k,l] (.)[2m+1, l].
// Semi coarsening is the identity in space and uses k_restrict<.., false>.
// One thread per coarse (mode, position, step).
// ---------------------------------------------------------------------------
template <typename T, int D, int Q>
__global__ void k_mrestrict(const T* __restrict__ r, T* __restrict__ fc, int nf, int nc, int Nc,
                            const T* __restrict__ ra, const T* __restrict__ rb, TimeCoef<T, Q> tc) {
  const int64_t nmc = (D == 1) ? 1 : (D == 2) ? nc : (int64_t)nc * nc;
  const int64_t nmf = (D == 1) ? 1 : (D == 2) ? nf : (int64_t)nf * nf;
  const int64_t Nxc = nmc * nc, Nxf = nmf * nf;
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (J >= Nxc || m >= Nc) return;
  const int64_t ic = J % nmc;
  const int pc = (int)(J / nmc);
  constexpr int NS = (D == 1) ? 1 : (D == 2) ? 2 : 4;
  int64_t src[NS];
  T wm[NS];
  if (D == 1) {
    src[0] = 0;
    wm[0] = T(1);
  } else if (D == 2) {
    src[0] = ic;
    src[1] = nf - 1 - ic;
    wm[0] = ra[ic];
    wm[1] = rb[ic];
  } else {
    const int cx = (int)(ic % nc), cy = (int)(ic / nc);
    const int fx[2] = {cx, nf - 1 - cx}, fy[2] = {cy, nf - 1 - cy};
    const T wx[2] = {ra[cx], rb[cx]}, wy[2] = {ra[cy], rb[cy]};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        src[(NS == 4) ? a * 2 + b : 0] = (int64_t)fy[a] * nf + fx[b];
        wm[(NS == 4) ? a * 2 + b : 0] = wy[a] * wx[b];
      }
  }
  T acc2[2][Q];
#pragma unroll
  for (int sl = 0; sl < 2; ++sl) {
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const T* rl = r + ((int64_t)(2 * m + sl) * Q + l) * Nxf + (int64_t)(2 * pc) * nmf;
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const T* b = rl + src[q];
        acc += wm[q] * (T(0.5) * (b[0] + b[2 * nmf]) + b[nmf]);
      }
      acc2[sl][l] = acc;
    }
  }
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    T acc = T(0);
#pragma unroll
    for (int l = 0; l < Q; ++l) acc += tc.R1[k * Q + l] * acc2[0][l] + tc.R2[k * Q + l] * acc2[1][l];
    fc[((int64_t)m * Q + k) * Nxc + J] = acc;
  }
}

// Full-coarsening prolongation and correction u^_f += (P e)^ in the mixed
// basis: per transformed axis fine mode i < nc takes 2 ra_i e^_i, fine mode
// i > nc takes 2 rb_j e^_j (j = nf - 1 - i), mode nc takes nothing; along the
// last axis linear interpolation (odd fine positions coincide with a coarse
// node, even ones average their two neighbours); in time R_sl^T.  The host
// passes the time blocks pre-multiplied by 2^(D-1), so the pair weights are ra,
// rb themselves.  One thread per fine (mode, position, step).
template <typename T>
__device__ __forceinline__ bool mode_source(int i, int nf, int nc, const T* __restrict__ ra,
                                            const T* __restrict__ rb, int& src, T& wgt) {
  if (i < nc) {
    src = i;
    wgt = ra[i];
    return true;
  }
  if (i > nc) {
    src = nf - 1 - i;
    wgt = rb[src];
    return true;
  }
  return false;
}

template <typename T, int D, int Q>
__global__ void k_mprolong(const T* __restrict__ ec, T* __restrict__ uf, int nf, int nc, int Nf_steps,
                           const T* __restrict__ ra, const T* __restrict__ rb, TimeCoef<T, Q> tc) {
  const int64_t nmc = (D == 1) ? 1 : (D == 2) ? nc : (int64_t)nc * nc;
  const int64_t nmf = (D == 1) ? 1 : (D == 2) ? nf : (int64_t)nf * nf;
  const int64_t Nxc = nmc * nc, Nxf = nmf * nf;
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (I >= Nxf || s >= Nf_steps) return;
  const int m = s >> 1, sl = s & 1;
  const int64_t i_f = I % nmf;
  const int pf = (int)(I / nmf);
  int64_t ic = 0;
  T wmode = T(1);
  bool has = true;
  if (D == 2) {
    int c;
    has = mode_source<T>((int)i_f, nf, nc, ra, rb, c, wmode);
    ic = c;
  } else if (D == 3) {
    int cx, cy;
    T wx, wy;
    has = mode_source<T>((int)(i_f % nf), nf, nc, ra, rb, cx, wx) &&
          mode_source<T>((int)(i_f / nf), nf, nc, ra, rb, cy, wy);
    if (has) {
      ic = (int64_t)cy * nc + cx;
      wmode = wx * wy;
    }
  }
  if (!has) return;   // the unpaired fine mode receives no correction
  T e[Q];
  const T* e0 = ec + (int64_t)m * Q * Nxc + ic;
  if (pf & 1) {
    const int64_t o = (int64_t)(pf >> 1) * nmc;
#pragma unroll
    for (int k = 0; k < Q; ++k) e[k] = wmode * e0[(int64_t)k * Nxc + o];
  } else {
    const int jl = (pf >> 1) - 1, jr = pf >> 1;
    const T wh = T(0.5) * wmode;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const T* ek = e0 + (int64_t)k * Nxc;
      T v;
      if (jl < 0) v = ek[(int64_t)jr * nmc];
      else if (jr >= nc) v = ek[(int64_t)jl * nmc];
      else v = ek[(int64_t)jl * nmc] + ek[(int64_t)jr * nmc];
      e[k] = wh * v;
    }
  }
  const T* Rb = sl ? tc.R2 : tc.R1;
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    T* dst = uf + ((int64_t)s * Q + l) * Nxf + I;
    T acc = *dst;
#pragma unroll
    for (int k = 0; k < Q; ++k) acc += Rb[k * Q + l] * e[k];
    *dst = acc;
  }
}

}  // namespace stmg
