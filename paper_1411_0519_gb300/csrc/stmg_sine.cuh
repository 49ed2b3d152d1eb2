// Kernels of the cycle with the exact block inverse, in the sine basis.
//
// The sine vectors diagonalise M_1 and K_1 (Section 3.1).  With v^ = S v
// (S = DST-I along every spatial axis, unnormalised), M_h and K_h act on
// spatial mode i = (k_1, .., k_d) as the scalars
//   lamM_i = prod_a m(k_a),  lamK_i = sum_a kappa(k_a) prod_{b != a} m(k_b),
// m(k) = h/3 (2 + cos(k pi / Nf)), kappa(k) = 2/h (1 - cos(k pi / Nf)).  So the
// space-time system decouples into one time problem per mode: the block rows
//   A_i u_s + B_i u_{s-1} = f_s,  A_i = lamM_i K_tau + lamK_i M_tau,  B_i = -lamM_i N_tau
// (q x q blocks, q = p_t + 1), and the smoother's exact block inverse is one
// q x q solve per (mode, step).  The full-coarsening transfer pairs modes along
// every axis: for linear interpolation P,
//   P phi^c_k = (1+c_k)/2 phi^f_k - (1-c_k)/2 phi^f_{Nf-k},  c_k = cos(k pi / Nf),
// so with R = P^T a coarse mode takes ra_k r^_k + rb_k r^_{Nf-k} per axis
// (ra = (1+c)/2, rb = -(1-c)/2), prolongation the same weights doubled (S P S^{-1}),
// and mode Nf/2 of each axis has no coarse partner.  The iterates of the cycle
// are the images under S of those of the same cycle written on nodes: one
// forward transform of the data and one inverse transform of the result per solve.
//
// Layout: index ((s * Q + l) * Nx + j): time step s, time dof l, spatial mode j
// (first axis fastest, Nx = n^d modes).  Consecutive threads take consecutive
// modes, so every access is coalesced; the per-mode q x q blocks are tabulated
// on the host as tab[e * Nx + j], e = k * Q + l.
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
__device__ __forceinline__ T step_trace(const T* nb, int64_t Nx, int64_t o) {
  T v = nb[o];
#pragma unroll
  for (int l = 1; l < Q; ++l) {
    const T x = nb[(int64_t)l * Nx + o];
    v = (ADJ && (l & 1)) ? v - x : v + x;
  }
  return v;
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

// Steps per thread of the pointwise kernels: a thread walks TS consecutive
// steps of one mode (forward in time for L, backward for L^T), loads the
// mode's table entries once and keeps each step's iterate in registers as the
// coupling trace of the next one.
constexpr int kStepsPerThread = 4;

// Coupling trace of the step before the first one a thread handles: forward,
// step sb - 1 of u (or the transformed initial value u0^ at sb = 0); adjoint,
// step se + 1 of u.  0 without one.
template <typename T, int Q, bool ADJ>
__device__ __forceinline__ T entry_trace(const T* u, const T* __restrict__ u0, int64_t Nx, int N, int sb, int se,
                                         int64_t j) {
  if (!ADJ) {
    if (sb > 0) return u != nullptr ? step_trace<T, Q, ADJ>(u + (int64_t)(sb - 1) * Q * Nx, Nx, j) : T(0);
    return u0 != nullptr ? u0[j] : T(0);
  }
  return (u != nullptr && se + 1 < N) ? step_trace<T, Q, ADJ>(u + (int64_t)(se + 1) * Q * Nx, Nx, j) : T(0);
}

// Trace of a step from its values held in registers.
template <typename T, int Q, bool ADJ>
__device__ __forceinline__ T reg_trace(const T (&v)[Q]) {
  T t = v[0];
#pragma unroll
  for (int l = 1; l < Q; ++l) t = (ADJ && (l & 1)) ? t - v[l] : t + v[l];
  return t;
}

// ---------------------------------------------------------------------------
// Residual r^ = f^ - L^ u^ (forward) or f^ - L^T u^ (adjoint) in the sine basis:
//   r_{s,k} = f_{s,k} - sum_l A_i[k,l] u_{s,l} + (-1)^k lamM_i sum_l u_{s-1,l}
// (adjoint: A_i^T and + lamM_i sum_l (-1)^l u_{s+1,l}); at s = 0 of the forward
// problem the trace is the transformed initial value u0^ (or 0).
// amat[e * Nx + j] = A_i[k,l] (adjoint tables hold A_i^T).  u == nullptr is a
// zero iterate.  Steps [s0, s1); one thread per (mode, kStepsPerThread
// consecutive steps).
// ---------------------------------------------------------------------------
template <typename T, int Q, bool ADJ>
__global__ void __launch_bounds__(256) k_fresidual(const T* __restrict__ f, const T* __restrict__ u,
                                                   const T* __restrict__ u0, T* __restrict__ r, int64_t Nx, int N,
                                                   int s0, int s1, const T* __restrict__ amat,
                                                   const T* __restrict__ lamM) {
  constexpr int TS = kStepsPerThread;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = s0 + blockIdx.y * TS;
  if (j >= Nx || sb >= s1) return;
  const int se = min(sb + TS, s1) - 1;
  T A[Q * Q];
#pragma unroll
  for (int e = 0; e < Q * Q; ++e) A[e] = amat[(int64_t)e * Nx + j];
  const T lam = lamM[j];
  T t = entry_trace<T, Q, ADJ>(u, u0, Nx, N, sb, se, j);
#pragma unroll
  for (int i = 0; i < TS; ++i) {
    const int s = ADJ ? se - i : sb + i;
    if (ADJ ? s < sb : s > se) break;
    T uv[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) uv[l] = (u != nullptr) ? u[((int64_t)s * Q + l) * Nx + j] : T(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int64_t idx = ((int64_t)s * Q + k) * Nx + j;
      T acc = f[idx] + ((!ADJ && (k & 1)) ? -lam : lam) * t;
#pragma unroll
      for (int l = 0; l < Q; ++l) acc -= A[k * Q + l] * uv[l];
      r[idx] = acc;
    }
    t = reg_trace<T, Q, ADJ>(uv);
  }
}

// ---------------------------------------------------------------------------
// FP64 residual of k_fresidual together with its squared l2 norm, the stopping
// quantity of Section 2 (and the norm that scales the refinement of the mixed
// form).  The squares are accumulated in double-float on the FP32 pipe from
// the residual split by integer operations (split_double), so the FP64 pipe
// does the residual only; per-block partial sums (fixed shuffle tree, then the
// warps in order) go to partial[pbase + block], reduced by k_sum_final.
// Entries outside 2^-40 ... 2^40 in magnitude (whose squares or rounding terms
// would leave the FP32 exponent range) are squared in FP64 instead; that sum
// is reduced only in blocks that have one.
// STORE32: the residual rounded to FP32 is stored in r32 (the right-hand side
// of the FP32 cycles); otherwise nothing but the partial sums is written.
// ---------------------------------------------------------------------------
// Rare path of k_fresidual_norm (entries outside the double-float range), kept
// out of line so that it is not predicated into the common path.
__device__ __noinline__ double fp64_square_add(double a, double w) { return fma(a, a, w); }
__device__ __noinline__ float fp64_narrow(double a) { return __double2float_rn(a); }

__device__ __forceinline__ dfloat df_square(dfloat x) {
  const float p = __fmul_rn(x.hi, x.hi);
  float e = __fmaf_rn(x.hi, x.hi, -p);
  e = __fmaf_rn(__fmul_rn(2.f, x.hi), x.lo, e);
  return dfloat(p, e);
}

// Block sum of a double-float per thread (all threads of the block call it);
// thread 0 receives the sum.  blockDim.x is a multiple of 32, at most 1024.
__device__ __forceinline__ dfloat df_block_sum(dfloat v) {
  __shared__ float rh[32], rl[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const dfloat o(__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off));
    v = v + o;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    rh[warp] = v.hi;
    rl[warp] = v.lo;
  }
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? dfloat(rh[lane], rl[lane]) : dfloat(0.f, 0.f);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const dfloat o(__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off));
      v = v + o;
    }
  }
  return v;
}

template <int Q, bool ADJ, bool STORE32>
__global__ void __launch_bounds__(256) k_fresidual_norm(const double* __restrict__ f, const double* __restrict__ u,
                                                        const double* __restrict__ u0, float* __restrict__ r32,
                                                        int64_t Nx, int N, int s0, int s1,
                                                        const double* __restrict__ amat,
                                                        const double* __restrict__ lamM, double* __restrict__ partial,
                                                        int64_t pbase) {
  constexpr int TS = kStepsPerThread;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = s0 + blockIdx.y * TS;
  dfloat acc(0.f, 0.f);
  double wide = 0.0;   // squares of the entries outside the double-float range
  if (j < Nx && sb < s1) {   // no early return: every thread takes part in the block sum
    const int se = min(sb + TS, s1) - 1;
    double A[Q * Q];
#pragma unroll
    for (int e = 0; e < Q * Q; ++e) A[e] = amat[(int64_t)e * Nx + j];
    const double lam = lamM[j];
    double t = entry_trace<double, Q, ADJ>(u, u0, Nx, N, sb, se, j);
    // all residuals of the thread first (every load ahead of the out-of-line rare path), then the squares
    double rv[TS][Q];
    int nsteps = 0;
#pragma unroll
    for (int i = 0; i < TS; ++i) {
      const int s = ADJ ? se - i : sb + i;
      if (ADJ ? s < sb : s > se) break;
      double uv[Q];
#pragma unroll
      for (int l = 0; l < Q; ++l) uv[l] = (u != nullptr) ? u[((int64_t)s * Q + l) * Nx + j] : 0.0;
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        double a = f[((int64_t)s * Q + k) * Nx + j] + ((!ADJ && (k & 1)) ? -lam : lam) * t;
#pragma unroll
        for (int l = 0; l < Q; ++l) a -= A[k * Q + l] * uv[l];
        rv[i][k] = a;
      }
      t = reg_trace<double, Q, ADJ>(uv);
      nsteps = i + 1;
    }
#pragma unroll
    for (int i = 0; i < TS; ++i) {
      if (i >= nsteps) break;
      const int s = ADJ ? se - i : sb + i;
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const int64_t idx = ((int64_t)s * Q + k) * Nx + j;
        const double a = rv[i][k];
        unsigned w_hi, w_lo;
        double_words(a, w_hi, w_lo);
        const int E = (int)((w_hi >> 20) & 0x7ffu);
        if (((w_hi << 1) | w_lo) == 0u || (E >= 1023 - 40 && E <= 1023 + 40)) {
          const dfloat rs = split_double(a);
          if (STORE32) r32[idx] = rs.hi;
          acc = acc + df_square(rs);
        } else {
          if (STORE32) r32[idx] = fp64_narrow(a);
          wide = fp64_square_add(a, wide);
        }
      }
    }
  }
  acc = df_block_sum(acc);
  if (__syncthreads_or(wide != 0.0)) {   // block-uniform
    __shared__ double rw[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wide += __shfl_down_sync(0xffffffffu, wide, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) rw[warp] = wide;
    __syncthreads();
    if (warp == 0) {
      wide = lane < (int)(blockDim.x >> 5) ? rw[lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) wide += __shfl_down_sync(0xffffffffu, wide, off);
    }
  }
  if (threadIdx.x == 0)
    partial[pbase + (int64_t)blockIdx.y * gridDim.x + blockIdx.x] =
        (float_bits_to_double(acc.hi) + float_bits_to_double(acc.lo)) + wide;
}

// ---------------------------------------------------------------------------
// One damped block-Jacobi step with the exact block inverse (eq. chap4_smoother,
// Section 3.1): out = (1 - w) u + w A_i^{-1} (f - B_i u_prev) per (mode, step);
// the block inverse of the block row removes A u and only the rank-one time
// coupling is applied.  DAMP: ainv holds w A_i^{-1} and out = that + wc u
// (wc = 1 - w); without DAMP ainv holds A_i^{-1}, out = A_i^{-1}(f - B_i u_prev)
// and u at the steps being written is never read, so `out` may be `u` itself
// for a single step (forward substitution of the coarsest solve, one step per
// launch).  u == nullptr is a zero iterate.  With DAMP, u and out must differ
// (steps read their neighbour's old value).  Steps [s0, s1); one thread per
// (mode, kStepsPerThread consecutive steps).
//
// The right-hand side is the same in every damped step of a level visit, so
// w A_i^{-1} f can be formed once: with the coupling vector
//   ws_i = lamM_i w A_i^{-1} sigma  (sigma_k = (-1)^k; adjoint: w A_i^{-T} 1)
// a damped step is out = wf + ws_i t + wc u, t the coupling trace — 2 FMA per
// unknown instead of q + 2.  FMODE selects the form:
//   kFromF  out from f as above (any DAMP);
//   kMakeWf (DAMP) forms wf = w A_i^{-1} f, stores it in `wf` and takes the step;
//   kUseWf  (DAMP) `f` holds wf from an earlier kMakeWf on the same f.
// ---------------------------------------------------------------------------
enum { kFromF = 0, kMakeWf = 1, kUseWf = 2 };

template <typename T, int Q, bool ADJ, bool DAMP, int FMODE = kFromF>
__global__ void __launch_bounds__(256) k_fsmooth(const T* __restrict__ f, typename PtrSel<const T, DAMP>::type u,
                                                 const T* __restrict__ u0, typename PtrSel<T, DAMP>::type out,
                                                 int64_t Nx, int N, int s0, int s1, T wc, const T* __restrict__ ainv,
                                                 const T* __restrict__ lamM, T* __restrict__ wf,
                                                 const T* __restrict__ ws) {
  static_assert(FMODE == kFromF || DAMP, "the tabulated right-hand side serves the damped step");
  constexpr int TS = kStepsPerThread;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = s0 + blockIdx.y * TS;
  if (j >= Nx || sb >= s1) return;
  const int se = min(sb + TS, s1) - 1;
  T W[FMODE == kUseWf ? 1 : Q * Q];
  if (FMODE != kUseWf) {
#pragma unroll
    for (int e = 0; e < Q * Q; ++e) W[e] = ainv[(int64_t)e * Nx + j];
  }
  T wsv[FMODE == kFromF ? 1 : Q];
  T lam = T(0);
  if (FMODE == kFromF) {
    lam = lamM[j];
  } else {
#pragma unroll
    for (int k = 0; k < Q; ++k) wsv[k] = ws[(int64_t)k * Nx + j];
  }
  T t = entry_trace<T, Q, ADJ>(u, u0, Nx, N, sb, se, j);
#pragma unroll
  for (int i = 0; i < TS; ++i) {
    const int s = ADJ ? se - i : sb + i;
    if (ADJ ? s < sb : s > se) break;
    T g[Q], uv[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const T fk = f[((int64_t)s * Q + k) * Nx + j];
      g[k] = (FMODE == kFromF) ? fk + ((!ADJ && (k & 1)) ? -lam : lam) * t : fk;
      uv[k] = (u != nullptr) ? u[((int64_t)s * Q + k) * Nx + j] : T(0);
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int64_t idx = ((int64_t)s * Q + k) * Nx + j;
      T x;
      if (FMODE == kUseWf) {
        x = g[k];
      } else {
        x = W[k * Q] * g[0];
#pragma unroll
        for (int l = 1; l < Q; ++l) x += W[k * Q + l] * g[l];
      }
      if (FMODE == kMakeWf) wf[idx] = x;
      if (FMODE != kFromF) x += wsv[k] * t;
      if (DAMP && u != nullptr) x += wc * uv[k];
      out[idx] = x;
    }
    t = (u != nullptr) ? reg_trace<T, Q, ADJ>(uv) : T(0);
  }
}

// ---------------------------------------------------------------------------
// Full-coarsening restriction in the sine basis (eqs. chap4_restrictionTime,
// chap4_spaceRestrictionProlongation): coarse mode (c_1, .., c_d) takes the
// 2^d fine modes with index c_a or nf - 1 - c_a per axis, weighted by the
// products of ra / rb, then the time blocks
//   fc[m, k] = sum_l R1[k,l] (.)[2m, l] + R2[k,l] (.)[2m+1, l].
// Semi coarsening is the identity in space and uses k_restrict<.., false>.
// One thread per coarse (mode, step).
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ int64_t pow_d(int64_t n) {
  return D == 1 ? n : D == 2 ? n * n : n * n * n;
}

template <typename T, int D, int Q>
__global__ void k_frestrict(const T* __restrict__ r, T* __restrict__ fc, int nf, int nc, int Nc,
                            const T* __restrict__ ra, const T* __restrict__ rb, TimeCoef<T, Q> tc) {
  const int64_t Nxc = pow_d<D>(nc), Nxf = pow_d<D>(nf);
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (J >= Nxc || m >= Nc) return;
  constexpr int NT = 1 << D;
  int c[3] = {0, 0, 0};
  {
    unsigned rest = (unsigned)J;   // spatial mode index: n <= 1023, so below 2^30
#pragma unroll
    for (int a = 0; a < D; ++a) {
      c[a] = (int)(rest % nc);
      rest /= nc;
    }
  }
  T wa[3], wb[3];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    wa[a] = ra[c[a]];
    wb[a] = rb[c[a]];
  }
  int64_t src[NT];
  T wm[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    int64_t idx = 0, stride = 1;
    T w = T(1);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const bool hi = (t >> a) & 1;
      idx += stride * (hi ? nf - 1 - c[a] : c[a]);
      w = (a == 0) ? (hi ? wb[a] : wa[a]) : w * (hi ? wb[a] : wa[a]);
      stride *= nf;
    }
    src[t] = idx;
    wm[t] = w;
  }
  T acc2[2][Q];
#pragma unroll
  for (int sl = 0; sl < 2; ++sl) {
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const T* rl = r + ((int64_t)(2 * m + sl) * Q + l) * Nxf;
      T acc = wm[0] * rl[src[0]];
#pragma unroll
      for (int t = 1; t < NT; ++t) acc += wm[t] * rl[src[t]];
      acc2[sl][l] = acc;
    }
  }
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    T acc = T(0);
#pragma unroll
    for (int l = 0; l <= k; ++l) acc += tc.R1[k * Q + l] * acc2[0][l] + tc.R2[k * Q + l] * acc2[1][l];
    fc[((int64_t)m * Q + k) * Nxc + J] = acc;   // R_s[k][l] = 0 for l > k (Legendre degrees)
  }
}

// Full-coarsening prolongation and correction u^_f += (P e)^ in the sine basis:
// per axis fine mode i < nc takes 2 ra_i e^_i, fine mode i > nc takes
// 2 rb_j e^_j (j = nf - 1 - i), mode nc takes nothing; in time R_sl^T.  The
// host passes the time blocks pre-multiplied by 2^d, so the pair weights are
// ra, rb themselves.  One thread per (fine mode, coarse step): both fine steps
// of the coarse step share the coarse values.
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
__global__ void k_fprolong(const T* __restrict__ ec, T* __restrict__ uf, int nf, int nc, int Nf_steps,
                           const T* __restrict__ ra, const T* __restrict__ rb, TimeCoef<T, Q> tc) {
  const int64_t Nxc = pow_d<D>(nc), Nxf = pow_d<D>(nf);
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;   // coarse step: fine steps 2m and 2m + 1
  if (I >= Nxf || 2 * m + 1 >= Nf_steps) return;
  unsigned rest = (unsigned)I;   // 32-bit: n <= 1023
  int64_t jc = 0, stride = 1;
  T w = T(1);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int src;
    T wa;
    if (!mode_source<T>((int)(rest % nf), nf, nc, ra, rb, src, wa)) return;   // unpaired mode: no correction
    rest /= nf;
    jc += stride * src;
    stride *= nc;
    w = (a == 0) ? wa : w * wa;
  }
  T e[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) e[k] = w * ec[((int64_t)m * Q + k) * Nxc + jc];
#pragma unroll
  for (int sl = 0; sl < 2; ++sl) {
    const T* Rb = sl ? tc.R2 : tc.R1;
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      T* dst = uf + ((int64_t)(2 * m + sl) * Q + l) * Nxf + I;
      T acc = *dst;
#pragma unroll
      for (int k = l; k < Q; ++k) acc += Rb[k * Q + l] * e[k];   // R_s[k][l] = 0 for l > k
      *dst = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// The coarse-grid correction fused into the first damped step after it (full
// coarsening): the step reads the uncorrected u, adds the prolongated
// correction of each fine step it touches (the mode pair weights and R_sl^T
// of k_fprolong, time blocks pre-multiplied by 2^d) and takes the damped step
// of k_fsmooth on the corrected iterate (FMODE kFromF or kUseWf).  The
// corrected iterate itself is not stored: the next step reads only `out`.
// Threads start on even fine steps, so both fine steps of a coarse step take
// the same coarse values.  Steps [s0, s1) of the fine level.
// ---------------------------------------------------------------------------
template <typename T, int Q>
__device__ __forceinline__ void fine_correction(const T* __restrict__ ec, int64_t Nxc, int64_t jc, T w, int s,
                                                const TimeCoef<T, Q>& tc, T (&corr)[Q]) {
  if (w == T(0)) {
#pragma unroll
    for (int l = 0; l < Q; ++l) corr[l] = T(0);
    return;
  }
  T e[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) e[k] = w * ec[((int64_t)(s >> 1) * Q + k) * Nxc + jc];
  const T* Rb = (s & 1) ? tc.R2 : tc.R1;
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    T acc = T(0);
#pragma unroll
    for (int k = l; k < Q; ++k) acc += Rb[k * Q + l] * e[k];   // R_s[k][l] = 0 for l > k
    corr[l] = acc;
  }
}

template <typename T, int D, int Q, bool ADJ, int FMODE>
__global__ void __launch_bounds__(256) k_fprolong_smooth(const T* __restrict__ ec, const T* __restrict__ f,
                                                         const T* __restrict__ u, const T* __restrict__ u0,
                                                         T* __restrict__ out, int nf, int nc, int N, int s0, int s1,
                                                         T wc, const T* __restrict__ ainv,
                                                         const T* __restrict__ lamM, const T* __restrict__ ws,
                                                         const T* __restrict__ ra, const T* __restrict__ rb,
                                                         TimeCoef<T, Q> tc) {
  static_assert(FMODE == kFromF || FMODE == kUseWf, "the step after the correction reads f or a ready wf");
  static_assert(kStepsPerThread % 2 == 0, "threads start on a coarse step");
  constexpr int TS = kStepsPerThread;
  const int64_t Nxf = pow_d<D>(nf), Nxc = pow_d<D>(nc);
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = s0 + blockIdx.y * TS;
  if (j >= Nxf || sb >= s1) return;
  const int se = min(sb + TS, s1) - 1;
  // coarse source mode of this fine mode and the product of its pair weights
  int64_t jc = 0;
  T w = T(1);
  {
    unsigned rest = (unsigned)j;   // 32-bit: n <= 1023
    int64_t stride = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      int src = 0;
      T wa = T(0);
      if (!mode_source<T>((int)(rest % nf), nf, nc, ra, rb, src, wa)) wa = T(0);   // unpaired: no correction
      rest /= nf;
      jc += stride * src;
      stride *= nc;
      w *= wa;
    }
  }
  T W[FMODE == kUseWf ? 1 : Q * Q];
  T wsv[FMODE == kFromF ? 1 : Q];
  T lam = T(0);
  if (FMODE == kFromF) {
#pragma unroll
    for (int e = 0; e < Q * Q; ++e) W[e] = ainv[(int64_t)e * Nxf + j];
    lam = lamM[j];
  } else {
#pragma unroll
    for (int k = 0; k < Q; ++k) wsv[k] = ws[(int64_t)k * Nxf + j];
  }
  // coupling trace of the corrected iterate at the step before the first one
  T t = T(0);
  {
    const int sn = ADJ ? se + 1 : sb - 1;
    if (sn >= 0 && sn < N) {
      T corr[Q];
      fine_correction<T, Q>(ec, Nxc, jc, w, sn, tc, corr);
      T v[Q];
#pragma unroll
      for (int l = 0; l < Q; ++l) v[l] = u[((int64_t)sn * Q + l) * Nxf + j] + corr[l];
      t = reg_trace<T, Q, ADJ>(v);
    } else if (!ADJ && u0 != nullptr) {
      t = u0[j];
    }
  }
#pragma unroll
  for (int i = 0; i < TS; ++i) {
    const int s = ADJ ? se - i : sb + i;
    if (ADJ ? s < sb : s > se) break;
    T corr[Q];
    fine_correction<T, Q>(ec, Nxc, jc, w, s, tc, corr);
    T g[Q], uv[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const T fk = f[((int64_t)s * Q + k) * Nxf + j];
      g[k] = (FMODE == kFromF) ? fk + ((!ADJ && (k & 1)) ? -lam : lam) * t : fk;
      uv[k] = u[((int64_t)s * Q + k) * Nxf + j] + corr[k];
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      T x;
      if (FMODE == kUseWf) {
        x = g[k] + wsv[k] * t;
      } else {
        x = W[k * Q] * g[0];
#pragma unroll
        for (int l = 1; l < Q; ++l) x += W[k * Q + l] * g[l];
      }
      out[((int64_t)s * Q + k) * Nxf + j] = x + wc * uv[k];
    }
    t = reg_trace<T, Q, ADJ>(uv);
  }
}

// ---------------------------------------------------------------------------
// Inexact block inverse (Remark on the V-cycle approximation in space) in the
// sine basis: one spatial V-cycle per time step for A = K_tau (x) M_h +
// M_tau (x) K_h.  The point-block Jacobi block D^x = (M_h)_jj K_tau +
// (K_h)_jj M_tau is the same at every node, so it commutes with the sine
// transform, and the spatial operator of every spatial level is A_i per mode:
// the sweep, the spatial residual and the exact one-node solve are pointwise,
// and the spatial transfers pair modes as in k_frestrict (without time blocks).
// k_fspace_solve, per (mode, step): xo = w Dinv b, the exact solve on the
// one-node spatial level (w = 1, Dinv = A^{-1}; adjoint: of the transposed
// block); the sweeps and residuals of the other levels are the fused
// k_fspace_pre / k_fspace_post.
// ---------------------------------------------------------------------------
template <typename T, int Q>
__global__ void __launch_bounds__(256) k_fspace_solve(const T* __restrict__ b, T* __restrict__ xo, int64_t Nx,
                                                      int nsteps, T w, SmallMat<T, Q> Dinv) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (j >= Nx || s >= nsteps) return;
  T r[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) r[k] = b[((int64_t)s * Q + k) * Nx + j];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    T acc = T(0);
#pragma unroll
    for (int l = 0; l < Q; ++l) acc += Dinv.a[k * Q + l] * r[l];
    xo[((int64_t)s * Q + k) * Nx + j] = w * acc;
  }
}

// The pointwise parts of one spatial V-cycle level, fused (the sweeps act per
// (mode, step) in registers):
//   k_fspace_pre:  x = nu_x damped Jacobi sweeps from x = 0 (the first one is
//                  w Dinv b), r = b - A_i x;  writes x and r.
//   k_fspace_post: x += (P e_c)^ (mode pairs, weights pscale ra / rb per axis),
//                  then nu_x sweeps;  updates x, or (upd given, the finest
//                  spatial grid of a damped smoothing step) adds wt x to upd
//                  instead of storing x.
// The same iterates as the sweeps done one launch at a time.
template <typename T, int Q>
__device__ __forceinline__ void fspace_sweeps(T (&xv)[Q], const T (&bv)[Q], const T (&A)[Q * Q],
                                              const SmallMat<T, Q>& Dinv, T w, int nu) {
  for (int it = 0; it < nu; ++it) {
    T r[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      T acc = bv[k];
#pragma unroll
      for (int l = 0; l < Q; ++l) acc -= A[k * Q + l] * xv[l];
      r[k] = acc;
    }
    T xn[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < Q; ++l) acc += Dinv.a[k * Q + l] * r[l];
      xn[k] = xv[k] + w * acc;
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) xv[k] = xn[k];
  }
}

template <typename T, int Q>
__global__ void __launch_bounds__(256) k_fspace_pre(const T* __restrict__ b, T* __restrict__ x, T* __restrict__ r,
                                                    int64_t Nx, int nsteps, T w, SmallMat<T, Q> Dinv,
                                                    const T* __restrict__ amat, int nu) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (j >= Nx || s >= nsteps) return;
  T A[Q * Q], bv[Q], xv[Q];
#pragma unroll
  for (int e = 0; e < Q * Q; ++e) A[e] = amat[(int64_t)e * Nx + j];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    bv[k] = b[((int64_t)s * Q + k) * Nx + j];
    xv[k] = T(0);
  }
  fspace_sweeps<T, Q>(xv, bv, A, Dinv, w, nu);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    T acc = bv[k];
#pragma unroll
    for (int l = 0; l < Q; ++l) acc -= A[k * Q + l] * xv[l];
    const int64_t idx = ((int64_t)s * Q + k) * Nx + j;
    x[idx] = xv[k];
    r[idx] = acc;
  }
}

template <typename T, int D, int Q>
__global__ void __launch_bounds__(256) k_fspace_post(const T* __restrict__ b, T* __restrict__ x,
                                                     const T* __restrict__ xc, int nf, int nc, int nsteps, T w,
                                                     SmallMat<T, Q> Dinv, const T* __restrict__ amat,
                                                     const T* __restrict__ ra, const T* __restrict__ rb, T pscale,
                                                     int nu, T* __restrict__ upd, T wt) {
  const int64_t Nxc = pow_d<D>(nc), Nxf = pow_d<D>(nf);
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (I >= Nxf || s >= nsteps) return;
  T A[Q * Q], bv[Q], xv[Q];
#pragma unroll
  for (int e = 0; e < Q * Q; ++e) A[e] = amat[(int64_t)e * Nxf + I];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    bv[k] = b[((int64_t)s * Q + k) * Nxf + I];
    xv[k] = x[((int64_t)s * Q + k) * Nxf + I];
  }
  unsigned rest = (unsigned)I;   // 32-bit: n <= 1023
  int64_t jc = 0, stride = 1;
  T wgt = pscale;
  bool has = true;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int src = 0;
    T wa = T(0);
    if (!mode_source<T>((int)(rest % nf), nf, nc, ra, rb, src, wa)) has = false;
    rest /= nf;
    jc += stride * src;
    stride *= nc;
    wgt = wgt * wa;
  }
  if (has) {
#pragma unroll
    for (int k = 0; k < Q; ++k) xv[k] += wgt * xc[((int64_t)s * Q + k) * Nxc + jc];
  }
  fspace_sweeps<T, Q>(xv, bv, A, Dinv, w, nu);
  if (upd != nullptr) {   // finest spatial grid of a smoothing step: u += w_t x, x itself not needed
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      T* up = upd + ((int64_t)s * Q + k) * Nxf + I;
      *up += wt * xv[k];
    }
  } else {
#pragma unroll
    for (int k = 0; k < Q; ++k) x[((int64_t)s * Q + k) * Nxf + I] = xv[k];
  }
}

// Space-only restriction in the sine basis (the spatial factor of k_frestrict,
// every step and time dof).
template <typename T, int D, int Q>
__global__ void k_fspace_restrict(const T* __restrict__ fine, T* __restrict__ coarse, int nf, int nc, int nsteps,
                                  const T* __restrict__ ra, const T* __restrict__ rb) {
  const int64_t Nxc = pow_d<D>(nc), Nxf = pow_d<D>(nf);
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (J >= Nxc || s >= nsteps) return;
  constexpr int NT = 1 << D;
  int c[3] = {0, 0, 0};
  unsigned rest = (unsigned)J;   // spatial mode index: n <= 1023, so below 2^30
#pragma unroll
  for (int a = 0; a < D; ++a) {
    c[a] = (int)(rest % nc);
    rest /= nc;
  }
  int64_t src[NT];
  T wm[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    int64_t idx = 0, stride = 1;
    T w = T(1);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const bool hi = (t >> a) & 1;
      idx += stride * (hi ? nf - 1 - c[a] : c[a]);
      w = (a == 0) ? (hi ? rb[c[a]] : ra[c[a]]) : w * (hi ? rb[c[a]] : ra[c[a]]);
      stride *= nf;
    }
    src[t] = idx;
    wm[t] = w;
  }
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const T* fl = fine + ((int64_t)s * Q + l) * Nxf;
    T acc = wm[0] * fl[src[0]];
#pragma unroll
    for (int t = 1; t < NT; ++t) acc += wm[t] * fl[src[t]];
    coarse[((int64_t)s * Q + l) * Nxc + J] = acc;
  }
}


// ===========================================================================
// Generic time degree (q > 4, up to kQmaxDyn): the same operators with q a
// runtime value.  The residual uses the structure of the Legendre K_tau,
//   K[k,l] = 1 - 2 [l < k and k - l odd],
// so (K u)_k = S - 2 sum_{l < k, k - l odd} u_l (S = sum_l u_l) and
// (K^T u)_k = S - 2 sum_{l > k, l - k odd} u_l: running sums by parity, O(q)
// per (mode, step) and no table; A_i u = lamM_i (K u) + (lamK_i tau) Mh o u.
// The smoother applies the tabulated w A_i^{-1} (q^2 per mode).  Transfers read
// the time blocks from shared memory.
// ===========================================================================
constexpr int kQmaxDyn = 48;

// Both traces of step s of a mode: sum_l u_l (forward coupling) and
// sum_l (-1)^l u_l (transposed coupling).
template <typename T>
__device__ __forceinline__ void traces_dyn(const T* us, int64_t Nx, int q, T& plain, T& alt) {
  plain = T(0);
  alt = T(0);
  for (int l = 0; l < q; ++l) {
    const T x = us[(int64_t)l * Nx];
    plain += x;
    alt = (l & 1) ? alt - x : alt + x;
  }
}

template <typename T, bool ADJ>
__device__ __forceinline__ T entry_trace_dyn(const T* u, const T* __restrict__ u0, int64_t Nx, int N, int q, int sb,
                                             int se, int64_t j) {
  T plain, alt;
  if (!ADJ) {
    if (sb > 0) {
      if (u == nullptr) return T(0);
      traces_dyn<T>(u + (int64_t)(sb - 1) * q * Nx + j, Nx, q, plain, alt);
      return plain;
    }
    return u0 != nullptr ? u0[j] : T(0);
  }
  if (u == nullptr || se + 1 >= N) return T(0);
  traces_dyn<T>(u + (int64_t)(se + 1) * q * Nx + j, Nx, q, plain, alt);
  return alt;
}

// mh[k] = M_tau[k][k] / tau = 1 / (2k + 1); lamKt[j] = lamK_j tau.
template <typename T, bool ADJ>
__global__ void __launch_bounds__(256) k_fresidual_dyn(const T* __restrict__ f, const T* __restrict__ u,
                                                       const T* __restrict__ u0, T* __restrict__ r, int64_t Nx,
                                                       int N, int s0, int s1, int q, const T* __restrict__ lamM,
                                                       const T* __restrict__ lamKt, const T* __restrict__ mh) {
  __shared__ T smh[kQmaxDyn];
  if (threadIdx.x < q) smh[threadIdx.x] = mh[threadIdx.x];
  __syncthreads();
  constexpr int TS = kStepsPerThread;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = s0 + blockIdx.y * TS;
  if (j >= Nx || sb >= s1) return;
  const int se = min(sb + TS, s1) - 1;
  const T lam = lamM[j], kt = lamKt[j];
  T t = entry_trace_dyn<T, ADJ>(u, u0, Nx, N, q, sb, se, j);
  for (int i = 0; i < TS; ++i) {
    const int s = ADJ ? se - i : sb + i;
    if (ADJ ? s < sb : s > se) break;
    if (u == nullptr) {   // zero iterate
      for (int k = 0; k < q; ++k) {
        const int64_t idx = ((int64_t)s * q + k) * Nx + j;
        r[idx] = f[idx] + ((!ADJ && (k & 1)) ? -lam : lam) * t;
      }
      t = T(0);
      continue;
    }
    const T* us = u + (int64_t)s * q * Nx + j;
    T S, alt;
    traces_dyn<T>(us, Nx, q, S, alt);
    T even = T(0), odd = T(0);   // running sums over the l already passed, by parity of l
    for (int c = 0; c < q; ++c) {
      const int k = ADJ ? q - 1 - c : c;
      const T uk = us[(int64_t)k * Nx];
      const T Ku = S - T(2) * ((k & 1) ? even : odd);
      const int64_t idx = ((int64_t)s * q + k) * Nx + j;
      r[idx] = f[idx] + ((!ADJ && (k & 1)) ? -lam : lam) * t - lam * Ku - kt * smh[k] * uk;
      if (k & 1) odd += uk; else even += uk;
    }
    t = ADJ ? alt : S;
  }
}

// FMODE as for k_fsmooth: with the tabulated wf = w A_i^{-1} f (kUseWf) a damped
// step costs O(q) per (mode, step) instead of q^2.
template <typename T, bool ADJ, bool DAMP, int FMODE = kFromF>
__global__ void __launch_bounds__(256) k_fsmooth_dyn(const T* __restrict__ f, typename PtrSel<const T, DAMP>::type u,
                                                     const T* __restrict__ u0, typename PtrSel<T, DAMP>::type out,
                                                     int64_t Nx, int N, int s0, int s1, int q, T wc,
                                                     const T* __restrict__ ainv, const T* __restrict__ lamM,
                                                     T* __restrict__ wf, const T* __restrict__ ws) {
  static_assert(FMODE == kFromF || DAMP, "the tabulated right-hand side serves the damped step");
  constexpr int TS = kStepsPerThread;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sb = s0 + blockIdx.y * TS;
  if (j >= Nx || sb >= s1) return;
  const int se = min(sb + TS, s1) - 1;
  const T lam = (FMODE == kFromF) ? lamM[j] : T(0);
  T t = entry_trace_dyn<T, ADJ>(u, u0, Nx, N, q, sb, se, j);
  T g[FMODE == kUseWf ? 1 : kQmaxDyn];
  for (int i = 0; i < TS; ++i) {
    const int s = ADJ ? se - i : sb + i;
    if (ADJ ? s < sb : s > se) break;
    if (FMODE != kUseWf)
      for (int k = 0; k < q; ++k) {
        const T fk = f[((int64_t)s * q + k) * Nx + j];
        g[k] = (FMODE == kFromF) ? fk + ((!ADJ && (k & 1)) ? -lam : lam) * t : fk;
      }
    T plain = T(0), alt = T(0);
    for (int k = 0; k < q; ++k) {
      const int64_t idx = ((int64_t)s * q + k) * Nx + j;
      T x;
      if (FMODE == kUseWf) {
        x = f[idx];
      } else {
        const T* wk = ainv + (int64_t)(k * q) * Nx + j;
        x = T(0);
        for (int l = 0; l < q; ++l) x += wk[(int64_t)l * Nx] * g[l];
      }
      if (FMODE == kMakeWf) wf[idx] = x;
      if (FMODE != kFromF) x += ws[(int64_t)k * Nx + j] * t;
      if (u != nullptr) {
        const T uk = u[idx];
        plain += uk;
        alt = (k & 1) ? alt - uk : alt + uk;
        if (DAMP) x += wc * uk;
      }
      out[idx] = x;
    }
    t = (u != nullptr) ? (ADJ ? alt : plain) : T(0);
  }
}

// Restriction (FULL: mode pairs along every axis; otherwise identity in space)
// and time blocks R1, R2 (q x q, row = coarse) staged in shared memory.
template <typename T, int D, bool FULL>
__global__ void k_frestrict_dyn(const T* __restrict__ r, T* __restrict__ fc, int nf, int nc, int Nc, int q,
                                const T* __restrict__ ra, const T* __restrict__ rb, const T* __restrict__ R1,
                                const T* __restrict__ R2) {
  extern __shared__ unsigned char smem_raw[];
  T* sR1 = reinterpret_cast<T*>(smem_raw);
  T* sR2 = sR1 + q * q;
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
    sR1[e] = R1[e];
    sR2[e] = R2[e];
  }
  __syncthreads();
  const int64_t Nxc = pow_d<D>(nc), Nxf = FULL ? pow_d<D>(nf) : Nxc;
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (J >= Nxc || m >= Nc) return;
  constexpr int NT = FULL ? (1 << D) : 1;
  int64_t src[NT];
  T wm[NT];
  if (!FULL) {
    src[0] = J;
    wm[0] = T(1);
  } else {
    int c[3] = {0, 0, 0};
    unsigned rest = (unsigned)J;   // spatial mode index: n <= 1023, so below 2^30
#pragma unroll
    for (int a = 0; a < D; ++a) {
      c[a] = (int)(rest % nc);
      rest /= nc;
    }
#pragma unroll
    for (int tt = 0; tt < NT; ++tt) {
      int64_t idx = 0, stride = 1;
      T w = T(1);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const bool hi = (tt >> a) & 1;
        idx += stride * (hi ? nf - 1 - c[a] : c[a]);
        w = (a == 0) ? (hi ? rb[c[a]] : ra[c[a]]) : w * (hi ? rb[c[a]] : ra[c[a]]);
        stride *= nf;
      }
      src[tt] = idx;
      wm[tt] = w;
    }
  }
  T a0[kQmaxDyn], a1[kQmaxDyn];
  for (int l = 0; l < q; ++l) {
    const T* r0 = r + ((int64_t)(2 * m) * q + l) * Nxf;
    const T* r1 = r + ((int64_t)(2 * m + 1) * q + l) * Nxf;
    T x0 = T(0), x1 = T(0);
#pragma unroll
    for (int tt = 0; tt < NT; ++tt) {
      x0 += wm[tt] * r0[src[tt]];
      x1 += wm[tt] * r1[src[tt]];
    }
    a0[l] = x0;
    a1[l] = x1;
  }
  for (int k = 0; k < q; ++k) {
    T acc = T(0);
    for (int l = 0; l <= k; ++l) acc += sR1[k * q + l] * a0[l] + sR2[k * q + l] * a1[l];   // R lower triangular
    fc[((int64_t)m * q + k) * Nxc + J] = acc;
  }
}

// Prolongation and correction; the host passes R1, R2 pre-multiplied by 2^d
// for full coarsening (the pair weights are then ra, rb themselves).
template <typename T, int D, bool FULL>
__global__ void k_fprolong_dyn(const T* __restrict__ ec, T* __restrict__ uf, int nf, int nc, int Nf_steps, int q,
                               const T* __restrict__ ra, const T* __restrict__ rb, const T* __restrict__ R1,
                               const T* __restrict__ R2) {
  extern __shared__ unsigned char smem_raw[];
  T* sR1 = reinterpret_cast<T*>(smem_raw);
  T* sR2 = sR1 + q * q;
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
    sR1[e] = R1[e];
    sR2[e] = R2[e];
  }
  __syncthreads();
  const int64_t Nxc = pow_d<D>(nc), Nxf = FULL ? pow_d<D>(nf) : Nxc;
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (I >= Nxf || s >= Nf_steps) return;
  const int m = s >> 1, sl = s & 1;
  int64_t jc = I;
  T w = T(1);
  if (FULL) {
    unsigned rest = (unsigned)I;   // 32-bit: n <= 1023
    int64_t stride = 1;
    jc = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      int src;
      T wa;
      if (!mode_source<T>((int)(rest % nf), nf, nc, ra, rb, src, wa)) return;   // unpaired mode
      rest /= nf;
      jc += stride * src;
      stride *= nc;
      w = (a == 0) ? wa : w * wa;
    }
  }
  T e[kQmaxDyn];
  for (int k = 0; k < q; ++k) e[k] = w * ec[((int64_t)m * q + k) * Nxc + jc];
  const T* Rb = sl ? sR2 : sR1;
  for (int l = 0; l < q; ++l) {
    T* dst = uf + ((int64_t)s * q + l) * Nxf + I;
    T acc = *dst;
    for (int k = l; k < q; ++k) acc += Rb[k * q + l] * e[k];   // R lower triangular: k >= l
    *dst = acc;
  }
}

}  // namespace stmg
