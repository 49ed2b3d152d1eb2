// Device kernels of the space-time multigrid V-cycle (FP64 and FP32).
//
// Vector layout: index ((s * Q + l) * Nx + j), time step s, time dof l,
// spatial node j = (z * n + y) * n + x with x fastest, Nx = n^D.
//
// Time matrices (Section 1) in the Legendre basis are passed by value in
// TimeCoef: K = K_tau (dimensionless), Mh = diag(M_tau) / tau, st = psi_k at
// the slab start, en = psi_k at the slab end (so N_tau = st en^T), and the
// time restriction blocks R1, R2 of eq. (chap4_restrictionTime).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace stmg {

template <typename T, int Q>
struct TimeCoef {
  T K[Q * Q];    // K_tau[k][l] row-major, k = test (row), l = trial
  T Mh[Q];       // M_tau[k][k] / tau
  T st[Q];       // psi_k(t_{n-1}^+)
  T en[Q];       // psi_k(t_n^-)
  T R1[Q * Q];   // coarse k <- fine l (first fine slab)
  T R2[Q * Q];   // coarse k <- fine l (second fine slab)
};

// ---------------------------------------------------------------------------
// Spatial stencils of M_h and K_h for Q1 (P1 in 1D), Section 1 / Section 3:
// M_1 = h/6 [1 4 1], K_1 = 1/h [-1 2 -1], M_h = (x)_a M_1,
// K_h = sum_a K_1 (axis a) (x)_{b != a} M_1.  Nodes outside [0, n) are zero
// (homogeneous Dirichlet).
// ---------------------------------------------------------------------------
// The weights are formed from h and 1/h (both passed by the host, exact since
// h = 1/(n+1) is a power of two) without a division on the device: an FP64
// division costs as much as a dozen FMAs on the FP64 pipe.
template <typename T, int D>
struct Stencil {
  // weights for offset o in {-1,0,1}: index o + 1
  T m1[3], k1[3];
  __device__ __forceinline__ Stencil(T h, T hinv) {
    m1[0] = h * T(1.0 / 6.0); m1[1] = h * T(2.0 / 3.0); m1[2] = m1[0];
    k1[0] = -hinv; k1[1] = T(2) * hinv; k1[2] = -hinv;
  }
};

// Apply M_h and K_h at node (ix, iy, iz) to a field given by an accessor
// get(j) -> T (flat spatial index j).  Out-of-range neighbours contribute 0.
template <typename T, int D, typename Get>
__device__ __forceinline__ void apply_mk(const Stencil<T, D>& S, int n, int ix, int iy, int iz,
                                         Get get, T& mu, T& ku) {
  mu = T(0);
  ku = T(0);
  if (D == 1) {
#pragma unroll
    for (int ox = -1; ox <= 1; ++ox) {
      int x = ix + ox;
      if (x < 0 || x >= n) continue;
      T v = get(x);
      mu += S.m1[ox + 1] * v;
      ku += S.k1[ox + 1] * v;
    }
  } else if (D == 2) {
#pragma unroll
    for (int oy = -1; oy <= 1; ++oy) {
      int y = iy + oy;
      if (y < 0 || y >= n) continue;
      // row pass: a = M_1 u, b = K_1 u along x
      T a = T(0), b = T(0);
#pragma unroll
      for (int ox = -1; ox <= 1; ++ox) {
        int x = ix + ox;
        if (x < 0 || x >= n) continue;
        T v = get(y * n + x);
        a += S.m1[ox + 1] * v;
        b += S.k1[ox + 1] * v;
      }
      mu += S.m1[oy + 1] * a;
      ku += S.k1[oy + 1] * a + S.m1[oy + 1] * b;
    }
  } else {
#pragma unroll
    for (int oz = -1; oz <= 1; ++oz) {
      int z = iz + oz;
      if (z < 0 || z >= n) continue;
      T am = T(0), ak = T(0);   // M_1(y) M_1(x) u, and the K part of the (x,y) plane
#pragma unroll
      for (int oy = -1; oy <= 1; ++oy) {
        int y = iy + oy;
        if (y < 0 || y >= n) continue;
        T a = T(0), b = T(0);
#pragma unroll
        for (int ox = -1; ox <= 1; ++ox) {
          int x = ix + ox;
          if (x < 0 || x >= n) continue;
          T v = get(((int64_t)z * n + y) * n + x);
          a += S.m1[ox + 1] * v;
          b += S.k1[ox + 1] * v;
        }
        am += S.m1[oy + 1] * a;
        ak += S.k1[oy + 1] * a + S.m1[oy + 1] * b;
      }
      mu += S.m1[oz + 1] * am;
      ku += S.k1[oz + 1] * am + S.m1[oz + 1] * ak;
    }
  }
}

// Only M_h (for the time-coupling trace term and the initial value).
template <typename T, int D, typename Get>
__device__ __forceinline__ T apply_m(const Stencil<T, D>& S, int n, int ix, int iy, int iz, Get get) {
  T mu = T(0);
#pragma unroll
  for (int oz = (D >= 3 ? -1 : 0); oz <= (D >= 3 ? 1 : 0); ++oz) {
    const int z = iz + oz;
    if (z < 0 || z >= (D >= 3 ? n : 1)) continue;
    T am = T(0);
#pragma unroll
    for (int oy = (D >= 2 ? -1 : 0); oy <= (D >= 2 ? 1 : 0); ++oy) {
      const int y = iy + oy;
      if (y < 0 || y >= (D >= 2 ? n : 1)) continue;
      T a = T(0);
#pragma unroll
      for (int ox = -1; ox <= 1; ++ox) {
        const int x = ix + ox;
        if (x < 0 || x >= n) continue;
        a += S.m1[ox + 1] * get(((int64_t)z * n + y) * n + x);
      }
      am += (D >= 2 ? S.m1[oy + 1] : T(1)) * a;
    }
    mu += (D >= 3 ? S.m1[oz + 1] : T(1)) * am;
  }
  return mu;
}

__device__ __forceinline__ void node_coords(int64_t j, int n, int D, int& ix, int& iy, int& iz) {
  ix = (int)(j % n);
  iy = D >= 2 ? (int)((j / n) % n) : 0;
  iz = D >= 3 ? (int)(j / ((int64_t)n * n)) : 0;
}

// ---------------------------------------------------------------------------
// Residual r = f - L u (system chap4_generalLinearSystem) or f - L^T u.
// Forward:  r_{s,k} = f_{s,k} - sum_l K[k,l] (M_h u_{s,l}) - tau Mh[k] (K_h u_{s,k})
//                     + st[k] M_h (sum_l en[l] u_{s-1,l})      (B = -N_tau (x) M_h)
//           for s = 0 the previous trace is the initial value u0 (may be null).
// Adjoint:  r_{s,k} = f_{s,k} - sum_l K[l,k] (M_h u_{s,l}) - tau Mh[k] (K_h u_{s,k})
//                     + en[k] M_h (sum_l st[l] u_{s+1,l}).
// One thread per (spatial node, time step); grid.y indexes the time step
// within [s0, s0 + gridDim.y).
// ---------------------------------------------------------------------------
template <typename T, int D, int Q, bool ADJ>
__global__ void k_residual(const T* __restrict__ f, const T* __restrict__ u,
                           const T* __restrict__ u0, T* __restrict__ r,
                           int n, int N, int s0, T tau, T h, T hinv, TimeCoef<T, Q> tc) {
  const int64_t Nx = (D == 1) ? n : (D == 2) ? (int64_t)n * n : (int64_t)n * n * n;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (j >= Nx || s >= N) return;
  int ix, iy, iz;
  node_coords(j, n, D, ix, iy, iz);
  Stencil<T, D> S(h, hinv);
  T mu[Q], ku[Q];
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const T* ul = u + ((int64_t)s * Q + l) * Nx;
    apply_mk<T, D>(S, n, ix, iy, iz, [&](int64_t q) { return ul[q]; }, mu[l], ku[l]);
  }
  T mt = T(0);
  if (!ADJ) {
    if (s > 0) {
      const T* up = u + (int64_t)(s - 1) * Q * Nx;
      mt = apply_m<T, D>(S, n, ix, iy, iz, [&](int64_t q) {
        T t = T(0);
#pragma unroll
        for (int l = 0; l < Q; ++l) t += tc.en[l] * up[(int64_t)l * Nx + q];
        return t;
      });
    } else if (u0 != nullptr) {
      mt = apply_m<T, D>(S, n, ix, iy, iz, [&](int64_t q) { return u0[q]; });
    }
  } else {
    if (s < N - 1) {
      const T* un = u + (int64_t)(s + 1) * Q * Nx;
      mt = apply_m<T, D>(S, n, ix, iy, iz, [&](int64_t q) {
        T t = T(0);
#pragma unroll
        for (int l = 0; l < Q; ++l) t += tc.st[l] * un[(int64_t)l * Nx + q];
        return t;
      });
    }
  }
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int64_t idx = ((int64_t)s * Q + k) * Nx + j;
    T acc = f[idx];
#pragma unroll
    for (int l = 0; l < Q; ++l) acc -= (ADJ ? tc.K[l * Q + k] : tc.K[k * Q + l]) * mu[l];
    acc -= tau * tc.Mh[k] * ku[k];
    acc += (ADJ ? tc.en[k] : tc.st[k]) * mt;
    r[idx] = acc;
  }
}

// ---------------------------------------------------------------------------
// The residual of k_residual for any q <= kNodeQmax, on nodes: the time
// matrices come from a table tab = [K_tau (q x q, row-major) | M_tau / tau (q) |
// psi_k(t_{n-1}^+) (q) | psi_k(t_n^-) (q)] instead of template parameters.  It
// is the node-basis residual of st_residual at high time degree, independent of
// the sine-basis kernels of the cycle; per (node, step) it keeps M_h u and K_h u
// of every time dof in local memory.
// ---------------------------------------------------------------------------
constexpr int kNodeQmax = 48;

template <typename T, int D, bool ADJ>
__global__ void k_residual_dyn(const T* __restrict__ f, const T* __restrict__ u, const T* __restrict__ u0,
                               T* __restrict__ r, int n, int N, int s0, int q, T tau, T h, T hinv,
                               const T* __restrict__ tab) {
  const int64_t Nx = (D == 1) ? n : (D == 2) ? (int64_t)n * n : (int64_t)n * n * n;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + blockIdx.y;
  if (j >= Nx || s >= N || q > kNodeQmax) return;
  const T* K = tab;
  const T* Mh = tab + q * q;
  const T* st = Mh + q;
  const T* en = st + q;
  int ix, iy, iz;
  node_coords(j, n, D, ix, iy, iz);
  Stencil<T, D> S(h, hinv);
  T mu[kNodeQmax], ku[kNodeQmax];
  for (int l = 0; l < q; ++l) {
    const T* ul = u + ((int64_t)s * q + l) * Nx;
    apply_mk<T, D>(S, n, ix, iy, iz, [&](int64_t x) { return ul[x]; }, mu[l], ku[l]);
  }
  T mt = T(0);
  const T* nb = nullptr;                       // neighbouring step (forward: s-1, adjoint: s+1)
  if (!ADJ && s > 0) nb = u + (int64_t)(s - 1) * q * Nx;
  if (ADJ && s < N - 1) nb = u + (int64_t)(s + 1) * q * Nx;
  if (nb != nullptr) {
    const T* w = ADJ ? st : en;
    mt = apply_m<T, D>(S, n, ix, iy, iz, [&](int64_t x) {
      T t = T(0);
      for (int l = 0; l < q; ++l) t += w[l] * nb[(int64_t)l * Nx + x];
      return t;
    });
  } else if (!ADJ && s == 0 && u0 != nullptr) {
    mt = apply_m<T, D>(S, n, ix, iy, iz, [&](int64_t x) { return u0[x]; });
  }
  for (int k = 0; k < q; ++k) {
    const int64_t idx = ((int64_t)s * q + k) * Nx + j;
    T acc = f[idx];
    for (int l = 0; l < q; ++l) acc -= (ADJ ? K[l * q + k] : K[k * q + l]) * mu[l];
    acc -= tau * Mh[k] * ku[k];
    acc += (ADJ ? en[k] : st[k]) * mt;
    r[idx] = acc;
  }
}

// ---------------------------------------------------------------------------
// 2D residual with a shared-memory tile (same result as k_residual<T, 2, Q, ADJ>).
// A CTA owns a TX x TY block of nodes of one time step.  It stages u (Q fields)
// and the coupling trace of the neighbouring step on the tile plus a one-node
// halo, applies the x passes of M_1 and K_1 once per staged row, then the y
// passes per node: M_h u = M_1y (M_1x u), K_h u = K_1y (M_1x u) + M_1y (K_1x u).
// ---------------------------------------------------------------------------
constexpr int kResTX = 32;
constexpr int kResTY = 8;

template <typename T, int Q, bool ADJ>
__global__ void __launch_bounds__(kResTX * kResTY) k_residual2d(const T* __restrict__ f, const T* __restrict__ u,
                                                                const T* __restrict__ u0, T* __restrict__ r,
                                                                int n, int N, int s0, T tau, T h, T hinv,
                                                                TimeCoef<T, Q> tc) {
  constexpr int HX = kResTX + 2, HY = kResTY + 2;
  __shared__ T su[Q + 1][HY][HX];        // fields 0..Q-1: u_s; field Q: coupling trace
  __shared__ T sa[Q + 1][HY][kResTX];    // M_1 along x
  __shared__ T sb[Q][HY][kResTX];        // K_1 along x
  const int s = s0 + blockIdx.z;
  const int x0 = blockIdx.x * kResTX, y0 = blockIdx.y * kResTY;
  const int tid = threadIdx.y * kResTX + threadIdx.x;
  const int64_t Nx = (int64_t)n * n;
  const T* nb = nullptr;                 // neighbouring step (forward: s-1, adjoint: s+1)
  if (!ADJ && s > 0) nb = u + (int64_t)(s - 1) * Q * Nx;
  if (ADJ && s < N - 1) nb = u + (int64_t)(s + 1) * Q * Nx;
  const bool use_u0 = !ADJ && s == 0 && u0 != nullptr;
  // stage u_s and the trace on tile + halo (zero outside the domain)
  for (int i = tid; i < HX * HY; i += kResTX * kResTY) {
    const int hy = i / HX, hx = i - hy * HX;
    const int x = x0 + hx - 1, y = y0 + hy - 1;
    const bool in = x >= 0 && x < n && y >= 0 && y < n;
    const int64_t j = (int64_t)y * n + x;
#pragma unroll
    for (int l = 0; l < Q; ++l) su[l][hy][hx] = in ? u[((int64_t)s * Q + l) * Nx + j] : T(0);
    T t = T(0);
    if (in) {
      if (nb != nullptr) {
#pragma unroll
        for (int l = 0; l < Q; ++l) t += (ADJ ? tc.st[l] : tc.en[l]) * nb[(int64_t)l * Nx + j];
      } else if (use_u0) {
        t = u0[j];
      }
    }
    su[Q][hy][hx] = t;
  }
  __syncthreads();
  const T m0 = h * T(1.0 / 6.0), m1 = h * T(2.0 / 3.0);
  const T k0 = -hinv, k1 = T(2) * hinv;
  // x passes on every staged row
  for (int i = tid; i < HY * kResTX; i += kResTX * kResTY) {
    const int hy = i / kResTX, tx = i - hy * kResTX;
#pragma unroll
    for (int l = 0; l <= Q; ++l) {
      const T a = su[l][hy][tx], b = su[l][hy][tx + 1], c = su[l][hy][tx + 2];
      sa[l][hy][tx] = m0 * (a + c) + m1 * b;
      if (l < Q) sb[l][hy][tx] = k0 * (a + c) + k1 * b;
    }
  }
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = x0 + tx, y = y0 + ty;
  if (x >= n || y >= n || s >= N) return;
  T mu[Q], ku[Q];
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const T a0 = sa[l][ty][tx], a1 = sa[l][ty + 1][tx], a2 = sa[l][ty + 2][tx];
    const T b0 = sb[l][ty][tx], b1 = sb[l][ty + 1][tx], b2 = sb[l][ty + 2][tx];
    mu[l] = m0 * (a0 + a2) + m1 * a1;
    ku[l] = k0 * (a0 + a2) + k1 * a1 + m0 * (b0 + b2) + m1 * b1;
  }
  const T mt = m0 * (sa[Q][ty][tx] + sa[Q][ty + 2][tx]) + m1 * sa[Q][ty + 1][tx];
  const int64_t j = (int64_t)y * n + x;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int64_t idx = ((int64_t)s * Q + k) * Nx + j;
    T acc = f[idx];
#pragma unroll
    for (int l = 0; l < Q; ++l) acc -= (ADJ ? tc.K[l * Q + k] : tc.K[k * Q + l]) * mu[l];
    acc -= tau * tc.Mh[k] * ku[k];
    acc += (ADJ ? tc.en[k] : tc.st[k]) * mt;
    r[idx] = acc;
  }
}

// ---------------------------------------------------------------------------
// Batched DST-I along one spatial axis, X_j = sum_{m=1}^{n} x_m sin(pi j m / Nf),
// Nf = n + 1 a power of two.  Exact block inverse of Section 3.1 (the
// eigenvectors of M_1 and K_1 are the sine vectors).
//
// Fast algorithm (O(n log n)): with x_0 = 0,
//   y_j = sin(j pi / Nf) (x_j + x_{Nf-j}) + (x_j - x_{Nf-j}) / 2,  j = 1..Nf-1, y_0 = 0;
//   the real DFT of y gives R_k = sum y_j cos(2 pi j k / Nf), I_k = sum y_j sin(2 pi j k / Nf);
//   then X_{2k} = I_k and X_{2k+1} = X_{2k-1} + R_k with X_1 = R_0 / 2.
// The real DFT of length Nf uses a complex radix-2 FFT of length Nf/2 on
// z_m = y_{2m} + i y_{2m+1} followed by the even/odd split.
//
// One warp transforms one line held in shared memory.  Rows of the x axis are
// contiguous: each warp streams its own rows (k_dst_rows).  Lines of the y / z
// axes are columns with stride n^a: a CTA stages a tile of W consecutive
// columns so that every global access is a W-wide contiguous segment
// (k_dst_cols).  Twiddles are staged in shared memory once per CTA.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Double-float arithmetic on the FP32 pipe, for the sine transforms of the
// mixed-precision form: a value is hi + lo with |lo| <= ulp(hi) / 2 (about 48
// significand bits).  Error-free transformations: Knuth's TwoSum, Dekker's
// FastTwoSum and the exact product through one FMA; the sum is the "sloppy"
// double-word addition and the product the double-word multiplication of
// Joldes, Muller and Popescu (ACM TOMS 43(2), 2017), whose absolute errors are
// a few units of 2^-48 of the operands' magnitudes -- the measure that bounds
// the error of a linear transform such as the FFT.  Exponent range is FP32's.
// ---------------------------------------------------------------------------
struct dfloat {
  float hi, lo;
  __host__ __device__ dfloat() : hi(0.f), lo(0.f) {}
  __host__ __device__ dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit dfloat(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ explicit dfloat(int v) : hi((float)v), lo(0.f) {}
};

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  return dfloat(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp)));
}
__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  const dfloat s = df_two_sum(x.hi, y.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }
__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }
__device__ __forceinline__ bool operator==(dfloat x, dfloat y) { return x.hi == y.hi && x.lo == y.lo; }

// Warp shuffles and storage conversions for the arithmetic types of the transforms.
template <typename T>
__device__ __forceinline__ T shfl_up_t(T v, int off, int width) { return __shfl_up_sync(0xffffffffu, v, off, width); }
template <>
__device__ __forceinline__ dfloat shfl_up_t<dfloat>(dfloat v, int off, int width) {
  return dfloat(__shfl_up_sync(0xffffffffu, v.hi, off, width), __shfl_up_sync(0xffffffffu, v.lo, off, width));
}
template <typename T>
__device__ __forceinline__ T shfl_t(T v, int src, int width) { return __shfl_sync(0xffffffffu, v, src, width); }
template <>
__device__ __forceinline__ dfloat shfl_t<dfloat>(dfloat v, int src, int width) {
  return dfloat(__shfl_sync(0xffffffffu, v.hi, src, width), __shfl_sync(0xffffffffu, v.lo, src, width));
}
// FP64 <-> double-float conversions by integer operations on the IEEE 754
// encodings: the conversion instructions between FP64 and FP32 issue on the
// FP64 pipe, which on this part runs at 1/64 of the FP32 rate, and a rare path
// through them would still be predicated into the common one.
// split_double: hi = x rounded to 24 significant bits (ties away from zero),
// lo = x - hi rounded to FP32 (nearest, into the subnormals where needed).  The
// pair has the FP32 exponent range: |x| below 2^-126 gives zero, |x| from 2^128
// on gives an infinite hi, NaN stays NaN.
// float_bits_to_double: exact widening of a normal FP32 value, zero and
// infinity; subnormal inputs give zero.
// The two 32-bit words of an FP64 value are read through an opaque move, so
// that the integer tests on them stay integer instructions (written on the
// 64-bit pattern, the compiler may turn them into FP64 comparisons).
__device__ __forceinline__ void double_words(double x, unsigned& hi, unsigned& lo) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
}

// eshift (split_double): an exact power-of-two scaling folded into the split,
// x 2^eshift, applied to the biased exponent of finite nonzero x; the callers
// choose it so that the data's largest magnitude lies near 1 when it would
// otherwise leave the FP32 range (see k_max_exponent).
__device__ __forceinline__ dfloat split_double(double x, int eshift = 0) {
  unsigned h32, l32;
  double_words(x, h32, l32);
  int E = (int)((h32 >> 20) & 0x7ffu);   // biased exponent
  if (E != 0 && E != 2047) E += eshift;
  const unsigned sign = h32 & 0x80000000u;
  if (E < 897) return dfloat(__uint_as_float(sign), 0.f);   // zero, or below the FP32 normal range
  if (E > 1150) {                                             // beyond FP32: infinity, or NaN
    const bool nan = E == 2047 && (((h32 & 0xfffffu) | l32) != 0u);
    return dfloat(__uint_as_float(sign | (nan ? 0x7fc00000u : 0x7f800000u)), 0.f);
  }
  const unsigned m23 = ((h32 & 0xfffffu) << 3) | (l32 >> 29);   // top 23 fraction bits
  const unsigned rem = l32 & 0x1fffffffu;                       // the 29 bits below them
  const unsigned up = rem >> 28;                                // round the magnitude up
  // hi = sign, exponent E - 1023 + 127, fraction m23 (+1: a carry moves into the exponent)
  const float hi = __uint_as_float((sign | ((unsigned)(E - 896) << 23) | m23) + up);
  // x - hi = (rem - up 2^29) 2^(E - 1075) on the magnitude: an integer m of at most
  // 28 bits, converted by FP32 arithmetic: its two 14-bit halves are exact floats
  // (2^23 + v read as a float, minus 2^23), and one FMA rounds m = hi 2^14 + lo to
  // 24 bits; the scale 2^(E - 1075) is then applied in one exact step, or (E < 949,
  // where it is not a normal float) as 2^(E - 1011) and then 2^-64, which rounds a
  // second time, into the subnormals: lo is then within one subnormal ulp (2^-149)
  // of the 24-bit rounding of x - hi, far below the pair's relative accuracy
  const int r = (int)rem - (int)(up << 29);
  const unsigned m = (unsigned)(r < 0 ? -r : r);
  const float mh = __fsub_rn(__uint_as_float(0x4B000000u | (m >> 14)), 8388608.f);
  const float ml = __fsub_rn(__uint_as_float(0x4B000000u | (m & 0x3fffu)), 8388608.f);
  const bool small = E < 949;
  const float scale = __uint_as_float((unsigned)(small ? E - 884 : E - 948) << 23);
  const float post = small ? 5.42101086242752217e-20f : 1.f;   // 2^-64
  const float lo = __fmul_rn(__fmul_rn(__fmaf_rn(mh, 16384.f, ml), scale), post);
  return dfloat(hi, ((r < 0) != (sign != 0u)) ? -lo : lo);
}
__device__ __forceinline__ double float_bits_to_double(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned sign = u & 0x80000000u;
  const unsigned m = u & 0x7fffffu;
  if (e == 0u) return __hiloint2double((int)sign, 0);   // zero (subnormals flushed)
  if (e == 0xffu) return __hiloint2double((int)(sign | 0x7ff00000u | (m ? 0x80000u : 0u)), 0);
  return __hiloint2double((int)(sign | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

// Storage conversions of the transforms.  For the double-float type the FP64
// data are scaled on the way in by 2^load_exp (exactly, in the split) and on
// the way out by 2^store_exp (one FP64 multiplication, only when store_exp is
// not zero); the other types ignore both.
template <typename T, typename S>
__device__ __forceinline__ T load_as(S x, int load_exp = 0) { return x; }
template <>
__device__ __forceinline__ dfloat load_as<dfloat, double>(double x, int load_exp) {
  return split_double(x, load_exp);
}
template <typename S, typename T>
__device__ __forceinline__ S store_as(T x, int store_exp = 0) { return x; }
template <>
__device__ __forceinline__ double store_as<double, dfloat>(dfloat x, int store_exp) {
  const double v = float_bits_to_double(x.hi) + float_bits_to_double(x.lo);   // one FP64 operation
  // 2^store_exp as an FP64 encoding; |store_exp| <= 1022 by construction (k_max_exponent)
  return store_exp == 0 ? v : v * __hiloint2double((1023 + store_exp) << 20, 0);
}

// Largest biased FP64 exponent among the finite entries of x (0 for all zeros),
// combined into *out by atomicMax (*out must start at 0).  Integer operations
// on the high word only: no FP64 instruction.
static __global__ void k_max_exponent(const double* __restrict__ x, int64_t n, unsigned* __restrict__ out) {
  unsigned m = 0u;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned hw, lw;
    double_words(x[i], hw, lw);
    const unsigned E = (hw >> 20) & 0x7ffu;
    if (E != 0x7ffu && E > m) m = E;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0 && m != 0u) atomicMax(out, m);
}

template <typename T>
struct DstTables {
  const T* sinp;   // sin(j pi / Nf), j < Nf
  const T* twc;    // cos(2 pi k / Nf), k < Nf
  const T* tws;    // sin(2 pi k / Nf)
};

// sm[0..Nf) = sin(j pi / Nf); sm[Nf..Nf+half) = cos(2 pi k / Nf); then sin(2 pi k / Nf).
template <typename T>
__device__ __forceinline__ void stage_tables(T* sm, int Nf, DstTables<T> tb) {
  const int half = Nf >> 1;
  for (int i = threadIdx.x; i < Nf; i += blockDim.x) sm[i] = tb.sinp[i];
  for (int i = threadIdx.x; i < half; i += blockDim.x) {
    sm[Nf + i] = tb.twc[i];
    sm[Nf + half + i] = tb.tws[i];
  }
}

// Transform one line in place: x[0..Nf-1] (x[0] unused on input, x[j] = x_j),
// zr/zi scratch of length Nf/2.  Output X_j in x[j], j = 1..Nf-1.
template <typename T>
__device__ void dst1_warp(T* x, T* zr, T* zi, int Nf, int logh, const T* sinp, const T* wc, const T* ws,
                          int lane) {
  const int half = Nf >> 1;
  // 1. pre-processing and packing into bit-reversed order
  for (int m = lane; m < half; m += 32) {
    const int j0 = 2 * m, j1 = 2 * m + 1;
    T y0 = T(0);
    if (j0 > 0) y0 = sinp[j0] * (x[j0] + x[Nf - j0]) + T(0.5) * (x[j0] - x[Nf - j0]);
    const T y1 = sinp[j1] * (x[j1] + x[Nf - j1]) + T(0.5) * (x[j1] - x[Nf - j1]);
    const int br = logh > 0 ? (int)(__brev((unsigned)m) >> (32 - logh)) : 0;
    zr[br] = y0;
    zi[br] = y1;
  }
  __syncwarp();
  // 2. radix-2 decimation-in-time FFT, e^{-2 pi i jk / half}
  for (int lhl = 0; lhl < logh; ++lhl) {
    const int hl = 1 << lhl;                 // half length of the butterfly group
    const int tshift = logh - lhl;           // twiddle index = jj * (Nf / (2 hl)) = jj << tshift
    for (int b = lane; b < (half >> 1); b += 32) {
      const int grp = b >> lhl, jj = b & (hl - 1);
      const int i0 = (grp << (lhl + 1)) + jj, i1 = i0 + hl;
      const T wr = wc[jj << tshift], wi = -ws[jj << tshift];   // w = e^{-2 pi i jj / (2 hl)}
      const T ar = zr[i1], ai = zi[i1];
      const T tr = wr * ar - wi * ai, ti = wr * ai + wi * ar;
      const T br0 = zr[i0], bi0 = zi[i0];
      zr[i1] = br0 - tr;
      zi[i1] = bi0 - ti;
      zr[i0] = br0 + tr;
      zi[i0] = bi0 + ti;
    }
    __syncwarp();
  }
  // 3. even/odd split: Y_k = E_k + W^k O_k, W = e^{-2 pi i / Nf};
  //    R_k -> x[2k+1], I_k = -Im Y_k -> x[2k]
  for (int k = lane; k < half; k += 32) {
    const int kc = (half - k) & (half - 1);
    const T zkr = zr[k], zki = zi[k];
    const T zcr = zr[kc], zci = -zi[kc];   // conj(Z_{half-k})
    const T er = T(0.5) * (zkr + zcr), ei = T(0.5) * (zki + zci);
    const T orr = T(0.5) * (zki - zci), oi = T(-0.5) * (zkr - zcr);   // (Zk - Zc) / (2i)
    const T wr = wc[k], wi = -ws[k];
    x[2 * k + 1] = er + (wr * orr - wi * oi);
    x[2 * k] = -(ei + (wr * oi + wi * orr));
  }
  __syncwarp();
  // 4. X_{2k+1} = sum_{k' <= k} R_k' - R_0 / 2  (warp prefix scan over half values)
  const T R0 = x[1];
  __syncwarp();
  const int per = half >= 32 ? (half >> 5) : 1;
  const int k0 = lane * per;
  T loc = T(0);
  if (k0 < half) {
    for (int c = 0; c < per; ++c) {
      loc += x[2 * (k0 + c) + 1];
      x[2 * (k0 + c) + 1] = loc;     // chunk-local inclusive prefix
    }
  }
  T incl = loc;                      // inclusive scan of chunk totals across lanes
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  const T shift = (incl - loc) - T(0.5) * R0;
  if (k0 < half) {
    for (int c = 0; c < per; ++c) x[2 * (k0 + c) + 1] += shift;
  }
  __syncwarp();
}

// x axis: `nrows` contiguous rows of length n; each CTA handles rows_per_cta
// rows, each warp its own rows with warp-private buffers.
// Shared memory: 2 Nf (tables) + nwarps * 2 Nf elements.
template <typename T>
__global__ void __launch_bounds__(256) k_dst_rows(T* __restrict__ data, int n, int logh, int64_t nrows,
                                                  int rows_per_cta, T scale, DstTables<T> tb) {
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int Nf = n + 1, half = Nf >> 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const T* sinp = sm;
  const T* wc = sm + Nf;
  const T* ws = sm + Nf + half;
  T* x = sm + 2 * Nf + (int64_t)warp * 2 * Nf;
  T* zr = x + Nf;
  T* zi = zr + half;
  stage_tables<T>(sm, Nf, tb);
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  for (int w = warp; w < rows_per_cta; w += nwarps) {
    const int64_t g = r0 + w;
    if (g >= nrows) break;                 // uniform across the warp
    T* row = data + g * n;
    for (int j = lane; j < n; j += 32) x[1 + j] = row[j];
    __syncwarp();
    dst1_warp<T>(x, zr, zi, Nf, logh, sinp, wc, ws, lane);
    for (int j = lane; j < n; j += 32) row[j] = scale * x[1 + j];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Register version of the x-axis sine transform for Nf = 2^(LP+LG+1) >= 64.
// Same algorithm as dst1_warp; the complex FFT of length H = Nf/2 = P G runs as
// a four-step FFT: a group of G threads owns one row, thread g holds the P
// points z_{g + G p}, does a P-point DFT in registers, multiplies by
// W_H^{g k1}, exchanges through shared memory, and does the G-point DFTs in
// registers:  Z_{k1 + P k2} = sum_g W_G^{g k2} W_H^{g k1} sum_p z_{g+Gp} W_P^{p k1}.
// Radix-2 stages are unrolled at compile time, so the multiplications by 1 and
// -i are skipped.  Rows are loaded and stored with whole warps (coalesced).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }
__host__ __device__ constexpr int brevc(int v, int bits) {
  return bits == 0 ? 0 : (((v & 1) << (bits - 1)) | brevc(v >> 1, bits - 1));
}

// In-place radix-2 decimation-in-frequency DFT of P points in registers,
// X_k = sum_m x_m e^{-2 pi i m k / P}; X_k ends at position brevc(k, log2 P).
// wc/ws: cos/sin(2 pi j / Nf), j < Nf, with Nf = 2^lnf >= 2 P.
template <typename T, int P>
__device__ __forceinline__ void fft_dif_reg(T (&re)[P], T (&im)[P], const T* wc, const T* ws, int lnf) {
  constexpr int LP = ilog2c(P);
#pragma unroll
  for (int st = 0; st < LP; ++st) {
    const int len = P >> st;
    const int hl = len >> 1;
    const int lsh = lnf - (LP - st);         // table index = j * (Nf / len)
#pragma unroll
    for (int b0 = 0; b0 < P; b0 += len) {
#pragma unroll
      for (int j = 0; j < hl; ++j) {
        const int i0 = b0 + j, i1 = i0 + hl;
        const T ar = re[i0], ai = im[i0], br = re[i1], bi = im[i1];
        re[i0] = ar + br;
        im[i0] = ai + bi;
        const T dr = ar - br, di = ai - bi;
        if (j == 0) {
          re[i1] = dr;
          im[i1] = di;
        } else if (4 * j == len) {             // times e^{-i pi / 2} = -i
          re[i1] = di;
          im[i1] = -dr;
        } else {
          const int idx = j << lsh;
          const T c = wc[idx], sn = ws[idx];   // e^{-2 pi i j / len} = c - i sn
          re[i1] = dr * c + di * sn;
          im[i1] = di * c - dr * sn;
        }
      }
    }
  }
}

// Shared-memory layout of k_dst_rows_reg (in elements of T), chosen so that
// every access of a warp touches distinct banks:
//  * per row one planar complex buffer (re part at 0, im part at BS): it holds
//    the input de-interleaved (x_{2k} in re[k], x_{2k+1} in im[k]), then the
//    stage-1 -> stage-2 exchange at k1 (G+1) + g, then Z_k at k + (k >> LP),
//    then the output (X_{2k} in re[k], X_{2k+1} in im[k]);
//  * BS = 16 mod 32 so re[k] and im[k] are half a bank cycle apart, and the
//    row stride RS = G mod 32 so the rows of one warp fall on disjoint banks;
//  * per CTA: sin(j pi / Nf) de-interleaved, the step-3 twiddles W_H^{g k1} at
//    k1 G + g, the split twiddles W_Nf^{g P + c} at c G + g, and
//    cos / sin(2 pi j / Nf) for j < Nf/2 (broadcast reads inside the register FFTs).
template <int LP, int LG>
struct DstRegLayout {
  static constexpr int P = 1 << LP, G = 1 << LG, H = P * G, NF = 2 * H;
  static constexpr int NEED = (H + H / P) > (P * (G + 1)) ? (H + H / P) : (P * (G + 1));
  static constexpr int BS = ((NEED + 31) / 32) * 32 + 16;
  static constexpr int RS = ((2 * BS + 31) / 32) * 32 + G;
  static constexpr int TAB = 4 * H + 4 * H + NF;   // sin +- 1/2 e/o, two twiddle tables (re, im), cos/sin half
};

// Per-CTA tables of the register sine transform (see DstRegLayout).
template <typename T, int LP, int LG>
__device__ __forceinline__ void dst_reg_stage_tables(T* sm, DstTables<T> tb) {
  using Lay = DstRegLayout<LP, LG>;
  constexpr int P = Lay::P, G = Lay::G, H = Lay::H, NF = Lay::NF;
  T* sep = sm;                // (sin(2m pi / Nf) + 1/2) / 2
  T* sem = sep + H;           // (sin(2m pi / Nf) - 1/2) / 2
  T* sop = sem + H;           // (sin((2m+1) pi / Nf) + 1/2) / 2
  T* som = sop + H;           // (sin((2m+1) pi / Nf) - 1/2) / 2
  T* t1r = som + H;
  T* t1i = t1r + H;
  T* t3r = t1i + H;           // W_Nf^{g P + c} at c G + g
  T* t3i = t3r + H;
  T* wc = t3i + H;
  T* ws = wc + NF / 2;
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    const T s0 = tb.sinp[2 * i], s1 = tb.sinp[2 * i + 1];
    sep[i] = T(0.5) * (s0 + T(0.5));   // the split's factor 1/2, folded into the (linear) pre-processing
    sem[i] = T(0.5) * (s0 - T(0.5));
    sop[i] = T(0.5) * (s1 + T(0.5));
    som[i] = T(0.5) * (s1 - T(0.5));
    const int k1 = i / G, gg = i - k1 * G;                 // t1 entry (k1, g)
    const int j1 = (2 * gg * k1) & (NF - 1);               // W_H^{g k1} = e^{-2 pi i (2 g k1) / Nf}
    t1r[i] = tb.twc[j1];
    t1i[i] = -tb.tws[j1];
    const int c = i / G, g3 = i - c * G;                   // t3 entry (c, g): W_Nf^{g P + c}
    const int j3 = g3 * P + c;
    t3r[i] = tb.twc[j3];
    t3i[i] = -tb.tws[j3];
  }
  for (int i = threadIdx.x; i < NF / 2; i += blockDim.x) {
    wc[i] = tb.twc[i];
    ws[i] = tb.tws[i];
  }
}

// Sine transform of one row by the G threads of a group (g = rank in the
// group).  On entry bre[k] = x_{2k}, bim[k] = x_{2k+1} (x_0 = 0); on exit
// bre[k] = X_{2k}, bim[k] = X_{2k+1}.  Only __syncwarp is used: a group never
// spans two warps.  The pre-processing is written as
// y_j = x_j (s_j + 1/2) + x_{Nf-j} (s_j - 1/2) and the even/odd split as
// Y_k = 1/2 [A + (w_i - i w_r) B], A = Z_k + conj Z_{H-k}, B = Z_k - conj Z_{H-k},
// W^k = w_r + i w_i, to save FP64 instructions; the split's factor 1/2 is
// applied to the pre-processing weights instead (every step in between is
// linear), so the split is two FMA per output after A and B.
template <typename T, int LP, int LG>
__device__ __forceinline__ void dst_reg_row(T* bre, T* bim, int g, const T* sm) {
  using Lay = DstRegLayout<LP, LG>;
  constexpr int P = Lay::P, G = Lay::G, H = Lay::H, NF = Lay::NF, LNF = LP + LG + 1;
  const T* sep = sm;
  const T* sem = sep + H;
  const T* sop = sem + H;
  const T* som = sop + H;
  const T* t1r = som + H;
  const T* t1i = t1r + H;
  const T* t3r = t1i + H;
  const T* t3i = t3r + H;
  const T* wc = t3i + H;
  const T* ws = wc + NF / 2;
  T re[P], im[P];
  // 1. pre-processing fused with the stage-1 gather, z_m = y_{2m} + i y_{2m+1}, m = g + G p
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int m = g + G * p;
    const T a0 = bre[m], b0 = bre[(H - m) & (H - 1)];      // x_{2m}, x_{Nf - 2m}
    const T a1 = bim[m], b1 = bim[H - 1 - m];              // x_{2m+1}, x_{Nf - 2m - 1}
    re[p] = (m == 0) ? T(0) : a0 * sep[m] + b0 * sem[m];
    im[p] = a1 * sop[m] + b1 * som[m];
  }
  __syncwarp();
  // 2. P-point DFTs over p
  fft_dif_reg<T, P>(re, im, wc, ws, LNF);
  // 3. twiddle and exchange at k1 (G + 1) + g (k1 = 0 has the twiddle 1)
#pragma unroll
  for (int pos = 0; pos < P; ++pos) {
    const int k1 = brevc(pos, LP);
    if (k1 == 0) {
      bre[g] = re[pos];
      bim[g] = im[pos];
    } else {
      const T c = t1r[k1 * G + g], sn = t1i[k1 * G + g];   // W = c + i sn
      bre[k1 * (G + 1) + g] = re[pos] * c - im[pos] * sn;
      bim[k1 * (G + 1) + g] = re[pos] * sn + im[pos] * c;
    }
  }
  __syncwarp();
  // 4. G-point DFTs over g for k1 = g + G i (results kept in registers)
  T zr2[P], zi2[P];
#pragma unroll
  for (int i = 0; i < P / G; ++i) {
    const int k1 = g + G * i;
    T r2[G], i2[G];
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
      r2[gg] = bre[k1 * (G + 1) + gg];
      i2[gg] = bim[k1 * (G + 1) + gg];
    }
    fft_dif_reg<T, G>(r2, i2, wc, ws, LNF);
#pragma unroll
    for (int pos = 0; pos < G; ++pos) {
      zr2[i * G + pos] = r2[pos];
      zi2[i * G + pos] = i2[pos];
    }
  }
  __syncwarp();
  // Z_{k1 + P k2} at k + (k >> LP)
#pragma unroll
  for (int i = 0; i < P / G; ++i) {
#pragma unroll
    for (int pos = 0; pos < G; ++pos) {
      const int k2 = brevc(pos, LG);
      const int k = g + G * i + P * k2;
      bre[k + k2] = zr2[i * G + pos];
      bim[k + k2] = zi2[i * G + pos];
    }
  }
  __syncwarp();
  // 5. even/odd split for k = g P + c: R_k (prefix-summed) and I_k
  T Rk[P], Ik[P];
#pragma unroll
  for (int c = 0; c < P; ++c) {
    const int k = g * P + c;
    const int kc = (H - k) & (H - 1);
    const T zkr = bre[k + (k >> LP)], zki = bim[k + (k >> LP)];
    const T zcr = bre[kc + (kc >> LP)], zcm = bim[kc + (kc >> LP)];   // Z_{H-k} = zcr + i zcm
    const T ar = zkr + zcr, ai = zki - zcm;                          // A = Z_k + conj Z_{H-k}
    const T br = zkr - zcr, bi = zki + zcm;                          // B = Z_k - conj Z_{H-k}
    const T hr = t3r[c * G + g], hi = t3i[c * G + g];                // W^k
    Rk[c] = (ar + hi * br) + hr * bi;                                // Re Y_k
    Ik[c] = (hr * br - ai) - hi * bi;                                // -Im Y_k
  }
  __syncwarp();
  T loc = T(0);
#pragma unroll
  for (int c = 0; c < P; ++c) {
    loc += Rk[c];
    Rk[c] = loc;
  }
  T incl = loc;
#pragma unroll
  for (int off = 1; off < G; off <<= 1) {
    const T v = shfl_up_t<T>(incl, off, G);
    if (g >= off) incl += v;
  }
  const T R0 = shfl_t<T>(Rk[0], 0, G);      // thread 0's first prefix is R_0
  const T shift = (incl - loc) - T(0.5) * R0;
#pragma unroll
  for (int c = 0; c < P; ++c) {
    const int k = g * P + c;
    bre[k] = Ik[c];             // X_{2k}
    bim[k] = Rk[c] + shift;     // X_{2k+1}
  }
}

// x-axis sine transform of nrows contiguous rows: data <- scale * DST(data).
// Reads src_data, writes dst_data (the same buffer for an in-place pass; a CTA
// reads all of its rows before it writes any).  SIN / SOUT: element types read
// and written (8 bytes each for the double-float transforms, which keep float
// pairs between their axis passes and convert only on the first read and the
// last write).
template <typename T, int LP, int LG, typename SIN = T, typename SOUT = SIN>
__global__ void __launch_bounds__(256) k_dst_rows_reg(const void* src_data, void* dst_data, int n, int64_t nrows,
                                                      T scale, DstTables<T> tb, int load_exp = 0,
                                                      int store_exp = 0) {
  using Lay = DstRegLayout<LP, LG>;
  constexpr int BS = Lay::BS, RS = Lay::RS;
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* rows = sm + Lay::TAB;
  const int tid = threadIdx.x;
  const int rpc = blockDim.x >> LG;
  dst_reg_stage_tables<T, LP, LG>(sm, tb);
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int rcount = (int)((nrows - r0) < rpc ? (nrows - r0) : rpc);
  const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int r = warp; r < rcount; r += nw) {     // coalesced, de-interleaved load
    const SIN* src = reinterpret_cast<const SIN*>(src_data) + (r0 + r) * n;
    T* br = rows + r * RS;
    for (int c = lane; c < n; c += 32) {
      const int j = c + 1;
      br[(j & 1) * BS + (j >> 1)] = load_as<T, SIN>(src[c], load_exp);
    }
    if (lane == 0) br[0] = T(0);
  }
  __syncthreads();
  const int rr = tid >> LG, g = tid & (Lay::G - 1);
  dst_reg_row<T, LP, LG>(rows + rr * RS, rows + rr * RS + BS, g, sm);   // rows >= rcount are not stored
  __syncthreads();
  const bool unit = scale == T(1);
  for (int r = warp; r < rcount; r += nw) {
    SOUT* dst = reinterpret_cast<SOUT*>(dst_data) + (r0 + r) * n;
    const T* br = rows + r * RS;
    for (int c = lane; c < n; c += 32) {
      const int j = c + 1;
      const T v = br[(j & 1) * BS + (j >> 1)];
      dst[c] = store_as<SOUT, T>(unit ? v : scale * v, store_exp);
    }
  }
}

// y / z axis with the register transform: line g = (outer, in), in < inner,
// starts at outer * inner * n + in and has stride inner.  A CTA takes the
// threads / G consecutive lines g (consecutive x positions, so each load and
// store of a line position is one contiguous segment), de-interleaves them into
// the per-line buffers of k_dst_rows_reg, transforms each line with a group of
// G threads and writes them back.  Shared memory: the k_dst_rows_reg layout
// followed by one int64 line base per line.
template <typename T, int LP, int LG, typename SIN = T, typename SOUT = SIN>
__global__ void __launch_bounds__(256) k_dst_cols_reg(const void* src_data, void* dst_data, int n, int64_t nlines,
                                                      int64_t inner, T scale, DstTables<T> tb, int load_exp = 0,
                                                      int store_exp = 0) {
  using Lay = DstRegLayout<LP, LG>;
  constexpr int BS = Lay::BS, RS = Lay::RS;
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* rows = sm + Lay::TAB;
  const int tid = threadIdx.x;
  const int rpc = blockDim.x >> LG;
  int64_t* base = reinterpret_cast<int64_t*>(rows + (int64_t)rpc * RS);
  dst_reg_stage_tables<T, LP, LG>(sm, tb);
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int rcount = (int)((nlines - r0) < rpc ? (nlines - r0) : rpc);
  if (tid < rcount) {
    const int64_t g = r0 + tid;
    const int64_t outer = g / inner, in = g - outer * inner;
    base[tid] = outer * inner * n + in;
  }
  __syncthreads();
  for (int idx = tid; idx < rpc * n; idx += blockDim.x) {   // consecutive threads: consecutive lines
    const int r = idx % rpc, c = idx / rpc;
    if (r < rcount) {
      const int j = c + 1;
      rows[r * RS + (j & 1) * BS + (j >> 1)] =
          load_as<T, SIN>(reinterpret_cast<const SIN*>(src_data)[base[r] + (int64_t)c * inner], load_exp);
    }
  }
  if (tid < rpc) rows[tid * RS] = T(0);
  __syncthreads();
  const int rr = tid >> LG, g = tid & (Lay::G - 1);
  dst_reg_row<T, LP, LG>(rows + rr * RS, rows + rr * RS + BS, g, sm);   // lines >= rcount are not stored
  __syncthreads();
  const bool unit = scale == T(1);
  for (int idx = tid; idx < rpc * n; idx += blockDim.x) {
    const int r = idx % rpc, c = idx / rpc;
    if (r < rcount) {
      const int j = c + 1;
      const T v = rows[r * RS + (j & 1) * BS + (j >> 1)];
      reinterpret_cast<SOUT*>(dst_data)[base[r] + (int64_t)c * inner] =
          store_as<SOUT, T>(unit ? v : scale * v, store_exp);
    }
  }
}

// y / z axis: line g = (outer, in), in < inner, starts at outer * inner * n + in
// and has stride inner.  Each CTA stages W consecutive lines.
// Shared memory: 2 Nf (tables) + W int64 bases + W (Nf + 1) tile + nwarps Nf.
template <typename T, int W>
__global__ void __launch_bounds__(256) k_dst_cols(T* __restrict__ data, int n, int logh, int64_t nlines,
                                                  int64_t inner, T scale, DstTables<T> tb) {
  extern __shared__ unsigned char smem_raw[];
  const int Nf = n + 1, half = Nf >> 1, ld = Nf + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  int64_t* base = reinterpret_cast<int64_t*>(smem_raw);
  T* sm = reinterpret_cast<T*>(smem_raw + W * sizeof(int64_t));
  const T* sinp = sm;
  const T* wc = sm + Nf;
  const T* ws = sm + Nf + half;
  T* tile = sm + 2 * Nf;
  T* zr = tile + (int64_t)W * ld + (int64_t)warp * Nf;
  T* zi = zr + half;
  const int64_t g0 = (int64_t)blockIdx.x * W;
  const int wcount = (int)((nlines - g0) < W ? (nlines - g0) : W);
  if (threadIdx.x < W && (int)threadIdx.x < wcount) {
    const int64_t g = g0 + threadIdx.x;
    const int64_t outer = g / inner, in = g - outer * inner;
    base[threadIdx.x] = outer * inner * n + in;
  }
  stage_tables<T>(sm, Nf, tb);
  __syncthreads();
  for (int idx = threadIdx.x; idx < W * n; idx += blockDim.x) {
    const int w = idx % W, j = idx / W;
    if (w < wcount) tile[w * ld + 1 + j] = data[base[w] + (int64_t)j * inner];
  }
  __syncthreads();
  for (int w = warp; w < wcount; w += nwarps) dst1_warp<T>(tile + w * ld, zr, zi, Nf, logh, sinp, wc, ws, lane);
  __syncthreads();
  for (int idx = threadIdx.x; idx < W * n; idx += blockDim.x) {
    const int w = idx % W, j = idx / W;
    if (w < wcount) data[base[w] + (int64_t)j * inner] = scale * tile[w * ld + 1 + j];
  }
}

// ---------------------------------------------------------------------------
// Restriction (eqs. chap4_restrictionTime, chap4_spaceRestrictionProlongation):
// fc[m, k, J] = sum_l R1[k,l] (Rx r)[2m, l, J] + R2[k,l] (Rx r)[2m+1, l, J],
// Rx = identity (semi) or (x)_a (1/2)[1 2 1] at fine nodes 2J, 2J+1, 2J+2 (0-based,
// full).  One thread per coarse (node, step).
// ---------------------------------------------------------------------------
template <typename T, int D, int Q, bool FULL>
__global__ void k_restrict(const T* __restrict__ r, T* __restrict__ fc, int nf, int nc, int Nc,
                           TimeCoef<T, Q> tc) {
  const int64_t Nxc = (D == 1) ? nc : (D == 2) ? (int64_t)nc * nc : (int64_t)nc * nc * nc;
  const int64_t Nxf = (D == 1) ? nf : (D == 2) ? (int64_t)nf * nf : (int64_t)nf * nf * nf;
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (J >= Nxc || m >= Nc) return;
  int jx, jy, jz;
  node_coords(J, nc, D, jx, jy, jz);
  T a[2][Q];
#pragma unroll
  for (int sl = 0; sl < 2; ++sl) {
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const T* rl = r + ((int64_t)(2 * m + sl) * Q + l) * Nxf;
      T acc = T(0);
      if (!FULL) {
        acc = rl[J];
      } else {
        const T w[3] = {T(0.5), T(1), T(0.5)};
        if (D == 1) {
#pragma unroll
          for (int ox = 0; ox < 3; ++ox) acc += w[ox] * rl[2 * jx + ox];
        } else if (D == 2) {
#pragma unroll
          for (int oy = 0; oy < 3; ++oy)
#pragma unroll
            for (int ox = 0; ox < 3; ++ox)
              acc += w[oy] * w[ox] * rl[(int64_t)(2 * jy + oy) * nf + 2 * jx + ox];
        } else {
#pragma unroll
          for (int oz = 0; oz < 3; ++oz)
#pragma unroll
            for (int oy = 0; oy < 3; ++oy)
#pragma unroll
              for (int ox = 0; ox < 3; ++ox)
                acc += w[oz] * w[oy] * w[ox] *
                       rl[((int64_t)(2 * jz + oz) * nf + 2 * jy + oy) * nf + 2 * jx + ox];
        }
      }
      a[sl][l] = acc;
    }
  }
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    T acc = T(0);
#pragma unroll
    for (int l = 0; l < Q; ++l) acc += tc.R1[k * Q + l] * a[0][l] + tc.R2[k * Q + l] * a[1][l];
    fc[((int64_t)m * Q + k) * Nxc + J] = acc;
  }
}

// Prolongation and correction u_f += P e_c, P = R^T: fine step 2m+sl, dof l gets
// sum_k R_sl[k,l] (Px e)[m, k, I]; Px = Rx^T is linear interpolation (fine node
// 2J+1 <- coarse J with weight 1, fine node 2J <- coarse J-1, J with weight 1/2).
// Per axis a fine index i maps to at most two coarse indices (c0, w0), (c1, w1);
// a missing neighbour gets weight 0 and a clamped index.
__device__ __forceinline__ void interp_pair(int i, int nc, int& c0, int& c1, float& w0, float& w1) {
  if (i & 1) {
    c0 = c1 = (i - 1) >> 1;
    w0 = 1.0f;
    w1 = 0.0f;
  } else {
    const int jl = (i >> 1) - 1, jr = i >> 1;
    c0 = jl >= 0 ? jl : 0;
    w0 = jl >= 0 ? 0.5f : 0.0f;
    c1 = jr < nc ? jr : nc - 1;
    w1 = jr < nc ? 0.5f : 0.0f;
  }
}

template <typename T, int D, int Q, bool FULL>
__global__ void k_prolong(const T* __restrict__ ec, T* __restrict__ uf, int nf, int nc, int Nf_steps,
                          TimeCoef<T, Q> tc) {
  const int64_t Nxc = (D == 1) ? nc : (D == 2) ? (int64_t)nc * nc : (int64_t)nc * nc * nc;
  const int64_t Nxf = (D == 1) ? nf : (D == 2) ? (int64_t)nf * nf : (int64_t)nf * nf * nf;
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (I >= Nxf || s >= Nf_steps) return;
  const int m = s >> 1, sl = s & 1;
  int ix, iy, iz;
  node_coords(I, nf, D, ix, iy, iz);
  int cx0 = 0, cx1 = 0, cy0 = 0, cy1 = 0, cz0 = 0, cz1 = 0;
  float wx0 = 1.f, wx1 = 0.f, wy0 = 1.f, wy1 = 0.f, wz0 = 1.f, wz1 = 0.f;
  if (FULL) {
    interp_pair(ix, nc, cx0, cx1, wx0, wx1);
    if (D >= 2) interp_pair(iy, nc, cy0, cy1, wy0, wy1);
    if (D >= 3) interp_pair(iz, nc, cz0, cz1, wz0, wz1);
  }
  T e[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const T* ek = ec + ((int64_t)m * Q + k) * Nxc;
    T acc;
    if (!FULL) {
      acc = ek[I];
    } else if (D == 1) {
      acc = T(wx0) * ek[cx0] + T(wx1) * ek[cx1];
    } else if (D == 2) {
      const T r0 = T(wx0) * ek[(int64_t)cy0 * nc + cx0] + T(wx1) * ek[(int64_t)cy0 * nc + cx1];
      const T r1 = T(wx0) * ek[(int64_t)cy1 * nc + cx0] + T(wx1) * ek[(int64_t)cy1 * nc + cx1];
      acc = T(wy0) * r0 + T(wy1) * r1;
    } else {
      T pz[2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int64_t zoff = (int64_t)(a ? cz1 : cz0) * nc;
        const T r0 = T(wx0) * ek[(zoff + cy0) * nc + cx0] + T(wx1) * ek[(zoff + cy0) * nc + cx1];
        const T r1 = T(wx0) * ek[(zoff + cy1) * nc + cx0] + T(wx1) * ek[(zoff + cy1) * nc + cx1];
        pz[a] = T(wy0) * r0 + T(wy1) * r1;
      }
      acc = T(wz0) * pz[0] + T(wz1) * pz[1];
    }
    e[k] = acc;
  }
  const T* Rb = sl ? tc.R2 : tc.R1;
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) acc += Rb[k * Q + l] * e[k];
    uf[((int64_t)s * Q + l) * Nxf + I] += acc;
  }
}

// M_h applied to sum_k c[k] v_{0,k} (block 0 of a space-time vector): gradient of
// the initial-value term, grad_u0 = M_h sum_k psi_k(t_0^+) lambda_{1,k}.
template <typename T, int D, int Q>
__global__ void k_ic_gradient(const T* __restrict__ lam, T* __restrict__ g, int n, T h, TimeCoef<T, Q> tc) {
  const int64_t Nx = (D == 1) ? n : (D == 2) ? (int64_t)n * n : (int64_t)n * n * n;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Nx) return;
  int ix, iy, iz;
  node_coords(j, n, D, ix, iy, iz);
  Stencil<T, D> S(h, T(0));   // M_h only
  g[j] = apply_m<T, D>(S, n, ix, iy, iz, [&](int64_t q) {
    T t = T(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) t += tc.st[k] * lam[(int64_t)k * Nx + q];
    return t;
  });
}

// The same for a runtime number q of time dofs (psi_k(t_0^+) = (-1)^k).
template <typename T, int D>
__global__ void k_ic_gradient_dyn(const T* __restrict__ lam, T* __restrict__ g, int n, T h, int q) {
  const int64_t Nx = (D == 1) ? n : (D == 2) ? (int64_t)n * n : (int64_t)n * n * n;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Nx) return;
  int ix, iy, iz;
  node_coords(j, n, D, ix, iy, iz);
  Stencil<T, D> S(h, T(0));   // M_h only
  g[j] = apply_m<T, D>(S, n, ix, iy, iz, [&](int64_t nd) {
    T t = T(0);
    for (int k = 0; k < q; ++k) t = (k & 1) ? t - lam[(int64_t)k * Nx + nd] : t + lam[(int64_t)k * Nx + nd];
    return t;
  });
}

// q x q matrix passed by value (the inverted node block of the inexact block inverse).
template <typename T, int Q>
struct SmallMat {
  T a[Q * Q];
};

// ---------------------------------------------------------------------------
// Elementwise helpers.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_axpy(T* __restrict__ y, const T* __restrict__ x, T a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

template <typename T>
__global__ void k_axpby(T* __restrict__ y, const T* __restrict__ x, T a, T b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * y[i] + b * x[i];
}

template <typename T>
__global__ void k_fill(T* __restrict__ y, T v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = v;
}

template <typename T>
__global__ void k_scale_copy(T* __restrict__ y, const T* __restrict__ x, T a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// y32 = (float)(a * x64)
static __global__ void k_cast_down(float* __restrict__ y, const double* __restrict__ x, double a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)(a * x[i]);
}

// y64 += a * (double)x32
static __global__ void k_axpy_up(double* __restrict__ y, const float* __restrict__ x, double a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * (double)x[i];
}

// y64 = (double)x32
static __global__ void k_cast_up(double* __restrict__ y, const float* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// ---------------------------------------------------------------------------
// Deterministic two-stage sum of squares: stage 1 writes one partial per block
// (fixed grid, fixed per-thread ranges, fixed tree), stage 2 reduces the
// partials in one block.  Accumulation in FP64.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_sumsq_partial(const T* __restrict__ x, int64_t n, double* __restrict__ partial) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)x[i];
    acc += v * v;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) partial[blockIdx.x] = acc;
  }
}

static __global__ void k_sum_final(const double* __restrict__ partial, int np, double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) out[0] = acc;
  }
}

}  // namespace stmg
