// Host side of the space-time multigrid library: handle, level hierarchy,
// V-cycle driver, solve loops and the C ABI declared in include/stmg.h.
//
// Method: Gander & Neumueller, arXiv:1411.0519.  Section 2 (V-cycle, damped
// block Jacobi, P = R^T, exact coarsest solve), Section 3 (exact block inverse,
// transfers), Section 4 (coarsening rule mu_L >= mu*).  The cycle runs in the
// sine basis of every spatial axis (see stmg_sine.cuh): the data are
// transformed once at the entry of a solve and the solution once at the exit.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "stmg.h"
#include "stmg_kernels.cuh"
#include "stmg_tc.cuh"
#include "stmg_sine.cuh"
#include "stmg_host_time.h"

using stmg::TimeCoef;

namespace {

constexpr int kQfix = 4;   // q <= kQfix: compile-time q kernels; above: the generic-q kernels

using namespace stmg_host;

template <typename T, int Q>
TimeCoef<T, Q> to_coef(const HostTime& t) {
  TimeCoef<T, Q> c{};
  for (int i = 0; i < Q * Q; ++i) {
    c.K[i] = (T)t.K[i];
    c.R1[i] = (T)t.R1[i];
    c.R2[i] = (T)t.R2[i];
  }
  for (int i = 0; i < Q; ++i) {
    c.Mh[i] = (T)t.Mh[i];
    c.st[i] = (T)t.st[i];
    c.en[i] = (T)t.en[i];
  }
  return c;
}

template <typename T>
struct Tables {
  T* sinp = nullptr;  // sin(j pi / Nf), j = 0..Nf-1
  T* twc = nullptr;   // cos(2 pi k / Nf), k = 0..Nf-1
  T* tws = nullptr;   // sin(2 pi k / Nf)
  // per spatial mode (sine basis), tab[e * Nx + j], e = k * q + l; [0] forward, [1] transposed
  T* amat[2] = {nullptr, nullptr};   // A_i = lamM_i K_tau + lamK_i M_tau
  T* ainv[2] = {nullptr, nullptr};   // A_i^{-1}
  T* ainvw[2] = {nullptr, nullptr};  // w A_i^{-1} (damped smoother)
  T* ws[2] = {nullptr, nullptr};     // coupling vectors lamM_i w A_i^{-1} sigma of the damped step on wf (q per mode)
  T* lamM = nullptr;                 // lamM_i (coupling B_i = -lamM_i N_tau)
  T* lamKt = nullptr;                // lamK_i tau (generic-q residual)
  T* ra = nullptr;     // full-coarsening pair weights to level L-1: (1 + c_k) / 2
  T* rb = nullptr;     //                                             -(1 - c_k) / 2
};

template <typename T>
struct Vecs {
  T* u = nullptr;
  T* f = nullptr;
  T* r = nullptr;
  T* wf = nullptr;   // w A_i^{-1} f of the level's current right-hand side (damped steps on wf)
};

// One spatial level of the inexact block inverse: iterate x, right-hand side
// b (not owned on the finest spatial level) and a ping-pong / residual buffer t.
template <typename T>
struct SpaceLvl {
  int n = 0;
  double h = 0;
  int64_t Nx = 0;
  T* x = nullptr;
  T* b = nullptr;
  T* t = nullptr;
  T* amat[2] = {nullptr, nullptr};   // A_i per mode of this spatial grid (forward, transposed)
  T* ra = nullptr;                   // mode-pair weights to the next coarser spatial grid
  T* rb = nullptr;
};

struct Level {
  int N = 0, n = 0;
  double tau = 0, h = 0, mu = 0;
  int coarsen_full = 0;   // how this level is restricted to level L-1 (L >= 1)
  int64_t Nx = 0, ndof = 0;
  Vecs<double> v64;
  Vecs<float> v32;
  Tables<double> t64;
  Tables<float> t32;
  stmg::DstTables<stmg::dfloat> tdf{nullptr, nullptr, nullptr};   // finest level, mixed form: double-float transforms
  uint8_t* tcS = nullptr;   // FP16 digits of S / 2 for the tensor-core transform (made on first use)
  std::vector<SpaceLvl<double>> sp64;   // spatial hierarchy of the inexact block inverse
  std::vector<SpaceLvl<float>> sp32;
};

}  // namespace

struct st_handle {
  int d = 0, p_t = 0, q = 0, N = 0;
  double T = 0;
  st_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<Level> levels;   // 0 = coarsest
  HostTime tm{};
  std::vector<void*> allocs;
  size_t bytes = 0;
  double* partial = nullptr;   // norm partial sums
  int64_t npartial = 0;
  double* dnorm = nullptr;     // device result of a norm
  double* hnorm = nullptr;     // pinned host copy (two words: the norm, then the tensor-core error flag)
  // tensor-core sine transform: digit planes and line exponents of one batch, device error flag
  uint8_t* tcD = nullptr;
  int64_t tc_cap = 0;   // lines the digit planes hold (at least one field's lines along an axis)
  int* tcE = nullptr;
  int* tcErr = nullptr;
  int num_sms = 152;
  unsigned* dmaxexp = nullptr;   // mixed form: largest biased exponent of the entry data (device)
  int df_shift = 0;              // mixed form: the data enter the double-float transforms scaled by 2^df_shift
  double* coarse64_u = nullptr;  // mixed precision: FP64 copies for the coarsest solve
  double* coarse64_f = nullptr;
  double* coarse64_r = nullptr;
  double* r64 = nullptr;         // mixed precision: finest FP64 residual
  double* u0m = nullptr;         // transformed initial value (sine basis)
  double* u_dev = nullptr;        // st_solve_host: device solution buffer (allocated on first use)
  // generic-q kernels: Mh (1/(2k+1)), R1, R2 and R1, R2 times 2^d (prolongation), q x q row-major
  double* tt64[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // q > kQfix: [K_tau | M_tau / tau | psi(t^+) | psi(t^-)] for the node-basis residual of st_residual
  double* node_time64 = nullptr;
  float* tt32[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  std::string err;
  // kernel timing
  bool prof = false;
  std::vector<cudaEvent_t> ev;          // pool, 2 per timed launch
  std::vector<int> ev_class;            // class of each recorded pair
  std::vector<int> ev_level;            // level of each recorded pair (-1: not level-specific)
  // per (class, level) totals of the last timed region: launches, ms, bytes, flops
  std::vector<double> lv_stats;
  int prof_launches[ST_K_COUNT] = {0};
  double prof_bytes[ST_K_COUNT] = {0};   // algorithmic HBM bytes of the counted launches
  double prof_flops[ST_K_COUNT] = {0};   // algorithmic floating-point operations
  int prof_dropped = 0;
};

namespace {

constexpr int kNormBlocks = 1024;
constexpr int kThreads = 256;

struct Fail {
  int code;
};

void check(st_handle* h, cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    h->err = std::string(what) + ": " + cudaGetErrorString(e);
    throw Fail{ST_ECUDA};
  }
}

void fail(st_handle* h, int code, const std::string& msg) {
  h->err = msg;
  throw Fail{code};
}

// Records an event pair around the launches made during its lifetime when the
// handle's kernel timing is on.
struct Prof {
  st_handle* h;
  int slot = -1;
  Prof(st_handle* hh, int cls, double bytes = 0.0, double flops = 0.0, int kernels = 1, int level = -1) : h(hh) {
    if (!h->prof) return;
    h->prof_launches[cls] += kernels;
    h->prof_bytes[cls] += bytes;
    h->prof_flops[cls] += flops;
    if (level >= 0) {
      const size_t b = ((size_t)cls * h->levels.size() + level) * 4;
      h->lv_stats[b + 0] += kernels;
      h->lv_stats[b + 2] += bytes;
      h->lv_stats[b + 3] += flops;
    }
    const int pair = (int)h->ev_class.size();
    if (2 * pair + 1 >= (int)h->ev.size()) { h->prof_dropped++; return; }
    slot = pair;
    h->ev_class.push_back(cls);
    h->ev_level.push_back(level);
    cudaEventRecord(h->ev[2 * pair], h->stream);
  }
  ~Prof() {
    if (slot >= 0) cudaEventRecord(h->ev[2 * slot + 1], h->stream);
  }
};

int level_of(st_handle* h, const Level& lv) { return (int)(&lv - h->levels.data()); }

template <typename T>
T* dalloc(st_handle* h, size_t count) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = sizeof(T);
  if (h->opt.max_workspace_bytes && h->bytes + bytes > h->opt.max_workspace_bytes)
    fail(h, ST_ENOMEM, "device workspace would exceed max_workspace_bytes");
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(h, ST_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  h->allocs.push_back(p);
  h->bytes += bytes;
  return static_cast<T*>(p);
}

template <typename T>
void upload(st_handle* h, T* dst, const std::vector<double>& src) {
  std::vector<T> tmp(src.begin(), src.end());
  check(h, cudaMemcpy(dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice), "upload table");
}

// Host FP64 per-mode time blocks of the sine basis: for spatial mode j with
// lamM_j = prod_a m(k_a), lamK_j = sum_a kappa(k_a) prod_{b != a} m(k_b)
// (m(k) = h/3 (2 + cos(k pi / Nf)), kappa(k) = 2/h (1 - cos(k pi / Nf)), the
// eigenvalues of the 1D mass and stiffness matrices), A_j = lamM_j K + lamK_j M_tau
// (K = K_tau, transposed for the adjoint) and its inverse (Gauss-Jordan with
// partial pivoting), laid out tab[e * Nx + j].
void mode_blocks(const HostTime& tm, int D, int n, double h, double tau, bool adj, std::vector<double>& amat,
                 std::vector<double>& ainv, std::vector<double>& lamMv, std::vector<double>& lamKtv) {
  const int q = tm.q, qq = q * q;
  const int Nf = n + 1;
  int64_t Nx = 1;
  for (int a = 0; a < D; ++a) Nx *= n;
  std::vector<double> m1(n), k1(n);
  for (int k = 1; k <= n; ++k) {
    const double c = std::cos(k * M_PI / Nf);
    m1[k - 1] = h / 3.0 * (2.0 + c);
    k1[k - 1] = 2.0 / h * (1.0 - c);
  }
  amat.assign((size_t)qq * Nx, 0.0);
  ainv.assign((size_t)qq * Nx, 0.0);
  lamMv.assign((size_t)Nx, 0.0);
  lamKtv.assign((size_t)Nx, 0.0);
  std::vector<double> A(qq), X(qq), M(qq);
  for (int64_t j = 0; j < Nx; ++j) {
    int idx[3] = {0, 0, 0};
    int64_t rest = j;
    for (int a = 0; a < D; ++a) {
      idx[a] = (int)(rest % n);
      rest /= n;
    }
    double lamM = 1.0, lamK = 0.0;
    for (int a = 0; a < D; ++a) {
      double prod = k1[idx[a]];
      for (int b = 0; b < D; ++b)
        if (b != a) prod *= m1[idx[b]];
      lamK += prod;
      lamM *= m1[idx[a]];
    }
    lamMv[j] = lamM;
    lamKtv[j] = lamK * tau;
    for (int k = 0; k < q; ++k)
      for (int l = 0; l < q; ++l)
        A[k * q + l] = lamM * (adj ? tm.K[l * q + k] : tm.K[k * q + l]) + (k == l ? lamK * tau * tm.Mh[k] : 0.0);
    // Gauss-Jordan with partial pivoting on a q x q matrix
    M = A;
    for (int i = 0; i < q; ++i)
      for (int c = 0; c < q; ++c) X[i * q + c] = (i == c) ? 1.0 : 0.0;
    for (int c = 0; c < q; ++c) {
      int p = c;
      for (int r = c + 1; r < q; ++r)
        if (std::fabs(M[r * q + c]) > std::fabs(M[p * q + c])) p = r;
      if (p != c)
        for (int i = 0; i < q; ++i) {
          std::swap(M[c * q + i], M[p * q + i]);
          std::swap(X[c * q + i], X[p * q + i]);
        }
      const double dv = 1.0 / M[c * q + c];
      for (int i = 0; i < q; ++i) {
        M[c * q + i] *= dv;
        X[c * q + i] *= dv;
      }
      for (int r = 0; r < q; ++r) {
        if (r == c) continue;
        const double fct = M[r * q + c];
        for (int i = 0; i < q; ++i) {
          M[r * q + i] -= fct * M[c * q + i];
          X[r * q + i] -= fct * X[c * q + i];
        }
      }
    }
    for (int e = 0; e < qq; ++e) {
      amat[(size_t)e * Nx + j] = A[e];
      ainv[(size_t)e * Nx + j] = X[e];
    }
  }
}

template <typename T>
void make_tables(st_handle* h, Level& lv, Tables<T>& tb) {
  const int n = lv.n, Nf = n + 1;
  std::vector<double> sp(Nf), tc(Nf), ts(Nf);
  for (int j = 0; j < Nf; ++j) {
    sp[j] = std::sin(j * M_PI / Nf);
    tc[j] = std::cos(2.0 * M_PI * j / Nf);
    ts[j] = std::sin(2.0 * M_PI * j / Nf);
  }
  tb.sinp = dalloc<T>(h, Nf);
  tb.twc = dalloc<T>(h, Nf);
  tb.tws = dalloc<T>(h, Nf);
  upload(h, tb.sinp, sp);
  upload(h, tb.twc, tc);
  upload(h, tb.tws, ts);
  for (int adj = 0; adj < 2; ++adj) {
    std::vector<double> am, ai, lm, lk;
    mode_blocks(h->tm, h->d, n, lv.h, lv.tau, adj != 0, am, ai, lm, lk);
    std::vector<double> aw(ai);
    for (double& x : aw) x *= h->opt.omega;
    {   // ws_k = lamM sum_l (w A^{-1})[k,l] sigma_l, sigma_l = (-1)^l (forward) or 1 (adjoint)
      const int q = h->q;
      const int64_t Nx = lv.Nx;
      std::vector<double> wsv((size_t)q * Nx);
      for (int64_t j = 0; j < Nx; ++j)
        for (int k = 0; k < q; ++k) {
          double acc = 0.0;
          for (int l = 0; l < q; ++l) {
            const double w = aw[(size_t)(k * q + l) * Nx + j];
            acc += (adj == 0 && (l & 1)) ? -w : w;
          }
          wsv[(size_t)k * Nx + j] = lm[j] * acc;
        }
      tb.ws[adj] = dalloc<T>(h, wsv.size());
      upload(h, tb.ws[adj], wsv);
    }
    if (h->q <= kQfix) {   // the generic-q residual uses the structure of K_tau instead
      tb.amat[adj] = dalloc<T>(h, am.size());
      upload(h, tb.amat[adj], am);
    }
    tb.ainv[adj] = dalloc<T>(h, ai.size());
    tb.ainvw[adj] = dalloc<T>(h, aw.size());
    upload(h, tb.ainv[adj], ai);
    upload(h, tb.ainvw[adj], aw);
    if (adj == 0) {
      tb.lamM = dalloc<T>(h, lm.size());
      tb.lamKt = dalloc<T>(h, lk.size());
      upload(h, tb.lamM, lm);
      upload(h, tb.lamKt, lk);
    }
  }
  if (lv.coarsen_full) {
    // coarse mode k (k = 1..nc) pairs with fine modes k and Nf - k, c_k = cos(k pi / Nf)
    const int nc = (n - 1) / 2;
    std::vector<double> a(std::max(nc, 1)), b(std::max(nc, 1));
    for (int k = 1; k <= nc; ++k) {
      const double c = std::cos(k * M_PI / Nf);
      a[k - 1] = 0.5 * (1.0 + c);
      b[k - 1] = -0.5 * (1.0 - c);
    }
    tb.ra = dalloc<T>(h, a.size());
    tb.rb = dalloc<T>(h, b.size());
    upload(h, tb.ra, a);
    upload(h, tb.rb, b);
  }
}

template <typename T>
void make_space(st_handle* h, Level& lv, std::vector<SpaceLvl<T>>& sp) {
  int nl = lv.n;
  double hl = lv.h;
  while (true) {
    SpaceLvl<T> s;
    s.n = nl;
    s.h = hl;
    s.Nx = 1;
    for (int a = 0; a < h->d; ++a) s.Nx *= nl;
    const int64_t cnt = (int64_t)lv.N * h->q * s.Nx;
    s.x = dalloc<T>(h, cnt);
    s.t = dalloc<T>(h, cnt);
    if (!sp.empty()) s.b = dalloc<T>(h, cnt);   // the finest spatial level reads the caller's vector
    for (int adj = 0; adj < 2; ++adj) {   // the spatial operator A_i of this grid, in the sine basis
      std::vector<double> am, ai, lm, lk;
      mode_blocks(h->tm, h->d, nl, hl, lv.tau, adj != 0, am, ai, lm, lk);
      s.amat[adj] = dalloc<T>(h, am.size());
      upload(h, s.amat[adj], am);
    }
    if (nl > 1) {
      const int nc = (nl - 1) / 2;
      std::vector<double> a(nc), b(nc);
      for (int k = 1; k <= nc; ++k) {
        const double c = std::cos(k * M_PI / (nl + 1));
        a[k - 1] = 0.5 * (1.0 + c);
        b[k - 1] = -0.5 * (1.0 - c);
      }
      s.ra = dalloc<T>(h, nc);
      s.rb = dalloc<T>(h, nc);
      upload(h, s.ra, a);
      upload(h, s.rb, b);
    }
    sp.push_back(s);
    if (nl == 1) break;
    nl = (nl - 1) / 2;
    hl *= 2.0;
  }
}

template <typename T> Vecs<T>& vecs(Level& lv);
template <> Vecs<double>& vecs<double>(Level& lv) { return lv.v64; }
template <> Vecs<float>& vecs<float>(Level& lv) { return lv.v32; }
template <typename T> std::vector<SpaceLvl<T>>& spaces(Level& lv);
template <> std::vector<SpaceLvl<double>>& spaces<double>(Level& lv) { return lv.sp64; }
template <> std::vector<SpaceLvl<float>>& spaces<float>(Level& lv) { return lv.sp32; }
template <typename T> Tables<T>& tables(Level& lv);
template <> Tables<double>& tables<double>(Level& lv) { return lv.t64; }
template <> Tables<float>& tables<float>(Level& lv) { return lv.t32; }

inline unsigned blocks_for(int64_t n, int threads = kThreads) {
  return (unsigned)((n + threads - 1) / threads);
}

// ------------------------------------------------------------------ dispatch
template <typename T, int D, int Q>
void launch_residual_t(st_handle* h, const Level& lv, bool adj, const T* f, const T* u, const T* u0, T* r,
                       int s0, int ns) {
  auto tc = to_coef<T, Q>(h->tm);
  if (D == 2) {
    dim3 block(stmg::kResTX, stmg::kResTY);
    dim3 grid((lv.n + stmg::kResTX - 1) / stmg::kResTX, (lv.n + stmg::kResTY - 1) / stmg::kResTY, 1);
    for (int c = 0; c < ns; c += 65535) {
      grid.z = std::min(65535, ns - c);
      if (adj)
        stmg::k_residual2d<T, Q, true><<<grid, block, 0, h->stream>>>(f, u, u0, r, lv.n, lv.N, s0 + c, (T)lv.tau,
                                                                       (T)lv.h, (T)(1.0 / lv.h), tc);
      else
        stmg::k_residual2d<T, Q, false><<<grid, block, 0, h->stream>>>(f, u, u0, r, lv.n, lv.N, s0 + c, (T)lv.tau,
                                                                        (T)lv.h, (T)(1.0 / lv.h), tc);
    }
    return;
  }
  dim3 grid(blocks_for(lv.Nx), 1);
  for (int c = 0; c < ns; c += 65535) {
    grid.y = std::min(65535, ns - c);
    if (adj)
      stmg::k_residual<T, D, Q, true><<<grid, kThreads, 0, h->stream>>>(f, u, u0, r, lv.n, lv.N, s0 + c,
                                                                         (T)lv.tau, (T)lv.h, (T)(1.0 / lv.h), tc);
    else
      stmg::k_residual<T, D, Q, false><<<grid, kThreads, 0, h->stream>>>(f, u, u0, r, lv.n, lv.N, s0 + c,
                                                                          (T)lv.tau, (T)lv.h, (T)(1.0 / lv.h), tc);
  }
}

template <typename T, int D, int Q>
void launch_mresidual_t(st_handle* h, Level& lv, bool adj, const T* f, const T* u, const T* u0, T* r, int s0,
                        int ns) {
  Tables<T>& tb = tables<T>(lv);
  constexpr int TS = stmg::kStepsPerThread;
  const int nblk = (ns + TS - 1) / TS;
  dim3 grid(blocks_for(lv.Nx), 1);
  for (int c = 0; c < nblk; c += 65535) {
    grid.y = std::min(65535, nblk - c);
    if (adj)
      stmg::k_fresidual<T, Q, true><<<grid, kThreads, 0, h->stream>>>(f, u, u0, r, lv.Nx, lv.N, s0 + c * TS, s0 + ns,
                                                                      tb.amat[1], tb.lamM);
    else
      stmg::k_fresidual<T, Q, false><<<grid, kThreads, 0, h->stream>>>(f, u, u0, r, lv.Nx, lv.N, s0 + c * TS,
                                                                       s0 + ns, tb.amat[0], tb.lamM);
  }
}

// fmode: stmg::kFromF, kMakeWf (also writes wf) or kUseWf (f holds wf); the
// last two only with damp.
template <typename T, int D, int Q>
void launch_msmooth_t(st_handle* h, Level& lv, bool adj, bool damp, int fmode, const T* f, const T* u, const T* u0,
                      T* out, T* wf, int s0, int ns) {
  Tables<T>& tb = tables<T>(lv);
  const int a = adj ? 1 : 0;
  const T* ai = damp ? tb.ainvw[a] : tb.ainv[a];
  const T* ws = tb.ws[a];
  const T wc = (T)(1.0 - h->opt.omega);
  constexpr int TS = stmg::kStepsPerThread;
  const int nblk = (ns + TS - 1) / TS;
  dim3 grid(blocks_for(lv.Nx), 1);
  for (int c = 0; c < nblk; c += 65535) {
    grid.y = std::min(65535, nblk - c);
#define STMG_FSMOOTH(ADJ, DAMP, FM)                                                                         \
  stmg::k_fsmooth<T, Q, ADJ, DAMP, FM><<<grid, kThreads, 0, h->stream>>>(f, u, u0, out, lv.Nx, lv.N, s0 + c * TS, \
                                                                         s0 + ns, wc, ai, tb.lamM, wf, ws)
#define STMG_FSMOOTH_DIR(ADJ)                                           \
  if (!damp) STMG_FSMOOTH(ADJ, false, stmg::kFromF);                    \
  else if (fmode == stmg::kMakeWf) STMG_FSMOOTH(ADJ, true, stmg::kMakeWf); \
  else if (fmode == stmg::kUseWf) STMG_FSMOOTH(ADJ, true, stmg::kUseWf);   \
  else STMG_FSMOOTH(ADJ, true, stmg::kFromF)
    if (adj) {
      STMG_FSMOOTH_DIR(true);
    } else {
      STMG_FSMOOTH_DIR(false);
    }
#undef STMG_FSMOOTH_DIR
#undef STMG_FSMOOTH
  }
}

// ---- generic-q launchers (q > kQfix)
template <typename T> T* const* ttabs(st_handle* h);
template <> double* const* ttabs<double>(st_handle* h) { return h->tt64; }
template <> float* const* ttabs<float>(st_handle* h) { return h->tt32; }

template <typename T>
void launch_mresidual_dyn(st_handle* h, Level& lv, bool adj, const T* f, const T* u, const T* u0, T* r, int s0,
                          int ns) {
  Tables<T>& tb = tables<T>(lv);
  constexpr int TS = stmg::kStepsPerThread;
  const int nblk = (ns + TS - 1) / TS;
  dim3 grid(blocks_for(lv.Nx), 1);
  for (int c = 0; c < nblk; c += 65535) {
    grid.y = std::min(65535, nblk - c);
    if (adj)
      stmg::k_fresidual_dyn<T, true><<<grid, kThreads, 0, h->stream>>>(f, u, u0, r, lv.Nx, lv.N, s0 + c * TS,
                                                                       s0 + ns, h->q, tb.lamM, tb.lamKt, ttabs<T>(h)[0]);
    else
      stmg::k_fresidual_dyn<T, false><<<grid, kThreads, 0, h->stream>>>(f, u, u0, r, lv.Nx, lv.N, s0 + c * TS,
                                                                        s0 + ns, h->q, tb.lamM, tb.lamKt, ttabs<T>(h)[0]);
  }
}

template <typename T>
void launch_msmooth_dyn(st_handle* h, Level& lv, bool adj, bool damp, int fmode, const T* f, const T* u, const T* u0,
                        T* out, T* wf, int s0, int ns) {
  Tables<T>& tb = tables<T>(lv);
  const int a = adj ? 1 : 0;
  const T* ai = damp ? tb.ainvw[a] : tb.ainv[a];
  const T* ws = tb.ws[a];
  const T wc = (T)(1.0 - h->opt.omega);
  constexpr int TS = stmg::kStepsPerThread;
  const int nblk = (ns + TS - 1) / TS;
  dim3 grid(blocks_for(lv.Nx), 1);
  for (int c = 0; c < nblk; c += 65535) {
    grid.y = std::min(65535, nblk - c);
#define STMG_FSMOOTH_DYN(ADJ, DAMP, FM)                                                                          \
  stmg::k_fsmooth_dyn<T, ADJ, DAMP, FM><<<grid, kThreads, 0, h->stream>>>(f, u, u0, out, lv.Nx, lv.N, s0 + c * TS, \
                                                                          s0 + ns, h->q, wc, ai, tb.lamM, wf, ws)
#define STMG_FSMOOTH_DYN_DIR(ADJ)                                           \
  if (!damp) STMG_FSMOOTH_DYN(ADJ, false, stmg::kFromF);                    \
  else if (fmode == stmg::kMakeWf) STMG_FSMOOTH_DYN(ADJ, true, stmg::kMakeWf); \
  else if (fmode == stmg::kUseWf) STMG_FSMOOTH_DYN(ADJ, true, stmg::kUseWf);   \
  else STMG_FSMOOTH_DYN(ADJ, true, stmg::kFromF)
    if (adj) {
      STMG_FSMOOTH_DYN_DIR(true);
    } else {
      STMG_FSMOOTH_DYN_DIR(false);
    }
#undef STMG_FSMOOTH_DYN_DIR
#undef STMG_FSMOOTH_DYN
  }
}

template <typename T, int D>
void launch_restrict_dyn_t(st_handle* h, Level& fine, const Level& coarse, const T* r, T* fc) {
  const size_t smem = 2 * sizeof(T) * h->q * h->q;
  T* const* tt = ttabs<T>(h);
  dim3 grid(blocks_for(coarse.Nx), coarse.N);
  if (fine.coarsen_full)
    stmg::k_frestrict_dyn<T, D, true><<<grid, kThreads, smem, h->stream>>>(
        r, fc, fine.n, coarse.n, coarse.N, h->q, tables<T>(fine).ra, tables<T>(fine).rb, tt[1], tt[2]);
  else
    stmg::k_frestrict_dyn<T, D, false><<<grid, kThreads, smem, h->stream>>>(
        r, fc, fine.n, coarse.n, coarse.N, h->q, (const T*)nullptr, (const T*)nullptr, tt[1], tt[2]);
}

template <typename T, int D>
void launch_prolong_dyn_t(st_handle* h, Level& fine, const Level& coarse, const T* ec, T* uf) {
  const size_t smem = 2 * sizeof(T) * h->q * h->q;
  T* const* tt = ttabs<T>(h);
  dim3 grid(blocks_for(fine.Nx), fine.N);
  if (fine.coarsen_full)   // time blocks pre-multiplied by 2^d (tt[3], tt[4])
    stmg::k_fprolong_dyn<T, D, true><<<grid, kThreads, smem, h->stream>>>(
        ec, uf, fine.n, coarse.n, fine.N, h->q, tables<T>(fine).ra, tables<T>(fine).rb, tt[3], tt[4]);
  else
    stmg::k_fprolong_dyn<T, D, false><<<grid, kThreads, smem, h->stream>>>(
        ec, uf, fine.n, coarse.n, fine.N, h->q, (const T*)nullptr, (const T*)nullptr, tt[1], tt[2]);
}

template <typename T, int D>
void launch_ic_grad_dyn_t(st_handle* h, const Level& lv, const T* lam, T* g) {
  stmg::k_ic_gradient_dyn<T, D><<<blocks_for(lv.Nx), kThreads, 0, h->stream>>>(lam, g, lv.n, (T)lv.h, h->q);
}

// Restriction / prolongation between levels L and L-1 in the sine basis: full
// coarsening pairs sine modes; semi coarsening is the identity in space (the
// node-basis kernel with FULL = false is the same operation in any basis).
template <typename T, int D, int Q>
void launch_restrict_t(st_handle* h, Level& fine, const Level& coarse, const T* r, T* fc) {
  auto tc = to_coef<T, Q>(h->tm);
  dim3 grid(blocks_for(coarse.Nx), coarse.N);
  if (!fine.coarsen_full)
    stmg::k_restrict<T, D, Q, false><<<grid, kThreads, 0, h->stream>>>(r, fc, fine.n, coarse.n, coarse.N, tc);
  else
    stmg::k_frestrict<T, D, Q><<<grid, kThreads, 0, h->stream>>>(r, fc, fine.n, coarse.n, coarse.N,
                                                                  tables<T>(fine).ra, tables<T>(fine).rb, tc);
}

template <typename T, int D, int Q>
void launch_prolong_t(st_handle* h, Level& fine, const Level& coarse, const T* ec, T* uf) {
  auto tc = to_coef<T, Q>(h->tm);
  dim3 grid(blocks_for(fine.Nx), fine.N);
  if (!fine.coarsen_full) {
    stmg::k_prolong<T, D, Q, false><<<grid, kThreads, 0, h->stream>>>(ec, uf, fine.n, coarse.n, fine.N, tc);
  } else {
    grid.y = coarse.N;   // one thread per (fine mode, coarse step)
    // pair weights of the prolongation are 2 ra, 2 rb per axis: fold 2^D into R^T
    for (int i = 0; i < Q * Q; ++i) {
      tc.R1[i] *= (T)(1 << D);
      tc.R2[i] *= (T)(1 << D);
    }
    stmg::k_fprolong<T, D, Q><<<grid, kThreads, 0, h->stream>>>(ec, uf, fine.n, coarse.n, fine.N,
                                                                 tables<T>(fine).ra, tables<T>(fine).rb, tc);
  }
}

// Coarse-grid correction and the first damped step after it in one pass
// (k_fprolong_smooth; full coarsening, q <= kQfix): out = step(u + P ec).
template <typename T, int D, int Q>
void launch_prolong_smooth_t(st_handle* h, Level& fine, const Level& coarse, bool adj, int fmode, const T* ec,
                             const T* f, const T* u, const T* u0, T* out) {
  auto tc = to_coef<T, Q>(h->tm);
  for (int i = 0; i < Q * Q; ++i) {   // pair weights of the prolongation: 2 ra, 2 rb per axis
    tc.R1[i] *= (T)(1 << D);
    tc.R2[i] *= (T)(1 << D);
  }
  Tables<T>& tb = tables<T>(fine);
  const int a = adj ? 1 : 0;
  const T wc = (T)(1.0 - h->opt.omega);
  constexpr int TS = stmg::kStepsPerThread;
  const int nblk = (fine.N + TS - 1) / TS;
  dim3 grid(blocks_for(fine.Nx), 1);
  for (int c = 0; c < nblk; c += 65535) {
    grid.y = std::min(65535, nblk - c);
#define STMG_FPS(ADJ, FM)                                                                                        \
  stmg::k_fprolong_smooth<T, D, Q, ADJ, FM><<<grid, kThreads, 0, h->stream>>>(                                   \
      ec, f, u, u0, out, fine.n, coarse.n, fine.N, c * TS, fine.N, wc, tb.ainvw[a], tb.lamM, tb.ws[a], tb.ra, tb.rb, \
      tc)
    if (adj) {
      if (fmode == stmg::kUseWf) STMG_FPS(true, stmg::kUseWf); else STMG_FPS(true, stmg::kFromF);
    } else {
      if (fmode == stmg::kUseWf) STMG_FPS(false, stmg::kUseWf); else STMG_FPS(false, stmg::kFromF);
    }
#undef STMG_FPS
  }
}

template <typename T, int D, int Q>
void launch_ic_grad_t(st_handle* h, const Level& lv, const T* lam, T* g) {
  auto tc = to_coef<T, Q>(h->tm);
  stmg::k_ic_gradient<T, D, Q><<<blocks_for(lv.Nx), kThreads, 0, h->stream>>>(lam, g, lv.n, (T)lv.h, tc);
}

template <typename T, int D, int Q>
void launch_space_solve_t(st_handle* h, const Level& lv, const SpaceLvl<T>& sl, const T* b, T* xo, double w,
                          const double* dinv) {
  stmg::SmallMat<T, Q> m{};
  for (int i = 0; i < Q * Q; ++i) m.a[i] = (T)dinv[i];
  dim3 grid(blocks_for(sl.Nx), lv.N);
  stmg::k_fspace_solve<T, Q><<<grid, kThreads, 0, h->stream>>>(b, xo, sl.Nx, lv.N, (T)w, m);
}

template <typename T, int D, int Q>
void launch_space_restrict_t(st_handle* h, const Level& lv, const SpaceLvl<T>& fine, const SpaceLvl<T>& coarse,
                             const T* in, T* out) {
  stmg::k_fspace_restrict<T, D, Q><<<dim3(blocks_for(coarse.Nx), lv.N), kThreads, 0, h->stream>>>(
      in, out, fine.n, coarse.n, lv.N, fine.ra, fine.rb);
}

template <typename T, int D, int Q>
void launch_space_pre_t(st_handle* h, const Level& lv, const SpaceLvl<T>& sl, bool adj, const T* b, T* x, T* r,
                        double w, const double* dinv) {
  stmg::SmallMat<T, Q> m{};
  for (int i = 0; i < Q * Q; ++i) m.a[i] = (T)dinv[i];
  stmg::k_fspace_pre<T, Q><<<dim3(blocks_for(sl.Nx), lv.N), kThreads, 0, h->stream>>>(
      b, x, r, sl.Nx, lv.N, (T)w, m, sl.amat[adj ? 1 : 0], h->opt.nu_x);
}

template <typename T, int D, int Q>
void launch_space_post_t(st_handle* h, const Level& lv, const SpaceLvl<T>& sl, const SpaceLvl<T>& cl, bool adj,
                         const T* b, T* x, const T* xc, double w, const double* dinv, T* upd, double wt) {
  stmg::SmallMat<T, Q> m{};
  for (int i = 0; i < Q * Q; ++i) m.a[i] = (T)dinv[i];
  stmg::k_fspace_post<T, D, Q><<<dim3(blocks_for(sl.Nx), lv.N), kThreads, 0, h->stream>>>(
      b, x, xc, sl.n, cl.n, lv.N, (T)w, m, sl.amat[adj ? 1 : 0], sl.ra, sl.rb, (T)(1 << D), h->opt.nu_x, upd,
      (T)wt);
}

#define STMG_DISPATCH(FN, ...)                                                   \
  do {                                                                           \
    switch (h->d * 10 + h->q) {                                                  \
      case 11: FN<T, 1, 1>(__VA_ARGS__); break;                                  \
      case 12: FN<T, 1, 2>(__VA_ARGS__); break;                                  \
      case 13: FN<T, 1, 3>(__VA_ARGS__); break;                                  \
      case 14: FN<T, 1, 4>(__VA_ARGS__); break;                                  \
      case 21: FN<T, 2, 1>(__VA_ARGS__); break;                                  \
      case 22: FN<T, 2, 2>(__VA_ARGS__); break;                                  \
      case 23: FN<T, 2, 3>(__VA_ARGS__); break;                                  \
      case 24: FN<T, 2, 4>(__VA_ARGS__); break;                                  \
      case 31: FN<T, 3, 1>(__VA_ARGS__); break;                                  \
      case 32: FN<T, 3, 2>(__VA_ARGS__); break;                                  \
      case 33: FN<T, 3, 3>(__VA_ARGS__); break;                                  \
      case 34: FN<T, 3, 4>(__VA_ARGS__); break;                                  \
      default: fail(h, ST_EINVAL, "unsupported (dim, q)");                       \
    }                                                                            \
  } while (0)

#define STMG_DISPATCH_D(FN, ...)                                                 \
  do {                                                                           \
    switch (h->d) {                                                              \
      case 1: FN<T, 1>(__VA_ARGS__); break;                                      \
      case 2: FN<T, 2>(__VA_ARGS__); break;                                      \
      case 3: FN<T, 3>(__VA_ARGS__); break;                                      \
      default: fail(h, ST_EINVAL, "unsupported dim");                            \
    }                                                                            \
  } while (0)

template <typename T, int D>
void launch_residual_dyn_t(st_handle* h, const Level& lv, bool adj, const T* f, const T* u, const T* u0, T* r,
                           int s0, int ns) {
  static_assert(sizeof(T) == 8, "the node-basis residual of high degree is FP64");
  dim3 grid(blocks_for(lv.Nx), 1);
  for (int c = 0; c < ns; c += 65535) {
    grid.y = std::min(65535, ns - c);
    if (adj)
      stmg::k_residual_dyn<T, D, true><<<grid, kThreads, 0, h->stream>>>(
          f, u, u0, r, lv.n, lv.N, s0 + c, h->q, (T)lv.tau, (T)lv.h, (T)(1.0 / lv.h), h->node_time64);
    else
      stmg::k_residual_dyn<T, D, false><<<grid, kThreads, 0, h->stream>>>(
          f, u, u0, r, lv.n, lv.N, s0 + c, h->q, (T)lv.tau, (T)lv.h, (T)(1.0 / lv.h), h->node_time64);
  }
}

template <typename T>
void residual(st_handle* h, Level& lv, bool adj, const T* f, const T* u, const T* u0, T* r, int s0 = 0,
              int ns = -1) {
  if (ns < 0) ns = lv.N;
  const int D = h->d, Q = h->q;
  const double nodes = (double)ns * lv.Nx;
  // per node: Q fields x (9D-3) FMA for M_h, K_h (tensor-product passes), trace Q + 3D,
  // time mixing Q^2 + 2Q; bytes: read u, f, write r (+ u0)
  const double fma = Q * (9.0 * D - 3.0) + Q + 3.0 * D + Q * Q + 2.0 * Q;
  Prof pr(h, ST_K_RESIDUAL, sizeof(T) * (3.0 * nodes * Q + (u0 ? (double)lv.Nx : 0.0)), 2.0 * fma * nodes, 1,
          level_of(h, lv));
  if (Q > kQfix) {
    if (sizeof(T) != 8 || h->node_time64 == nullptr || &lv != &h->levels.back())
      fail(h, ST_EINVAL, "internal: the node-basis residual above q = 4 is FP64 on the finest level");
    STMG_DISPATCH_D(launch_residual_dyn_t, h, lv, adj, f, u, u0, r, s0, ns);
    return;
  }
  STMG_DISPATCH(launch_residual_t, h, lv, adj, f, u, u0, r, s0, ns);
}

// Residual in the sine basis, steps [s0, s0 + ns).
template <typename T>
void mresidual(st_handle* h, Level& lv, bool adj, const T* f, const T* u, const T* u0, T* r, int s0 = 0,
               int ns = -1) {
  if (ns < 0) ns = lv.N;
  const double Q = h->q, nodes = (double)ns * lv.Nx;
  // per (mode, step): trace Q - 1 adds and lamM (1), coupling Q, A_i u Q^2 FMA (q > kQfix: the
  // structured K_tau product, 12 flops per time dof); bytes: read u, f, write r (+ u0).  u == nullptr
  // is a zero iterate: r = f plus the initial-value coupling.
  Prof pr(h, ST_K_RESIDUAL, sizeof(T) * ((u ? 3.0 : 2.0) * nodes * Q + (u0 ? (double)lv.Nx : 0.0)),
          u ? nodes * (h->q > kQfix ? 12.0 * Q : 2.0 * Q * Q + 2.0 * Q) : 0.0, 1, level_of(h, lv));
  if (h->q > kQfix) launch_mresidual_dyn<T>(h, lv, adj, f, u, u0, r, s0, ns);
  else STMG_DISPATCH(launch_mresidual_t, h, lv, adj, f, u, u0, r, s0, ns);
}

// Fused damped block-Jacobi step with the exact block inverse in the sine
// basis (k_fsmooth): out = (1 - w) u + w A^{-1}(f - B u_prev) (damp), or
// out = A^{-1}(f - B u_prev) (no damping), steps [s0, s0 + ns); u may be null.
// fmode (damped steps): kMakeWf also stores w A^{-1} f in wf; kUseWf takes
// f = wf of an earlier kMakeWf on the same right-hand side.
template <typename T>
void msmooth(st_handle* h, Level& lv, bool adj, bool damp, const T* f, const T* u, const T* u0, T* out, int s0 = 0,
             int ns = -1, int fmode = stmg::kFromF, T* wf = nullptr) {
  if (ns < 0) ns = lv.N;
  if (!damp) fmode = stmg::kFromF;
  const double Q = h->q, nodes = (double)ns * lv.Nx;
  // read f or wf (and u), write out (and wf)
  const double passes = 2.0 + ((damp && u) ? 1.0 : 0.0) + (fmode == stmg::kMakeWf ? 1.0 : 0.0);
  // per (mode, step): trace Q - 1 adds, coupling Q FMA (lamM or ws), A_i^{-1} Q^2 FMA
  // (not with kUseWf), damping Q FMA
  const double flops = (fmode == stmg::kUseWf ? 0.0 : 2.0 * Q * Q) + 4.0 * Q + (fmode == stmg::kFromF ? Q : 0.0);
  Prof pr(h, ST_K_SMOOTH, sizeof(T) * passes * nodes * Q, nodes * flops, 1, level_of(h, lv));
  if (h->q > kQfix) launch_msmooth_dyn<T>(h, lv, adj, damp, fmode, f, u, u0, out, wf, s0, ns);
  else STMG_DISPATCH(launch_msmooth_t, h, lv, adj, damp, fmode, f, u, u0, out, wf, s0, ns);
}

template <typename T>
void restrict_to(st_handle* h, int L, const T* r, T* fc) {
  Level& fine = h->levels[L];
  Level& coarse = h->levels[L - 1];
  const double cn = (double)coarse.ndof, fn_ = (double)fine.ndof;
  const double ns = fine.coarsen_full ? std::pow(2.0, h->d) : 1.0;
  // time blocks: (q + 1) / 2 FMA per coarse dof and block (R is lower triangular; the kernels skip its zeros)
  const double tq = 0.5 * (h->q + 1);
  Prof pr(h, ST_K_RESTRICT, sizeof(T) * (cn + fn_), 2.0 * cn * (2.0 * ns + 2.0 * tq), 1, L);
  if (h->q > kQfix) STMG_DISPATCH_D(launch_restrict_dyn_t, h, fine, coarse, r, fc);
  else STMG_DISPATCH(launch_restrict_t, h, fine, coarse, r, fc);
}

// The coarse-grid correction of level L fused into its first post-smoothing
// step: out = damped step of (u + P ec), u itself unchanged.  fmode: kFromF
// (f is the right-hand side) or kUseWf (f holds a ready wf).
template <typename T>
void prolong_smooth(st_handle* h, int L, bool adj, int fmode, const T* ec, const T* f, const T* u, const T* u0,
                    T* out) {
  Level& fine = h->levels[L];
  Level& coarse = h->levels[L - 1];
  const double Q = h->q, nodes = (double)fine.N * fine.Nx, fn_ = (double)fine.ndof;
  const double tq = 0.5 * (h->q + 1);
  // bytes: read f or wf, u and the coarse correction, write out; flops: the correction
  // (2 (1 + tq) per fine unknown, as k_fprolong) and the damped step (as k_fsmooth)
  const double step_flops = (fmode == stmg::kUseWf ? 0.0 : 2.0 * Q * Q) + 4.0 * Q + (fmode == stmg::kFromF ? Q : 0.0);
  Prof pr(h, ST_K_SMOOTH, sizeof(T) * (3.0 * fn_ + (double)coarse.ndof),
          2.0 * fn_ * (1.0 + tq) + nodes * step_flops, 1, L);
  if constexpr (sizeof(T) == 4) {   // used by the FP32 cycles only
    STMG_DISPATCH(launch_prolong_smooth_t, h, fine, coarse, adj, fmode, ec, f, u, u0, out);
  } else {
    fail(h, ST_EINVAL, "internal: the fused correction serves the FP32 cycles");
  }
}

template <typename T>
void prolong_add(st_handle* h, int L, const T* ec, T* uf) {
  Level& fine = h->levels[L];
  Level& coarse = h->levels[L - 1];
  const double cn = (double)coarse.ndof, fn_ = (double)fine.ndof;
  const double ns = 1.0;
  const double tq = 0.5 * (h->q + 1);
  Prof pr(h, ST_K_PROLONG, sizeof(T) * (cn + 2.0 * fn_), 2.0 * fn_ * (ns + tq), 1, L);
  if (h->q > kQfix) STMG_DISPATCH_D(launch_prolong_dyn_t, h, fine, coarse, ec, uf);
  else STMG_DISPATCH(launch_prolong_t, h, fine, coarse, ec, uf);
}

template <typename T>
void zero(st_handle* h, T* y, int64_t n) {
  Prof pr(h, ST_K_VECTOR, sizeof(T) * (double)n, 0.0);
  stmg::k_fill<T><<<std::min<int64_t>(blocks_for(n), 152 * 16), kThreads, 0, h->stream>>>(y, T(0), n);
}

template <typename T>
void copy(st_handle* h, T* y, const T* x, int64_t n) {
  Prof pr(h, ST_K_VECTOR, 2.0 * sizeof(T) * (double)n, 0.0);
  stmg::k_scale_copy<T><<<std::min<int64_t>(blocks_for(n), 152 * 16), kThreads, 0, h->stream>>>(y, x, T(1), n);
}

// Shared-memory bytes of the sine-transform kernels (see stmg_kernels.cuh).
constexpr int kDstWarps = 8;
constexpr int kDstRowsPerCta = 32;
template <typename T>
size_t dst_rows_smem(int Nf) { return (size_t)(2 + 2 * kDstWarps) * Nf * sizeof(T); }
template <typename T, int W>
size_t dst_cols_smem(int Nf) {
  return W * sizeof(int64_t) + ((size_t)2 * Nf + (size_t)W * (Nf + 1) + (size_t)kDstWarps * Nf) * sizeof(T);
}

// Register sine transform (k_dst_rows_reg): rows per CTA = threads / G;
// 256 threads for FP32, 128 for FP64 (FP64 is bound by the FP64 pipe, so fewer
// rows per CTA keep the shared-memory footprint down).
template <typename T>
int dst_reg_threads() { return sizeof(T) == 8 ? 128 : 256; }
template <typename T, int LP, int LG>
size_t dst_reg_smem() {
  using Lay = stmg::DstRegLayout<LP, LG>;
  const int rows = dst_reg_threads<T>() / Lay::G;
  return ((size_t)Lay::TAB + (size_t)rows * Lay::RS) * sizeof(T);
}
// k_dst_cols_reg: the same plus one int64 line base per line.
template <typename T, int LP, int LG>
size_t dst_cols_reg_smem() {
  using Lay = stmg::DstRegLayout<LP, LG>;
  return dst_reg_smem<T, LP, LG>() + (size_t)(dst_reg_threads<T>() / Lay::G) * sizeof(int64_t);
}

constexpr size_t kMaxSmem = 227 * 1024;

// Opt the sine-transform kernels into the dynamic shared memory they need for
// the line lengths this hierarchy uses (every level transforms along every axis).
template <typename T>
void dst_set_smem_limits(st_handle* h) {
  int maxNf = 2;
  for (const Level& l : h->levels) maxNf = std::max(maxNf, l.n + 1);
  auto set = [&](const void* fn, size_t bytes) {
    if (bytes > kMaxSmem) fail(h, ST_EINVAL, "n too large for the sine-transform kernels");
    check(h, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
          "cudaFuncSetAttribute");
  };
  for (const Level& l : h->levels) {
    const int Nf = l.n + 1;
    if (Nf >= 64 && Nf <= 512) {
      if (Nf == 64) set((const void*)stmg::k_dst_rows_reg<T, 3, 2>, dst_reg_smem<T, 3, 2>());
      if (Nf == 128) set((const void*)stmg::k_dst_rows_reg<T, 3, 3>, dst_reg_smem<T, 3, 3>());
      if (Nf == 256) set((const void*)stmg::k_dst_rows_reg<T, 4, 3>, dst_reg_smem<T, 4, 3>());
      if (Nf == 512) set((const void*)stmg::k_dst_rows_reg<T, 4, 4>, dst_reg_smem<T, 4, 4>());
    } else {
      set((const void*)stmg::k_dst_rows<T>, dst_rows_smem<T>(Nf));
    }
  }
  if (h->d >= 2) {   // y (and z) axes: register transform for 64 <= Nf <= 512, else column tiles
    int max16 = 0, max32 = 0;
    for (const Level& l : h->levels) {
      const int Nf = l.n + 1;
      if (Nf >= 64 && Nf <= 512) {
        if (Nf == 64) set((const void*)stmg::k_dst_cols_reg<T, 3, 2>, dst_cols_reg_smem<T, 3, 2>());
        if (Nf == 128) set((const void*)stmg::k_dst_cols_reg<T, 3, 3>, dst_cols_reg_smem<T, 3, 3>());
        if (Nf == 256) set((const void*)stmg::k_dst_cols_reg<T, 4, 3>, dst_cols_reg_smem<T, 4, 3>());
        if (Nf == 512) set((const void*)stmg::k_dst_cols_reg<T, 4, 4>, dst_cols_reg_smem<T, 4, 4>());
        continue;
      }
      if (sizeof(T) == 8 && Nf >= 512) max16 = std::max(max16, Nf); else max32 = std::max(max32, Nf);
    }
    if (max16) set((const void*)stmg::k_dst_cols<T, 16>, dst_cols_smem<T, 16>(max16));
    if (max32) set((const void*)stmg::k_dst_cols<T, 32>, dst_cols_smem<T, 32>(max32));
  }
  (void)maxNf;
}

// Algorithmic flops of one sine transform of a line of n = Nf - 1 values:
// pre-processing 5 Nf, complex FFT of Nf/2 points 5 (Nf/2) log2(Nf/2),
// even/odd split 12 (Nf/2), prefix scan Nf, scaling n.
double dst_line_flops(int n) {
  const int Nf = n + 1;
  int logh = 0;
  while ((1 << (logh + 1)) <= Nf / 2) ++logh;
  const double hf = Nf / 2.0;
  return 5.0 * Nf + 5.0 * hf * logh + 12.0 * hf + Nf + n;
}

// ---- sine transforms on the tensor cores (stmg_tc.cuh) ----
// Lines per split / tensor-core batch (digit planes: 16 bytes per value, 537 MB at Nf = 256): each
// tensor-pass launch fills and drains its pipeline once, so fewer, larger batches run faster.
constexpr int64_t kTcCapLines = 131072;

bool tc_len(int Nf) { return Nf >= stmg_tc::kMinNf && Nf <= stmg_tc::kMaxNf; }
// ST_DST_AUTO and ST_DST_TENSOR: the tensor cores replace the FP64 FFTs and the mixed form's
// double-float FFTs at these lengths (faster than both).
bool use_tc(const st_handle* h, const Level& lv) { return h->opt.transform != ST_DST_FFT && tc_len(lv.n + 1); }

// FP16 bits of an integer |d| <= 64.
uint16_t fp16_of_small_int(int d) {
  if (d == 0) return 0;
  const int a = d < 0 ? -d : d;
  int e = 0;
  while ((a >> (e + 1)) != 0) ++e;
  return (uint16_t)((d < 0 ? 0x8000 : 0) | ((e + 15) << 10) | ((a << (10 - e)) & 0x3ff));
}

// FP16 digits of S / 2, S[k][m] = sin(pi k m / Nf): eight balanced base-128 digits in [-64, 64] each,
// most significant first, from long-double sines.  Layout of the tensor kernel's shared-memory stage:
// per (N tile nt, K chunk c) eight planes t of 64 (m) x 16 (k) values in K-major 8 x 8 core matrices.
std::vector<uint16_t> tc_sine_digits(int Nf) {
  const int nch = Nf / stmg_tc::BK, ntn = Nf / stmg_tc::BNP;
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<long double> sv(2 * (size_t)Nf);
  for (int j = 0; j < 2 * Nf; ++j) sv[j] = sinl(pi * (long double)j / (long double)Nf);
  std::vector<uint16_t> tab((size_t)ntn * nch * stmg_tc::B_STAGE / 2);
  for (int nt = 0; nt < ntn; ++nt)
    for (int c = 0; c < nch; ++c)
      for (int mm = 0; mm < stmg_tc::BNP; ++mm)
        for (int kk = 0; kk < stmg_tc::BK; ++kk) {
          const int m = nt * stmg_tc::BNP + mm, k = c * stmg_tc::BK + kk;
          long double v = sv[(size_t)((k * m) % (2 * Nf))] / 2.0L;
          for (int t = 0; t < stmg_tc::NSL; ++t) {
            v *= 128.0L;
            const long double dg = nearbyintl(v);
            v -= dg;
            const size_t off = (((size_t)nt * nch + c) * stmg_tc::NSL + t) * (stmg_tc::B_PLANE / 2) +
                               ((mm / 8) * 2 + kk / 8) * 64 + (mm % 8) * 8 + (kk % 8);
            tab[off] = fp16_of_small_int((int)dg);
          }
        }
  return tab;
}

void tc_prepare(st_handle* h, Level& lv) {
  if (!h->tcD) {
    int64_t cap = kTcCapLines;   // a batch is whole fields: hold at least one field's lines
    for (const Level& l : h->levels)
      if (tc_len(l.n + 1)) cap = std::max<int64_t>(cap, (l.Nx / l.n + stmg_tc::BM - 1) / stmg_tc::BM * stmg_tc::BM);
    h->tc_cap = cap;
    h->tcD = dalloc<uint8_t>(h, stmg_tc::plane_bytes_for(cap, stmg_tc::kMaxNf));
    h->tcE = dalloc<int>(h, cap);
    h->tcErr = dalloc<int>(h, 1);
    check(h, cudaMemsetAsync(h->tcErr, 0, sizeof(int), h->stream), "memset");
    auto attr = [&](const void* fn) {
      check(h, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, stmg_tc::Smem::bytes),
            "cudaFuncSetAttribute");
    };
    attr((const void*)stmg_tc::k_dst_tc<true, stmg_tc::NEPI>);
    attr((const void*)stmg_tc::k_dst_tc<false, stmg_tc::NEPI>);
    attr((const void*)stmg_tc::k_dst_tc<true, stmg_tc::NEPI_SHORT>);
    attr((const void*)stmg_tc::k_dst_tc<false, stmg_tc::NEPI_SHORT>);
  }
  if (!lv.tcS) {
    const std::vector<uint16_t> tab = tc_sine_digits(lv.n + 1);
    lv.tcS = reinterpret_cast<uint8_t*>(dalloc<uint16_t>(h, tab.size()));
    check(h, cudaMemcpy(lv.tcS, tab.data(), tab.size() * sizeof(uint16_t), cudaMemcpyHostToDevice), "upload sine digits");
  }
}

// A tensor-core wait that timed out (read back with a norm or by st_transform) fails the call.
void tc_check_flag(st_handle* h) {
  if (!h->tcErr) return;
  int flag = 0;
  std::memcpy(&flag, h->hnorm + 1, sizeof(int));
  if (flag != 0) {
    std::memset(h->hnorm + 1, 0, sizeof(int));
    cudaMemsetAsync(h->tcErr, 0, sizeof(int), h->stream);
    fail(h, ST_ECUDA, "tensor-core sine transform: an mbarrier wait timed out (code " + std::to_string(flag) + ")");
  }
}

// 2^axis_exp S along every axis of `slabs` FP64 fields of level lv (src / mid / dst as in dst_axes),
// the first pass scaled by 2^load_exp, the last by 2^store_exp: per axis a digit-splitting pass
// (lines' exponents and FP16 digit planes) and a tensor-core pass, in batches of whole slabs.
void dst_axes_tc(st_handle* h, Level& lv, const double* src, double* mid, double* dst, int64_t slabs, int axis_exp,
                 int load_exp, int store_exp) {
  tc_prepare(h, lv);
  const int n = lv.n, Nf = n + 1, nch = Nf / stmg_tc::BK, ntn = Nf / stmg_tc::BNP;
  const int64_t lps = lv.Nx / n;   // lines per field along any axis
  const int64_t bs = std::max<int64_t>(1, h->tc_cap / lps);   // tc_cap >= lps rounded up to 128
  const int lvl = level_of(h, lv);
  for (int64_t s0 = 0; s0 < slabs; s0 += bs) {
    const int64_t ns = std::min(bs, slabs - s0);
    const int64_t nlines = ns * lps;
    const int64_t nlpad = (nlines + stmg_tc::BM - 1) / stmg_tc::BM * stmg_tc::BM;
    const int64_t off = s0 * lv.Nx;
    int64_t inner = 1;
    for (int a = 0; a < h->d; ++a) {
      const double* in = (a == 0 ? src : mid) + off;
      double* out = (a == h->d - 1 ? dst : mid) + off;
      const int oe = axis_exp + (a == 0 ? load_exp : 0) + (a == h->d - 1 ? store_exp : 0);
      {
        Prof pr(h, ST_K_DST, 8.0 * (double)nlines * n, 0.0, 1, lvl);
        const unsigned blocks = (unsigned)(nlpad / stmg_tc::SPLIT_LINES);
        uint4* planes = reinterpret_cast<uint4*>(h->tcD);
        if (a == 0)
          stmg_tc::k_split_planes<true><<<blocks, 256, 0, h->stream>>>(in, n, nlines, inner, nch, h->tcE, planes);
        else
          stmg_tc::k_split_planes<false><<<blocks, 256, 0, h->stream>>>(in, n, nlines, inner, nch, h->tcE, planes);
      }
      {
        const int64_t ntiles = nlpad / stmg_tc::BM * ntn;
        const unsigned grid = (unsigned)std::min<int64_t>(ntiles, h->num_sms);
        Prof pr(h, ST_K_DSTTC, 8.0 * (double)nlines * n, 2.0 * 36.0 * Nf * (double)Nf * (double)nlpad, 1, lvl);
        // the epilogue sets the pace when a tile has few K-chunks: more warps for it there
        constexpr int NL = stmg_tc::NEPI, NS = stmg_tc::NEPI_SHORT;
        const bool shortk = Nf <= 128;
        const unsigned thr = (unsigned)stmg_tc::threads_for(shortk ? NS : NL);
        if (a == 0 && !shortk)
          stmg_tc::k_dst_tc<true, NL><<<grid, thr, stmg_tc::Smem::bytes, h->stream>>>(
              h->tcD, out, n, nlines, inner, h->tcE, lv.tcS, nch, ntn, oe, h->tcErr);
        else if (!shortk)
          stmg_tc::k_dst_tc<false, NL><<<grid, thr, stmg_tc::Smem::bytes, h->stream>>>(
              h->tcD, out, n, nlines, inner, h->tcE, lv.tcS, nch, ntn, oe, h->tcErr);
        else if (a == 0)
          stmg_tc::k_dst_tc<true, NS><<<grid, thr, stmg_tc::Smem::bytes, h->stream>>>(
              h->tcD, out, n, nlines, inner, h->tcE, lv.tcS, nch, ntn, oe, h->tcErr);
        else
          stmg_tc::k_dst_tc<false, NS><<<grid, thr, stmg_tc::Smem::bytes, h->stream>>>(
              h->tcD, out, n, nlines, inner, h->tcE, lv.tcS, nch, ntn, oe, h->tcErr);
      }
      inner *= n;
    }
  }
  check(h, cudaGetLastError(), "tensor-core sine transform");
}

// log2 of an exact power of two (the transform scales 1 and 2 / Nf).
int exact_log2(double s) {
  int e = 0;
  const double m = std::frexp(s, &e);
  return m == 0.5 ? e - 1 : 0x7fffffff;
}

// scale * DST-I along every spatial axis of `slabs` consecutive spatial fields
// of level lv.  The first pass reads src, the last writes dst, intermediate
// results live in mid (src == mid == dst: in place).  `scale` is applied once
// per axis.  src / dst other than mid need the register kernels
// (64 <= n + 1 <= 512); the other kernels work in place on mid.
template <typename T>
void dst_axes(st_handle* h, Level& lv, const T* src, T* mid, T* dst, int64_t slabs, double axis_scale) {
  if (sizeof(T) == 8 && use_tc(h, lv) && exact_log2(axis_scale) != 0x7fffffff) {
    dst_axes_tc(h, lv, reinterpret_cast<const double*>(src), reinterpret_cast<double*>(mid),
                reinterpret_cast<double*>(dst), slabs, exact_log2(axis_scale), 0, 0);
    return;
  }
  const int n = lv.n, Nf = n + 1;
  const int naxes = h->d;
  const bool reg = Nf >= 64 && Nf <= 512;
  if (!reg && src != mid) fail(h, ST_EINVAL, "out-of-place sine transform needs 64 <= n + 1 <= 512");
  if (!reg && dst != mid) fail(h, ST_EINVAL, "out-of-place sine transform needs 64 <= n + 1 <= 512");
  int logh = 0;
  while ((1 << (logh + 1)) <= Nf / 2) ++logh;
  Tables<T>& tb = tables<T>(lv);
  stmg::DstTables<T> dt{tb.sinp, tb.twc, tb.tws};
  const int64_t nlines = slabs * lv.Nx / n;
  const double line_flops = dst_line_flops(n);
  int64_t inner = 1;
  for (int a = 0; a < naxes; ++a) {
    const T scale = (T)axis_scale;
    const T* in = (a == 0) ? src : mid;
    T* out = (a == naxes - 1) ? dst : mid;
    T* data = mid;
    Prof pr(h, ST_K_DST, sizeof(T) * 2.0 * (double)nlines * n, line_flops * (double)nlines, 1, level_of(h, lv));
    if (reg) {
      const int thr = dst_reg_threads<T>();
      const int G = (Nf == 64) ? 4 : (Nf == 512) ? 16 : 8;
      const int rows = thr / G;
      const unsigned grid = (unsigned)((nlines + rows - 1) / rows);
#define STMG_DST_REG(LP, LG)                                                                                   \
  do {                                                                                                         \
    if (a == 0)                                                                                                \
      stmg::k_dst_rows_reg<T, LP, LG><<<grid, thr, dst_reg_smem<T, LP, LG>(), h->stream>>>(in, out, n, nlines, \
                                                                                           scale, dt);         \
    else                                                                                                       \
      stmg::k_dst_cols_reg<T, LP, LG><<<grid, thr, dst_cols_reg_smem<T, LP, LG>(), h->stream>>>(               \
          in, out, n, nlines, inner, scale, dt);                                                               \
  } while (0)
      switch (Nf) {
        case 64: STMG_DST_REG(3, 2); break;
        case 128: STMG_DST_REG(3, 3); break;
        case 256: STMG_DST_REG(4, 3); break;
        default: STMG_DST_REG(4, 4); break;
      }
#undef STMG_DST_REG
    } else if (a == 0) {
      const unsigned grid = (unsigned)((nlines + kDstRowsPerCta - 1) / kDstRowsPerCta);
      stmg::k_dst_rows<T><<<grid, kDstWarps * 32, dst_rows_smem<T>(Nf), h->stream>>>(data, n, logh, nlines,
                                                                                     kDstRowsPerCta, scale, dt);
    } else if (sizeof(T) == 8 && Nf >= 512) {
      const unsigned grid = (unsigned)((nlines + 15) / 16);
      stmg::k_dst_cols<T, 16><<<grid, kDstWarps * 32, dst_cols_smem<T, 16>(Nf), h->stream>>>(data, n, logh, nlines,
                                                                                             inner, scale, dt);
    } else {
      const unsigned grid = (unsigned)((nlines + 31) / 32);
      stmg::k_dst_cols<T, 32><<<grid, kDstWarps * 32, dst_cols_smem<T, 32>(Nf), h->stream>>>(data, n, logh, nlines,
                                                                                             inner, scale, dt);
    }
    inner *= n;
  }
}

template <typename T>
void dst_axes(st_handle* h, Level& lv, T* data, int64_t slabs, double axis_scale) {
  dst_axes<T>(h, lv, data, data, data, slabs, axis_scale);
}

// ---- double-float sine transforms (mixed form): the register kernels with
// dfloat arithmetic on FP64 storage; other line lengths use the FP64 kernels.
bool df_len(int Nf) { return Nf >= 64 && Nf <= 512; }

void make_df_tables(st_handle* h, Level& lv) {
  const int Nf = lv.n + 1;
  std::vector<stmg::dfloat> sp(Nf), tc(Nf), ts(Nf);
  for (int j = 0; j < Nf; ++j) {
    sp[j] = stmg::dfloat(std::sin(j * M_PI / Nf));
    tc[j] = stmg::dfloat(std::cos(2.0 * M_PI * j / Nf));
    ts[j] = stmg::dfloat(std::sin(2.0 * M_PI * j / Nf));
  }
  stmg::dfloat* d[3];
  const std::vector<stmg::dfloat>* src[3] = {&sp, &tc, &ts};
  for (int i = 0; i < 3; ++i) {
    d[i] = reinterpret_cast<stmg::dfloat*>(dalloc<double>(h, Nf));   // 8-byte elements
    check(h, cudaMemcpy(d[i], src[i]->data(), Nf * sizeof(stmg::dfloat), cudaMemcpyHostToDevice), "upload table");
  }
  lv.tdf = stmg::DstTables<stmg::dfloat>{d[0], d[1], d[2]};
}

template <int LP, int LG, typename SIN, typename SOUT>
void df_set_smem_io(st_handle* h) {
  using DF = stmg::dfloat;
  check(h, cudaFuncSetAttribute((const void*)stmg::k_dst_rows_reg<DF, LP, LG, SIN, SOUT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dst_reg_smem<DF, LP, LG>()),
        "cudaFuncSetAttribute");
  check(h, cudaFuncSetAttribute((const void*)stmg::k_dst_cols_reg<DF, LP, LG, SIN, SOUT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dst_cols_reg_smem<DF, LP, LG>()),
        "cudaFuncSetAttribute");
}
template <int LP, int LG>
void df_set_smem(st_handle* h) {
  using DF = stmg::dfloat;
  df_set_smem_io<LP, LG, double, double>(h);
  df_set_smem_io<LP, LG, double, DF>(h);
  df_set_smem_io<LP, LG, DF, DF>(h);
  df_set_smem_io<LP, LG, DF, double>(h);
}

template <int LP, int LG, typename SIN, typename SOUT>
void df_launch_io(st_handle* h, const void* in, void* out, int n, int64_t nlines, int64_t inner, stmg::dfloat scale,
                  stmg::DstTables<stmg::dfloat> dt, bool rows, int load_exp, int store_exp) {
  using DF = stmg::dfloat;
  constexpr int G = 1 << LG;
  const int thr = dst_reg_threads<DF>();
  const unsigned grid = (unsigned)((nlines + thr / G - 1) / (thr / G));
  if (rows)
    stmg::k_dst_rows_reg<DF, LP, LG, SIN, SOUT><<<grid, thr, dst_reg_smem<DF, LP, LG>(), h->stream>>>(
        in, out, n, nlines, scale, dt, load_exp, store_exp);
  else
    stmg::k_dst_cols_reg<DF, LP, LG, SIN, SOUT><<<grid, thr, dst_cols_reg_smem<DF, LP, LG>(), h->stream>>>(
        in, out, n, nlines, inner, scale, dt, load_exp, store_exp);
}

// first / last axis pass: FP64 in / out; between passes the 8-byte slots hold float pairs.
// The first pass scales the FP64 input by 2^load_exp, the last the FP64 output by 2^store_exp.
template <int LP, int LG>
void df_launch(st_handle* h, const void* in, void* out, int n, int64_t nlines, int64_t inner, stmg::dfloat scale,
               stmg::DstTables<stmg::dfloat> dt, bool rows, bool first, bool last, int load_exp, int store_exp) {
  using DF = stmg::dfloat;
  const int le = first ? load_exp : 0, se = last ? store_exp : 0;
  if (first && last) df_launch_io<LP, LG, double, double>(h, in, out, n, nlines, inner, scale, dt, rows, le, se);
  else if (first) df_launch_io<LP, LG, double, DF>(h, in, out, n, nlines, inner, scale, dt, rows, le, se);
  else if (last) df_launch_io<LP, LG, DF, double>(h, in, out, n, nlines, inner, scale, dt, rows, le, se);
  else df_launch_io<LP, LG, DF, DF>(h, in, out, n, nlines, inner, scale, dt, rows, le, se);
}

// Whether the mixed form's boundary transforms of the finest level run in double-float.
bool df_transforms(const st_handle* h, const Level& lv) {
  return h->opt.precision == ST_MIXED && !use_tc(h, lv) && df_len(lv.n + 1) && lv.tdf.sinp != nullptr;
}

// Whether the mixed form's boundary transforms scale the data by 2^df_shift on entry and undo it
// on exit: the double-float transforms and the tensor-core transforms both do (exactly).
bool shift_transforms(const st_handle* h, const Level& lv) {
  return h->opt.precision == ST_MIXED && (use_tc(h, lv) || df_transforms(h, lv));
}

// 2^load_exp * scale * DST-I along every axis of `slabs` FP64 fields, computed in
// double-float (src / mid / dst as in dst_axes), the FP64 result times 2^store_exp.
void dst_axes_df(st_handle* h, Level& lv, const double* src, double* mid, double* dst, int64_t slabs,
                 double axis_scale, int load_exp, int store_exp) {
  const int n = lv.n, Nf = n + 1;
  if (use_tc(h, lv) && exact_log2(axis_scale) != 0x7fffffff) {   // exact FP64 transform, scaled on entry / exit
    dst_axes_tc(h, lv, src, mid, dst, slabs, exact_log2(axis_scale), load_exp, store_exp);
    return;
  }
  if (!df_len(Nf) || lv.tdf.sinp == nullptr) {
    dst_axes<double>(h, lv, src, mid, dst, slabs, axis_scale);
    return;
  }
  const int64_t nlines = slabs * lv.Nx / n;
  const double line_flops = dst_line_flops(n);
  const stmg::dfloat scale(axis_scale);   // 1 or 2 / Nf: exact in FP32
  int64_t inner = 1;
  for (int a = 0; a < h->d; ++a) {
    Prof pr(h, ST_K_DST, 8.0 * 2.0 * (double)nlines * n, line_flops * (double)nlines, 1, level_of(h, lv));
    const bool rows = a == 0, first = a == 0, last = a == h->d - 1;
    const void* in = first ? (const void*)src : (const void*)mid;
    void* out = last ? (void*)dst : (void*)mid;
    switch (Nf) {
      case 64: df_launch<3, 2>(h, in, out, n, nlines, inner, scale, lv.tdf, rows, first, last, load_exp, store_exp);
        break;
      case 128: df_launch<3, 3>(h, in, out, n, nlines, inner, scale, lv.tdf, rows, first, last, load_exp, store_exp);
        break;
      case 256: df_launch<4, 3>(h, in, out, n, nlines, inner, scale, lv.tdf, rows, first, last, load_exp, store_exp);
        break;
      default: df_launch<4, 4>(h, in, out, n, nlines, inner, scale, lv.tdf, rows, first, last, load_exp, store_exp);
        break;
    }
    inner *= n;
  }
}

// Change of basis of `slabs` spatial fields of level lv: nodes -> sine basis
// (S, the unnormalised DST-I along every axis) and back (S^{-1} = (2/Nf)^d S).
template <typename T>
void to_modal(st_handle* h, Level& lv, T* data, int64_t slabs) {
  dst_axes<T>(h, lv, data, slabs, 1.0);
}
template <typename T>
void from_modal(st_handle* h, Level& lv, T* data, int64_t slabs) {
  dst_axes<T>(h, lv, data, slabs, 2.0 / (lv.n + 1));
}

// d = A^{-1} r on nodes, time steps [s0, s0 + ns) (exact block inverse,
// Section 3.1): sine transform along every axis, one q x q solve per mode,
// inverse transform.  r is overwritten (transformed); r and d must differ.
template <typename T>
void block_solve(st_handle* h, Level& lv, bool adj, T* r, T* d, int s0, int ns) {
  const int64_t off = (int64_t)s0 * h->q * lv.Nx;
  to_modal<T>(h, lv, r + off, (int64_t)ns * h->q);
  msmooth<T>(h, lv, adj, false, r, (const T*)nullptr, (const T*)nullptr, d, s0, ns);
  from_modal<T>(h, lv, d + off, (int64_t)ns * h->q);
}

template <typename T>
void axpby(st_handle* h, T* y, const T* x, T a, T b, int64_t n) {
  Prof pr(h, ST_K_VECTOR, 3.0 * sizeof(T) * (double)n, 3.0 * (double)n);
  stmg::k_axpby<T><<<std::min<int64_t>(blocks_for(n), 152 * 16), kThreads, 0, h->stream>>>(y, x, a, b, n);
}

template <typename T>
void axpy(st_handle* h, T* y, const T* x, T a, int64_t n) {
  Prof pr(h, ST_K_VECTOR, 3.0 * sizeof(T) * (double)n, 2.0 * (double)n);
  stmg::k_axpy<T><<<std::min<int64_t>(blocks_for(n), 152 * 16), kThreads, 0, h->stream>>>(y, x, a, n);
}

// Node block D^x = (M_h)_jj K + (K_h)_jj tau Mh of a uniform Q1 grid with spacing hl
// ((M_h)_jj = (2hl/3)^d, (K_h)_jj = d (2/hl)(2hl/3)^(d-1)), inverted; transposed
// K for the adjoint.  On a one-node grid this block is A itself.
void node_block_inverse(const st_handle* h, double hl, double tau, bool adj, double* out) {
  const int q = h->q, d = h->d;
  const double md = std::pow(2.0 * hl / 3.0, d);
  const double kd = d * (2.0 / hl) * std::pow(2.0 * hl / 3.0, d - 1);
  double A[kQmax * kQmax], X[kQmax * kQmax];
  for (int k = 0; k < q; ++k)
    for (int l = 0; l < q; ++l) {
      A[k * q + l] = md * (adj ? h->tm.K[l * q + k] : h->tm.K[k * q + l]) + (k == l ? kd * tau * h->tm.Mh[k] : 0.0);
      X[k * q + l] = (k == l) ? 1.0 : 0.0;
    }
  for (int c = 0; c < q; ++c) {   // Gauss-Jordan with partial pivoting
    int p = c;
    for (int r = c + 1; r < q; ++r)
      if (std::fabs(A[r * q + c]) > std::fabs(A[p * q + c])) p = r;
    if (p != c)
      for (int j = 0; j < q; ++j) {
        std::swap(A[c * q + j], A[p * q + j]);
        std::swap(X[c * q + j], X[p * q + j]);
      }
    const double dv = 1.0 / A[c * q + c];
    for (int j = 0; j < q; ++j) {
      A[c * q + j] *= dv;
      X[c * q + j] *= dv;
    }
    for (int r = 0; r < q; ++r) {
      if (r == c) continue;
      const double f = A[r * q + c];
      for (int j = 0; j < q; ++j) {
        A[r * q + j] -= f * A[c * q + j];
        X[r * q + j] -= f * X[c * q + j];
      }
    }
  }
  for (int i = 0; i < q * q; ++i) out[i] = X[i];
}

// Exact solve on the one-node spatial level, xo = w Dinv b per (mode, step).
template <typename T>
void space_solve(st_handle* h, Level& lv, const SpaceLvl<T>& sl, const T* b, T* xo, double w, const double* dinv) {
  const double nodes = (double)lv.N * sl.Nx, Q = h->q;
  // per (mode, step): Dinv b, Q^2 FMA; read b, write xo
  Prof pr(h, ST_K_SPACEMG, sizeof(T) * Q * nodes * 2.0, 2.0 * nodes * Q * Q, 1, level_of(h, lv));
  STMG_DISPATCH(launch_space_solve_t, h, lv, sl, b, xo, w, dinv);
}

template <typename T>
void space_restrict(st_handle* h, Level& lv, const SpaceLvl<T>& fine, const SpaceLvl<T>& coarse, const T* in,
                    T* out) {
  Prof pr(h, ST_K_SPACEMG, sizeof(T) * h->q * (double)lv.N * (fine.Nx + coarse.Nx),
          2.0 * h->q * (double)lv.N * coarse.Nx * std::pow(2.0, h->d), 1, level_of(h, lv));
  STMG_DISPATCH(launch_space_restrict_t, h, lv, fine, coarse, in, out);
}

// x = D~^{-1} b on every time step of level lv: one spatial V-cycle from x = 0
// (Remark on the V-cycle approximation in space), spatial level ell.
template <typename T>
// upd (finest spatial grid only, which must have more than one node): the
// result is not stored in x but added to upd, times omega_t (the damped update
// of the smoothing step).
void space_vcycle(st_handle* h, Level& lv, int ell, bool adj, T* x, const T* b, T* upd = nullptr) {
  std::vector<SpaceLvl<T>>& sp = spaces<T>(lv);
  const SpaceLvl<T>& sl = sp[ell];
  double dinv[kQmax * kQmax];
  node_block_inverse(h, sl.h, lv.tau, adj, dinv);
  if (sl.n == 1) {   // one node: D^x = A, exact solve
    space_solve<T>(h, lv, sl, b, x, 1.0, dinv);
    return;
  }
  // pre-smoothing (nu_x sweeps from 0) and the spatial residual in one pass per
  // (mode, step); restriction; coarse cycle; correction and post-smoothing in one pass
  const double w = h->opt.omega_x;
  const double nodes = (double)lv.N * sl.Nx, Q = h->q, nu = h->opt.nu_x;
  {
    Prof pr(h, ST_K_SPACEMG, sizeof(T) * Q * nodes * 3.0, 2.0 * nodes * (nu * (2.0 * Q * Q + Q) + Q * Q), 1,
            level_of(h, lv));
    STMG_DISPATCH(launch_space_pre_t, h, lv, sl, adj, b, x, sl.t, w, dinv);
  }
  const SpaceLvl<T>& cl = sp[ell + 1];
  space_restrict<T>(h, lv, sl, cl, sl.t, cl.b);
  space_vcycle<T>(h, lv, ell + 1, adj, cl.x, cl.b);
  Prof pr(h, ST_K_SPACEMG, sizeof(T) * Q * (double)lv.N * ((upd ? 4.0 : 3.0) * sl.Nx + cl.Nx),
          2.0 * nodes * (nu * (2.0 * Q * Q + Q) + Q + (upd ? 1.0 : 0.0)), 1, level_of(h, lv));
  STMG_DISPATCH(launch_space_post_t, h, lv, sl, cl, adj, b, x, cl.x, w, dinv, upd, h->opt.omega);
}

bool inexact(const st_handle* h) { return h->opt.smoother == ST_SMOOTH_VCYCLE; }

// d = D~^{-1} r on nodes, the smoother's block inverse (exact, or one spatial
// V-cycle), computed in the sine basis.  r and d may be the same buffer.
template <typename T>
void smoother_block_solve(st_handle* h, Level& lv, bool adj, const T* r, T* d) {
  T* tmp = vecs<T>(lv).f;
  copy<T>(h, tmp, r, lv.ndof);
  if (!inexact(h)) {
    block_solve<T>(h, lv, adj, tmp, d, 0, lv.N);
    return;
  }
  const int64_t slabs = (int64_t)lv.N * h->q;
  to_modal<T>(h, lv, tmp, slabs);
  space_vcycle<T>(h, lv, 0, adj, d, tmp);
  from_modal<T>(h, lv, d, slabs);
}

// One damped block-Jacobi step with the inexact block inverse in the sine
// basis (eq. chap4_smootherApprox): u <- u + w D~^{-1} (f - L u).
template <typename T>
void smooth_step_inexact(st_handle* h, Level& lv, bool adj, T* u, const T* f, const T* u0, T* work) {
  mresidual<T>(h, lv, adj, f, u, u0, work);
  T* d = spaces<T>(lv)[0].x;
  if (spaces<T>(lv)[0].n > 1) {   // the update u += omega_t d done by the last spatial pass
    space_vcycle<T>(h, lv, 0, adj, d, work, u);
  } else {
    space_vcycle<T>(h, lv, 0, adj, d, work);
    axpy<T>(h, u, d, (T)h->opt.omega, lv.ndof);
  }
}

// nu damped block-Jacobi steps (eq. chap4_smoother) with the exact block
// inverse in the sine basis, u <- (1 - w) u + w A^{-1} (f - B u_prev) (the
// block inverse of the block row removes A u, so only the rank-one time
// coupling is applied).  Each step reads one buffer and writes the other
// (Jacobi in time); the first destination is chosen so that the last step
// lands in u.  u_zero: u holds zero on entry and is not read.
// Where the level has a wf buffer the steps run on wf = w A^{-1} f: wf_ready
// says that it already holds that product for this f and direction (an
// earlier smoothing of the same right-hand side); otherwise the first step
// forms it.
// in_tmp: the current iterate is in tmp (after a fused first step), not in u.
template <typename T>
void smooth_modal(st_handle* h, Level& lv, bool adj, T* u, const T* f, const T* u0, T* tmp, int nu, bool u_zero,
                  bool wf_ready = false, bool in_tmp = false) {
  if (nu <= 0) {
    if (u_zero) zero<T>(h, u, lv.ndof);
    if (in_tmp) copy<T>(h, u, tmp, lv.ndof);
    return;
  }
  T* wf = vecs<T>(lv).wf;
  T* buf[2] = {u, tmp};
  int cur = u_zero ? -1 : (in_tmp ? 1 : 0);
  int dst = u_zero ? ((nu & 1) ? 0 : 1) : 1 - cur;
  for (int i = 0; i < nu; ++i) {
    const T* ui = cur < 0 ? (const T*)nullptr : buf[cur];
    if (wf == nullptr) {
      msmooth<T>(h, lv, adj, true, f, ui, u0, buf[dst]);
    } else if (!wf_ready) {
      msmooth<T>(h, lv, adj, true, f, ui, u0, buf[dst], 0, -1, stmg::kMakeWf, wf);
      wf_ready = true;
    } else {
      msmooth<T>(h, lv, adj, true, (const T*)wf, ui, u0, buf[dst], 0, -1, stmg::kUseWf);
    }
    cur = dst;
    dst = 1 - dst;
  }
  if (cur != 0) copy<T>(h, u, tmp, lv.ndof);
}

// Exact coarsest solve (Section 2) by forward (adjoint: backward) substitution,
// one block inverse per step with the coupling to the step solved before.
// One undamped k_fsmooth launch per step (sine basis).
template <typename T>
void coarsest_modal(st_handle* h, bool adj, T* u, const T* f, const T* u0) {
  Level& lv = h->levels[0];
  for (int i = 0; i < lv.N; ++i) {
    const int s = adj ? lv.N - 1 - i : i;
    msmooth<T>(h, lv, adj, false, f, u, u0, u, s, 1);
  }
}

void coarsest_fp64(st_handle* h, bool adj, double* u, const double* f, const double* u0) {
  coarsest_modal<double>(h, adj, u, f, u0);
}

// Mixed precision: the coarsest level is solved in FP64.
void coarsest_mixed(st_handle* h, bool adj, float* u, const float* f) {
  Level& lv = h->levels[0];
  const int64_t n = lv.ndof;
  {
    Prof pr(h, ST_K_VECTOR, 12.0 * (double)n, 0.0);
    stmg::k_cast_up<<<blocks_for(n), kThreads, 0, h->stream>>>(h->coarse64_f, f, n);
  }
  coarsest_modal<double>(h, adj, h->coarse64_u, h->coarse64_f, (const double*)nullptr);
  Prof pr(h, ST_K_VECTOR, 12.0 * (double)n, 0.0);
  stmg::k_cast_down<<<blocks_for(n), kThreads, 0, h->stream>>>(u, h->coarse64_u, 1.0, n);
}

template <typename T>
void coarsest_solve(st_handle* h, bool adj, T* u, const T* f, const T* u0);
template <>
void coarsest_solve<double>(st_handle* h, bool adj, double* u, const double* f, const double* u0) {
  coarsest_fp64(h, adj, u, f, u0);
}
template <>
void coarsest_solve<float>(st_handle* h, bool adj, float* u, const float* f, const float* u0) {
  (void)u0;   // inner cycles of the mixed form carry no initial value
  coarsest_mixed(h, adj, u, f);
}

// Multigrid cycle on level L for L u = f (+ the initial-value term u0 on the
// finest level), Section 2: the coarse correction equation is treated by gamma
// cycles on level L-1 (1: V-cycle, 2: W-cycle; once when L-1 is the coarsest
// level, whose solve is exact).  With the exact block inverse every vector is
// in the sine basis.  u_zero: u holds zero on entry (coarse-grid corrections).
// wf_ready: the level's wf already holds w A^{-1} f for this f and direction
// (a cycle repeated on the same right-hand side).
template <typename T>
void vcycle(st_handle* h, int L, bool adj, T* u, const T* f, const T* u0, bool u_zero, bool wf_ready = false) {
  Level& lv = h->levels[L];
  T* work = vecs<T>(lv).r;
  if (L == 0) {
    coarsest_solve<T>(h, adj, u, f, u0);
    return;
  }
  if (!inexact(h)) {
    smooth_modal<T>(h, lv, adj, u, f, u0, work, h->opt.nu1, u_zero, wf_ready);
  } else {
    if (u_zero) zero<T>(h, u, lv.ndof);
    for (int i = 0; i < h->opt.nu1; ++i) smooth_step_inexact<T>(h, lv, adj, u, f, u0, work);
  }
  mresidual<T>(h, lv, adj, f, u, u0, work);
  Level& cl = h->levels[L - 1];
  Vecs<T>& cv = vecs<T>(cl);
  restrict_to<T>(h, L, work, cv.f);
  const int reps = (L - 1 == 0) ? 1 : h->opt.gamma;
  for (int g = 0; g < reps; ++g) vcycle<T>(h, L - 1, adj, cv.u, cv.f, (const T*)nullptr, g == 0, g > 0);
  const bool post_ready = wf_ready || h->opt.nu1 > 0;   // wf holds w A^{-1} f (where the level has wf)
  T* wf = vecs<T>(lv).wf;
  // the correction fused into the first post-smoothing step (FP32 cycles, which are HBM-bound: the
  // fused pass saves reading and writing u; the FP64 pipe-bound cycles gain nothing and recompute the
  // correction of the neighbouring step): full coarsening, q <= kQfix, an even number of post-steps
  // (the last one lands in u) and a step that reads f or a ready wf
  const bool fuse = sizeof(T) == 4 && !inexact(h) && lv.coarsen_full && h->q <= kQfix && h->opt.nu2 >= 2 &&
                    h->opt.nu2 % 2 == 0 && (wf == nullptr || post_ready);
  if (fuse) {
    const int fm = wf ? stmg::kUseWf : stmg::kFromF;
    prolong_smooth<T>(h, L, adj, fm, cv.u, wf ? (const T*)wf : f, u, u0, work);
    smooth_modal<T>(h, lv, adj, u, f, u0, work, h->opt.nu2 - 1, false, true, true);
  } else if (!inexact(h)) {
    prolong_add<T>(h, L, cv.u, u);
    smooth_modal<T>(h, lv, adj, u, f, u0, work, h->opt.nu2, false, post_ready);
  } else {
    prolong_add<T>(h, L, cv.u, u);
    for (int i = 0; i < h->opt.nu2; ++i) smooth_step_inexact<T>(h, lv, adj, u, f, u0, work);
  }
}

// Residual of the finest level in the basis of the cycle.
template <typename T>
void cycle_residual(st_handle* h, Level& lv, bool adj, const T* f, const T* u, const T* u0, T* r) {
  mresidual<T>(h, lv, adj, f, u, u0, r);
}

template <typename T>
double norm2(st_handle* h, const T* x, int64_t n) {
  {
    Prof pr(h, ST_K_NORM, sizeof(T) * (double)n, 2.0 * (double)n, 2);
    stmg::k_sumsq_partial<T><<<kNormBlocks, kThreads, 0, h->stream>>>(x, n, h->partial);
    stmg::k_sum_final<<<1, 1024, 0, h->stream>>>(h->partial, kNormBlocks, h->dnorm);
  }
  check(h, cudaMemcpyAsync(h->hnorm, h->dnorm, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "norm copy");
  if (h->tcErr)
    check(h, cudaMemcpyAsync(h->hnorm + 1, h->tcErr, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "flag copy");
  check(h, cudaStreamSynchronize(h->stream), "norm sync");
  tc_check_flag(h);
  return std::sqrt(*h->hnorm);
}

Level& finest(st_handle* h) { return h->levels.back(); }

template <typename T, int D, int Q>
void launch_residual_norm_t(st_handle* h, Level& lv, bool adj, const double* f, const double* u, const double* u0,
                            float* r32) {
  static_assert(sizeof(T) == 8, "the residual with norm is the FP64 outer residual");
  Tables<double>& tb = lv.t64;
  constexpr int TS = stmg::kStepsPerThread;
  const int nblk = (lv.N + TS - 1) / TS;
  dim3 grid(blocks_for(lv.Nx), 1);
  for (int c = 0; c < nblk; c += 65535) {
    grid.y = std::min(65535, nblk - c);
    const int64_t pbase = (int64_t)c * grid.x;
#define STMG_RN(ADJ, S32)                                                                                  \
  stmg::k_fresidual_norm<Q, ADJ, S32><<<grid, kThreads, 0, h->stream>>>(f, u, u0, r32, lv.Nx, lv.N, c * TS, lv.N, \
                                                                        tb.amat[adj ? 1 : 0], tb.lamM, h->partial, \
                                                                        pbase)
    if (adj) {
      if (r32) STMG_RN(true, true); else STMG_RN(true, false);
    } else {
      if (r32) STMG_RN(false, true); else STMG_RN(false, false);
    }
#undef STMG_RN
  }
}

// ||f - L u|| on the finest level (u == nullptr: zero iterate) in one pass with
// the residual (k_fresidual_norm; q <= kQfix), storing the residual rounded to
// FP32 in r32 when given; larger q: residual into the work vector, then norm2.
double residual_norm(st_handle* h, bool adj, const double* f, const double* u, const double* u0, float* r32) {
  Level& lv = finest(h);
  if (h->q > kQfix) {   // the residual stays in the finest FP64 work vector (the mixed form's r64)
    if (r32) fail(h, ST_EINVAL, "internal: FP32 residual output needs q <= 4");
    cycle_residual<double>(h, lv, adj, f, u, u0, lv.v64.r);
    return norm2<double>(h, lv.v64.r, lv.ndof);
  }
  {
    const double Q = h->q, nodes = (double)lv.N * lv.Nx;
    using T = double;
    Prof pr(h, ST_K_RESIDUAL,
            8.0 * ((u ? 2.0 : 1.0) * nodes * Q + (u0 ? (double)lv.Nx : 0.0)) + (r32 ? 4.0 * nodes * Q : 0.0),
            (u ? nodes * (2.0 * Q * Q + 2.0 * Q) : 0.0) + 2.0 * nodes * Q, 1, level_of(h, lv));
    STMG_DISPATCH(launch_residual_norm_t, h, lv, adj, f, u, u0, r32);
    const int64_t np = (int64_t)blocks_for(lv.Nx) * ((lv.N + stmg::kStepsPerThread - 1) / stmg::kStepsPerThread);
    stmg::k_sum_final<<<1, 1024, 0, h->stream>>>(h->partial, (int)np, h->dnorm);
  }
  check(h, cudaMemcpyAsync(h->hnorm, h->dnorm, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "norm copy");
  if (h->tcErr)
    check(h, cudaMemcpyAsync(h->hnorm + 1, h->tcErr, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "flag copy");
  check(h, cudaStreamSynchronize(h->stream), "norm sync");
  tc_check_flag(h);
  return std::sqrt(*h->hnorm);
}

// One FP64 refinement step of the mixed-precision form: given the FP64 residual
// r (norm s), solve L e = r / s approximately with FP32 V-cycles and update
// u += s e in FP64 (all in the basis of the cycle).
// r == nullptr: the FP32 right-hand side is already in the finest FP32 f
// (the unscaled residual from residual_norm) and s must be 1.
void mixed_step(st_handle* h, bool adj, double* u, const double* r, double s) {
  Level& lv = finest(h);
  const int L = (int)h->levels.size() - 1;
  Vecs<float>& v = lv.v32;
  if (r != nullptr) {
    Prof pr(h, ST_K_VECTOR, 12.0 * (double)lv.ndof, (double)lv.ndof);
    stmg::k_cast_down<<<std::min<int64_t>(blocks_for(lv.ndof), 152 * 16), kThreads, 0, h->stream>>>(
        v.f, r, 1.0 / s, lv.ndof);
  }
  for (int c = 0; c < std::max(1, h->opt.inner_cycles); ++c)
    vcycle<float>(h, L, adj, v.u, v.f, (const float*)nullptr, c == 0, c > 0);
  Prof pr(h, ST_K_VECTOR, 20.0 * (double)lv.ndof, 2.0 * (double)lv.ndof);
  stmg::k_axpy_up<<<std::min<int64_t>(blocks_for(lv.ndof), 152 * 16), kThreads, 0, h->stream>>>(u, v.u, s, lv.ndof);
}

// Inputs of a finest-level cycle in its basis: f and u0 are transformed into
// handle buffers (u in place).
struct CycleInputs {
  const double* f;
  const double* u0;
};

// Basis change of the finest-level FP64 vectors at the boundary of a solve: in
// FP64, or in double-float on the FP32 pipe for the mixed form.
// The double-float transforms take the data scaled by 2^df_shift on entry and
// undo the scaling on exit (inverse).
void boundary_dst(st_handle* h, const double* src, double* mid, double* dst, int64_t slabs, bool inverse) {
  Level& lv = finest(h);
  const double sc = inverse ? 2.0 / (lv.n + 1) : 1.0;
  if (h->opt.precision == ST_MIXED)
    dst_axes_df(h, lv, src, mid, dst, slabs, sc, inverse ? 0 : h->df_shift, inverse ? -h->df_shift : 0);
  else dst_axes<double>(h, lv, src, mid, dst, slabs, sc);
}

// Mixed form: the FP32 cycles (and the double-float pairs) have the FP32 exponent range,
// and the FP64 norms square the data, so data whose largest magnitude lies outside
// 2^-64 ... 2^64 enter the transforms scaled by the power of two that brings it into
// [1, 2) (exact; every later step is linear, so the cycles solve the scaled problem and
// the inverse transform undoes the scale).
// Sets h->df_shift from the finite entries of f, u0 and u (u0, u may be null);
// reads one device word back (synchronises the stream).
void choose_df_shift(st_handle* h, const double* f, const double* u0, const double* u) {
  Level& lv = finest(h);
  h->df_shift = 0;
  if (!shift_transforms(h, lv)) return;
  check(h, cudaMemsetAsync(h->dmaxexp, 0, sizeof(unsigned), h->stream), "memset");
  auto scan = [&](const double* x, int64_t n) {
    if (x == nullptr || n == 0) return;
    Prof pr(h, ST_K_VECTOR, 8.0 * (double)n, 0.0);
    stmg::k_max_exponent<<<(unsigned)std::min<int64_t>(blocks_for(n), 152 * 8), kThreads, 0, h->stream>>>(
        x, n, h->dmaxexp);
  };
  scan(f, lv.ndof);
  scan(u0, lv.Nx);
  scan(u, lv.ndof);
  unsigned emax = 0;
  check(h, cudaMemcpyAsync(h->hnorm, h->dmaxexp, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream), "copy");
  check(h, cudaStreamSynchronize(h->stream), "sync");
  std::memcpy(&emax, h->hnorm, sizeof(unsigned));
  if (emax == 0u) return;                            // all entries zero (or FP64 subnormal)
  const int e = (int)emax - 1023;                    // 2^e <= max |x| < 2^(e+1)
  if (e < -64 || e > 64) h->df_shift = -e;
}
void boundary_dst(st_handle* h, double* data, int64_t slabs, bool inverse) {
  boundary_dst(h, data, data, data, slabs, inverse);
}

CycleInputs enter_cycle_basis(st_handle* h, const double* f, const double* u0, double* u, bool u_given) {
  Level& lv = finest(h);
  choose_df_shift(h, f, u0, u_given ? u : nullptr);
  if (lv.n + 1 >= 64 && lv.n + 1 <= 512) {   // the register transforms read f and write the handle's copy
    boundary_dst(h, f, lv.v64.f, lv.v64.f, (int64_t)lv.N * h->q, false);
  } else {
    copy<double>(h, lv.v64.f, f, lv.ndof);
    boundary_dst(h, lv.v64.f, (int64_t)lv.N * h->q, false);
  }
  const double* u0m = nullptr;
  if (u0) {
    copy<double>(h, h->u0m, u0, lv.Nx);
    boundary_dst(h, h->u0m, 1, false);
    u0m = h->u0m;
  }
  if (u_given) boundary_dst(h, u, (int64_t)lv.N * h->q, false);
  return {lv.v64.f, u0m};
}

void leave_cycle_basis(st_handle* h, double* u) {
  Level& lv = finest(h);
  boundary_dst(h, u, (int64_t)lv.N * h->q, true);
}

// The cycles of a solve with the inputs already in the basis of the cycle.
// Without a given iterate the FP64 form starts from u = 0 without storing it:
// the first residual and the first cycle treat u as zero, and u is only
// filled with zeros when no cycle runs.
int solve_core(st_handle* h, bool adj, const CycleInputs& in, double* u, bool given, int* iters, double* relres) {
  Level& lv = finest(h);
  const int L = (int)h->levels.size() - 1;
  const bool mixed = h->opt.precision == ST_MIXED;
  if (!given && mixed) zero<double>(h, u, lv.ndof);   // the refinement adds into u
  bool u_zero = !given && !mixed;
  double* r = mixed ? h->r64 : lv.v64.r;
  // the residual and its norm in one pass; the mixed form also gets the residual
  // rounded to FP32, the right-hand side of its next FP32 cycles
  float* r32 = (mixed && h->q <= kQfix) ? lv.v32.f : nullptr;
  // the sine transform is orthogonal up to a constant factor, so the relative
  // residual is the same in both bases
  const double r0 = residual_norm(h, adj, in.f, u_zero ? (const double*)nullptr : u, in.u0, r32);
  double rn = r0;
  // the unscaled FP32 residual serves as right-hand side while its entries stay far from the FP32
  // range limits; otherwise the FP64 residual is recomputed and scaled by its norm
  auto fp32_rhs_ok = [&](double nrm) {
    const double rms = nrm / std::sqrt((double)lv.ndof);
    return r32 != nullptr && rms > 1e-20 && rms < 1e20;
  };
  int it = 0;
  int status = ST_OK;
  if (!std::isfinite(r0)) status = ST_ENAN;
  while (status == ST_OK && r0 > 0.0 && rn > h->opt.rtol * r0) {
    if (it >= h->opt.maxit) { status = ST_ENOTCONV; h->err = "maxit reached"; break; }
    if (mixed) {
      if (fp32_rhs_ok(rn)) {
        mixed_step(h, adj, u, nullptr, 1.0);
      } else {
        // q > kQfix: residual_norm left the FP64 residual in r already
        if (h->q <= kQfix) cycle_residual<double>(h, lv, adj, in.f, u, in.u0, r);
        mixed_step(h, adj, u, r, rn);
      }
    } else {
      vcycle<double>(h, L, adj, u, in.f, in.u0, u_zero, it > 0);   // in.f is fixed for the whole solve
      u_zero = false;
    }
    ++it;
    rn = residual_norm(h, adj, in.f, u, in.u0, r32);
    if (!std::isfinite(rn)) { status = ST_ENAN; h->err = "residual norm is not finite"; break; }
    if (rn > 1e6 * r0) { status = ST_ENOTCONV; h->err = "residual grew by 1e6"; break; }
  }
  if (u_zero) zero<double>(h, u, lv.ndof);
  if (iters) *iters = it;
  if (relres) *relres = r0 > 0.0 ? rn / r0 : 0.0;
  return status;
}

int solve_impl(st_handle* h, bool adj, const double* f, const double* u0, double* u, int flags, int* iters,
               double* relres) {
  const bool given = (flags & ST_INIT_GIVEN) != 0;
  const CycleInputs in = enter_cycle_basis(h, f, u0, u, given);
  const int status = solve_core(h, adj, in, u, given, iters, relres);
  leave_cycle_basis(h, u);
  return status;
}

// Device address of a host buffer that kernels may read and write in place:
// page-locked memory registered with CUDA, reached over the CPU-GPU
// interconnect (on this system the host pointer itself is the device
// address).  nullptr for pageable or unknown memory.
const void* device_view(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr) return nullptr;
  return at.devicePointer;
}

// Solve with host buffers.  With a register sine-transform length, the first
// transform pass reads f from registered host
// memory and the last inverse pass writes u to it, so the transfers ride on the
// transforms instead of separate copies; otherwise plain copies.
int solve_host_impl(st_handle* h, const double* f, const double* u0, double* u, int flags, int* iters,
                    double* relres) {
  Level& lv = finest(h);
  const bool given = (flags & ST_INIT_GIVEN) != 0;
  const int64_t slabs = (int64_t)lv.N * h->q;
  const size_t bytes = sizeof(double) * lv.ndof;
  if (!h->u_dev) h->u_dev = dalloc<double>(h, lv.ndof);
  const bool md = true;   // every cycle runs in the sine basis
  const bool in_place = lv.n + 1 >= 64 && lv.n + 1 <= 512;
  const double* fv = in_place ? static_cast<const double*>(device_view(f)) : nullptr;
  double* uv = in_place ? static_cast<double*>(const_cast<void*>(device_view(u))) : nullptr;
  CycleInputs in{lv.v64.f, nullptr};
  if (u0) {
    check(h, cudaMemcpyAsync(h->u0m, u0, sizeof(double) * lv.Nx, cudaMemcpyHostToDevice, h->stream), "copy u0");
    in.u0 = h->u0m;
  }
  if (!fv) check(h, cudaMemcpyAsync(lv.v64.f, f, bytes, cudaMemcpyHostToDevice, h->stream), "copy f");
  if (given && !uv) check(h, cudaMemcpyAsync(h->u_dev, u, bytes, cudaMemcpyHostToDevice, h->stream), "copy u");
  choose_df_shift(h, fv ? fv : lv.v64.f, in.u0, given ? (uv ? (const double*)uv : h->u_dev) : nullptr);
  if (u0 && md) boundary_dst(h, h->u0m, 1, false);
  if (fv) boundary_dst(h, fv, lv.v64.f, lv.v64.f, slabs, false);
  else if (md) boundary_dst(h, lv.v64.f, slabs, false);
  if (given) {
    if (uv) boundary_dst(h, uv, h->u_dev, h->u_dev, slabs, false);
    else if (md) boundary_dst(h, h->u_dev, slabs, false);
  }
  const int status = solve_core(h, false, in, h->u_dev, given, iters, relres);
  if (uv) {
    boundary_dst(h, h->u_dev, h->u_dev, uv, slabs, true);
  } else {
    if (md) boundary_dst(h, h->u_dev, slabs, true);
    check(h, cudaMemcpyAsync(u, h->u_dev, bytes, cudaMemcpyDeviceToHost, h->stream), "copy u back");
  }
  check(h, cudaStreamSynchronize(h->stream), "solve_host sync");
  return status;
}

bool is_pow2m1(int n) { return n >= 1 && ((n + 1) & n) == 0; }
bool is_pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

template <typename F>
int guarded(st_handle* h, F&& fn) {
  if (!h) return ST_EINVAL;
  try {
    h->err.clear();
    return fn();
  } catch (const Fail& e) {
    return e.code;
  } catch (const std::bad_alloc&) {
    h->err = "host allocation failed";
    return ST_ENOMEM;
  } catch (...) {
    h->err = "unexpected error";
    return ST_ECUDA;
  }
}

void after_launch(st_handle* h) { check(h, cudaGetLastError(), "kernel launch"); }

int level_index(st_handle* h, int L) {
  if (L < 0 || L >= (int)h->levels.size()) fail(h, ST_EINVAL, "level out of range");
  return L;
}

}  // namespace

// =========================================================================== C ABI
extern "C" {

void st_default_options(st_options* o) {
  if (!o) return;
  o->nu1 = 2;
  o->nu2 = 2;
  o->omega = 0.5;
  o->rtol = 1e-8;
  o->maxit = 50;
  o->precision = ST_FP64;
  o->coarsening = ST_AUTO;
  o->coarsest_steps = 1;
  o->inner_cycles = 1;
  o->max_workspace_bytes = 0;
  o->smoother = ST_SMOOTH_EXACT;
  o->nu_x = 2;
  o->omega_x = 2.0 / 3.0;
  o->gamma = 1;
  o->transform = ST_DST_AUTO;
}

namespace {

// Argument checks of st_setup (and st_plan): the message of the first
// violation, or nullptr.  o receives the options with defaults applied.
const char* check_setup_args(const st_mesh* mesh, int p_t, int N, double T, const st_options* opt,
                             st_options& o) {
  if (!mesh || mesh->dim < 1 || mesh->dim > 3 || !is_pow2m1(mesh->n)) return "mesh: dim 1..3, n = 2^k-1";
  if (mesh->n > 1023) return "mesh: n <= 1023";
  if (p_t < 0 || p_t > ST_MAX_PT) return "p_t out of range";
  if (!is_pow2(N)) return "N must be a power of 2";
  if (N > 32768) return "N <= 32768 (the transfer and spatial kernels put the steps on the second grid axis)";
  if (!(T > 0.0) || !std::isfinite(T)) return "T must be positive";
  if (opt) o = *opt; else st_default_options(&o);
  if (o.nu1 < 0 || o.nu2 < 0 || !(o.omega > 0.0) || o.maxit < 0 || !(o.rtol >= 0.0)) return "bad options";
  if (o.precision != ST_FP64 && o.precision != ST_MIXED) return "bad precision";
  if (o.coarsening < ST_AUTO || o.coarsening > ST_FULL) return "bad coarsening";
  if (o.smoother != ST_SMOOTH_EXACT && o.smoother != ST_SMOOTH_VCYCLE) return "bad smoother";
  if (o.smoother == ST_SMOOTH_VCYCLE && (o.nu_x < 1 || !(o.omega_x > 0.0))) return "bad spatial smoothing options";
  if (o.smoother == ST_SMOOTH_VCYCLE && p_t + 1 > kQfix) return "the inexact block inverse supports p_t <= 3";
  if (o.gamma < 1 || o.gamma > 2) return "gamma must be 1 (V-cycle) or 2 (W-cycle)";
  if (o.transform < ST_DST_AUTO || o.transform > ST_DST_TENSOR) return "bad transform";
  if (o.transform == ST_DST_TENSOR && !tc_len(mesh->n + 1)) return "the tensor-core transform needs 64 <= n + 1 <= 256";
  if (o.coarsest_steps < 1) o.coarsest_steps = 1;
  if (!is_pow2(o.coarsest_steps) || o.coarsest_steps > N) return "bad coarsest_steps";
  return nullptr;
}

struct PlanLevel {
  int N = 0, n = 0;
  double tau = 0, h = 0, mu = 0;
  int coarsen_full = 0;   // how this level is restricted to the next coarser one
};

// Coarsening plan, finest level first (Section 2; Section 4 with the Remark on
// the critical parameter): halve the steps on every level; also halve the
// spatial grid (full coarsening) when mu_L = tau_L / h_L^2 >= mu* (automatic
// rule; up to a relative 1e-12) and the grid has at least 3 nodes; stop at
// coarsest_steps steps.
std::vector<PlanLevel> plan_levels(int n, int p_t, int N, double T, const st_options& o) {
  const double ms = mu_star(p_t);
  std::vector<PlanLevel> out;
  int Nl = N, nl = n;
  double tau = T / N;
  while (true) {
    PlanLevel L;
    L.N = Nl;
    L.n = nl;
    L.tau = tau;
    L.h = 1.0 / (nl + 1);
    L.mu = tau / (L.h * L.h);
    if (Nl <= o.coarsest_steps) {
      out.push_back(L);
      break;
    }
    bool full;
    if (o.coarsening == ST_SEMI) full = false;
    else if (o.coarsening == ST_FULL) full = nl >= 3;
    else full = (L.mu >= ms * (1.0 - 1e-12)) && nl >= 3;
    L.coarsen_full = full ? 1 : 0;
    out.push_back(L);
    Nl /= 2;
    tau *= 2.0;
    if (full) nl = (nl - 1) / 2;
  }
  return out;
}

}  // namespace

int st_setup(const st_mesh* mesh, int p_t, int N, double T, const st_options* opt, void* cuda_stream,
             st_handle** out) {
  if (!out) return ST_EINVAL;
  *out = nullptr;
  st_handle* h = new (std::nothrow) st_handle();
  if (!h) return ST_ENOMEM;
  int rc = guarded(h, [&]() -> int {
    if (const char* bad = check_setup_args(mesh, p_t, N, T, opt, h->opt)) fail(h, ST_EINVAL, bad);
    h->d = mesh->dim;
    h->p_t = p_t;
    h->q = p_t + 1;
    h->N = N;
    h->T = T;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->tm = make_time(p_t);
    // hierarchy, finest first, then reversed to the paper's numbering (0 = coarsest)
    std::vector<Level> lv;
    for (const PlanLevel& P : plan_levels(mesh->n, p_t, N, T, h->opt)) {
      Level L;
      L.N = P.N;
      L.n = P.n;
      L.tau = P.tau;
      L.h = P.h;
      L.mu = P.mu;
      L.coarsen_full = P.coarsen_full;
      L.Nx = 1;
      for (int a = 0; a < h->d; ++a) L.Nx *= P.n;
      L.ndof = (int64_t)P.N * h->q * L.Nx;
      lv.push_back(L);
    }
    std::reverse(lv.begin(), lv.end());
    h->levels = lv;
    const int nlev = (int)h->levels.size();
    const bool mixed = h->opt.precision == ST_MIXED;
    for (int L = 0; L < nlev; ++L) {
      Level& l = h->levels[L];
      if (L < nlev - 1) l.v64.u = dalloc<double>(h, l.ndof);
      l.v64.f = dalloc<double>(h, l.ndof);   // finest level: the transformed right-hand side
      l.v64.r = dalloc<double>(h, l.ndof);
      // damped steps on wf = w A^{-1} f (FP64 cycles are bound by the FP64 pipe; FP32 ones by HBM, where
      // the extra wf store would cost, except at generic q with its q^2 inverse per step)
      if (!inexact(h) && !mixed && L > 0) l.v64.wf = dalloc<double>(h, l.ndof);
      make_tables<double>(h, l, l.t64);
      if (h->opt.smoother == ST_SMOOTH_VCYCLE) make_space<double>(h, l, l.sp64);
      if (mixed) {
        l.v32.u = dalloc<float>(h, l.ndof);
        l.v32.f = dalloc<float>(h, l.ndof);
        l.v32.r = dalloc<float>(h, l.ndof);
        if (!inexact(h) && h->q > kQfix && L > 0) l.v32.wf = dalloc<float>(h, l.ndof);
        make_tables<float>(h, l, l.t32);
        if (h->opt.smoother == ST_SMOOTH_VCYCLE) make_space<float>(h, l, l.sp32);
      }
    }
    if (mixed) {
      Level& c = h->levels[0];
      h->coarse64_u = dalloc<double>(h, c.ndof);
      h->coarse64_f = dalloc<double>(h, c.ndof);
      h->coarse64_r = dalloc<double>(h, c.ndof);
      h->r64 = finest(h).v64.r;
    }
    h->u0m = dalloc<double>(h, finest(h).Nx);
    {   // time tables of the generic-q kernels
      const int q = h->q;
      std::vector<double> mh(q), r1(q * q), r2(q * q), p1(q * q), p2(q * q);
      const double sc = (double)(1 << h->d);
      for (int k = 0; k < q; ++k) mh[k] = h->tm.Mh[k];
      for (int e = 0; e < q * q; ++e) {
        r1[e] = h->tm.R1[e];
        r2[e] = h->tm.R2[e];
        p1[e] = sc * r1[e];
        p2[e] = sc * r2[e];
      }
      const std::vector<double>* src[5] = {&mh, &r1, &r2, &p1, &p2};
      for (int i = 0; i < 5; ++i) {
        h->tt64[i] = dalloc<double>(h, src[i]->size());
        upload(h, h->tt64[i], *src[i]);
        if (mixed) {
          h->tt32[i] = dalloc<float>(h, src[i]->size());
          upload(h, h->tt32[i], *src[i]);
        }
      }
      if (q > kQfix) {
        std::vector<double> nt(q * q + 3 * q);
        for (int e = 0; e < q * q; ++e) nt[e] = h->tm.K[e];
        for (int k = 0; k < q; ++k) {
          nt[q * q + k] = h->tm.Mh[k];
          nt[q * q + q + k] = h->tm.st[k];
          nt[q * q + 2 * q + k] = h->tm.en[k];
        }
        h->node_time64 = dalloc<double>(h, nt.size());
        upload(h, h->node_time64, nt);
      }
    }
    dst_set_smem_limits<double>(h);
    if (mixed) {
      dst_set_smem_limits<float>(h);
      Level& fl = finest(h);
      if (df_len(fl.n + 1)) {
        make_df_tables(h, fl);
        switch (fl.n + 1) {
          case 64: df_set_smem<3, 2>(h); break;
          case 128: df_set_smem<3, 3>(h); break;
          case 256: df_set_smem<4, 3>(h); break;
          default: df_set_smem<4, 4>(h); break;
        }
      }
    }
    {   // partial sums: the norm kernel, or one per block of the finest-level residual with norm
      const int64_t nres = (int64_t)blocks_for(finest(h).Nx) *
                           ((finest(h).N + stmg::kStepsPerThread - 1) / stmg::kStepsPerThread);
      h->npartial = std::max<int64_t>(kNormBlocks, nres);
      h->partial = dalloc<double>(h, h->npartial);
    }
    h->dnorm = dalloc<double>(h, 1);
    h->dmaxexp = reinterpret_cast<unsigned*>(dalloc<double>(h, 1));
    check(h, cudaMallocHost(&h->hnorm, 2 * sizeof(double)), "cudaMallocHost");
    std::memset(h->hnorm, 0, 2 * sizeof(double));
    {
      int dev = 0, sms = 0;
      check(h, cudaGetDevice(&dev), "cudaGetDevice");
      check(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
      h->num_sms = std::max(1, sms);
    }
    check(h, cudaDeviceSynchronize(), "setup sync");
    return ST_OK;
  });
  if (rc != ST_OK) {
    // keep the message readable through a temporary handle is not possible; print once
    std::fprintf(stderr, "st_setup: %s\n", h->err.c_str());
    st_destroy(h);
    return rc;
  }
  *out = h;
  return ST_OK;
}

void st_destroy(st_handle* h) {
  if (!h) return;
  for (void* p : h->allocs) cudaFree(p);
  if (h->hnorm) cudaFreeHost(h->hnorm);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  delete h;
}

const char* st_last_error(const st_handle* h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

size_t st_ndof(const st_handle* h) { return h ? (size_t)h->levels.back().ndof : 0; }

int st_num_levels(const st_handle* h) { return h ? (int)h->levels.size() : 0; }

int st_plan(const st_mesh* mesh, int p_t, int N, double T, const st_options* opt, int max_levels, int* N_L,
            int* n_L, double* mu_L, int* full, int* nlev, double* mu_star_out) {
  try {
    st_options o{};
    if (check_setup_args(mesh, p_t, N, T, opt, o)) return ST_EINVAL;
    std::vector<PlanLevel> plan = plan_levels(mesh->n, p_t, N, T, o);
    std::reverse(plan.begin(), plan.end());   // 0 = coarsest, as st_level_info
    const int nl = (int)plan.size();
    if (nlev) *nlev = nl;
    if (mu_star_out) *mu_star_out = mu_star(p_t);
    if ((N_L || n_L || mu_L || full) && max_levels < nl) return ST_EINVAL;
    for (int L = 0; L < nl; ++L) {
      if (N_L) N_L[L] = plan[L].N;
      if (n_L) n_L[L] = plan[L].n;
      if (mu_L) mu_L[L] = plan[L].mu;
      if (full) full[L] = (L == nl - 1) ? -1 : plan[L + 1].coarsen_full;
    }
    return ST_OK;
  } catch (...) {
    return ST_ENOMEM;
  }
}

int st_level_info(const st_handle* h, int L, int* N_L, int* n_L, double* mu_L, int* full) {
  if (!h || L < 0 || L >= (int)h->levels.size()) return ST_EINVAL;
  const Level& l = h->levels[L];
  if (N_L) *N_L = l.N;
  if (n_L) *n_L = l.n;
  if (mu_L) *mu_L = l.mu;
  if (full) *full = (L == (int)h->levels.size() - 1) ? -1 : h->levels[L + 1].coarsen_full;
  return ST_OK;
}

int st_residual(st_handle* h, const double* f, const double* u0_ic, const double* u, double* r) {
  return guarded(h, [&]() -> int {
    if (!f || !u || !r) fail(h, ST_EINVAL, "null pointer");
    Level& lv = finest(h);
    residual<double>(h, lv, false, f, u, u0_ic, r);   // on nodes, for every q
    after_launch(h);
    return ST_OK;
  });
}

int st_vcycle(st_handle* h, double* u, const double* f, const double* u0_ic) {
  return guarded(h, [&]() -> int {
    if (!f || !u) fail(h, ST_EINVAL, "null pointer");
    const int L = (int)h->levels.size() - 1;
    Level& lv = finest(h);
    const CycleInputs in = enter_cycle_basis(h, f, u0_ic, u, true);
    if (h->opt.precision == ST_MIXED) {
      cycle_residual<double>(h, lv, false, in.f, u, in.u0, h->r64);
      const double s = norm2<double>(h, h->r64, lv.ndof);
      if (!std::isfinite(s)) fail(h, ST_ENAN, "residual norm is not finite");
      if (s > 0.0) mixed_step(h, false, u, h->r64, s);
    } else {
      vcycle<double>(h, L, false, u, in.f, in.u0, false);
    }
    leave_cycle_basis(h, u);
    after_launch(h);
    return ST_OK;
  });
}

int st_solve(st_handle* h, const double* f, const double* u0_ic, double* u, int flags, int* iters, double* relres) {
  return guarded(h, [&]() -> int {
    if (!f || !u) fail(h, ST_EINVAL, "null pointer");
    int rc = solve_impl(h, false, f, u0_ic, u, flags, iters, relres);
    after_launch(h);
    return rc;
  });
}

int st_solve_host(st_handle* h, const double* f, const double* u0_ic, double* u, int flags, int* iters,
                  double* relres) {
  return guarded(h, [&]() -> int {
    if (!f || !u) fail(h, ST_EINVAL, "null pointer");
    int rc = solve_host_impl(h, f, u0_ic, u, flags, iters, relres);
    after_launch(h);
    return rc;
  });
}

int st_adjoint_solve(st_handle* h, const double* g, double* lambda, double* grad_u0, int* iters, double* relres) {
  return guarded(h, [&]() -> int {
    if (!g || !lambda) fail(h, ST_EINVAL, "null pointer");
    int rc = solve_impl(h, true, g, nullptr, lambda, 0, iters, relres);
    if (grad_u0) {
      using T = double;
      if (h->q > kQfix) STMG_DISPATCH_D(launch_ic_grad_dyn_t, h, finest(h), lambda, grad_u0);
      else STMG_DISPATCH(launch_ic_grad_t, h, finest(h), lambda, grad_u0);
    }
    after_launch(h);
    return rc;
  });
}

int st_level_residual(st_handle* h, int L, int adjoint, const double* f, const double* u, double* r) {
  return guarded(h, [&]() -> int {
    if (!f || !u || !r) fail(h, ST_EINVAL, "null pointer");
    Level& lv = h->levels[level_index(h, L)];
    const int64_t slabs = (int64_t)lv.N * h->q;
    copy<double>(h, lv.v64.f, f, lv.ndof);
    to_modal<double>(h, lv, lv.v64.f, slabs);
    copy<double>(h, lv.v64.r, u, lv.ndof);
    to_modal<double>(h, lv, lv.v64.r, slabs);
    mresidual<double>(h, lv, adjoint != 0, lv.v64.f, lv.v64.r, (const double*)nullptr, r);
    from_modal<double>(h, lv, r, slabs);
    after_launch(h);
    return ST_OK;
  });
}

int st_level_block_solve(st_handle* h, int L, int adjoint, const double* r, double* d) {
  return guarded(h, [&]() -> int {
    if (!r || !d) fail(h, ST_EINVAL, "null pointer");
    Level& lv = h->levels[level_index(h, L)];
    smoother_block_solve<double>(h, lv, adjoint != 0, r, d);
    after_launch(h);
    return ST_OK;
  });
}

int st_level_smooth(st_handle* h, int L, int adjoint, int nu, const double* f, double* u) {
  return guarded(h, [&]() -> int {
    if (!f || !u || nu < 0) fail(h, ST_EINVAL, "bad argument");
    Level& lv = h->levels[level_index(h, L)];
    const int64_t slabs = (int64_t)lv.N * h->q;
    copy<double>(h, lv.v64.f, f, lv.ndof);
    to_modal<double>(h, lv, lv.v64.f, slabs);
    to_modal<double>(h, lv, u, slabs);
    if (!inexact(h)) {
      smooth_modal<double>(h, lv, adjoint != 0, u, lv.v64.f, (const double*)nullptr, lv.v64.r, nu, false);
    } else {
      for (int i = 0; i < nu; ++i)
        smooth_step_inexact<double>(h, lv, adjoint != 0, u, lv.v64.f, (const double*)nullptr, lv.v64.r);
    }
    from_modal<double>(h, lv, u, slabs);
    after_launch(h);
    return ST_OK;
  });
}

int st_level_restrict(st_handle* h, int L, const double* r_fine, double* f_coarse) {
  return guarded(h, [&]() -> int {
    if (!r_fine || !f_coarse || level_index(h, L) < 1) fail(h, ST_EINVAL, "bad argument");
    Level& fine = h->levels[L];
    Level& coarse = h->levels[L - 1];
    copy<double>(h, fine.v64.r, r_fine, fine.ndof);
    to_modal<double>(h, fine, fine.v64.r, (int64_t)fine.N * h->q);
    restrict_to<double>(h, L, fine.v64.r, f_coarse);
    from_modal<double>(h, coarse, f_coarse, (int64_t)coarse.N * h->q);
    after_launch(h);
    return ST_OK;
  });
}

int st_level_prolong(st_handle* h, int L, const double* e_coarse, double* u_fine) {
  return guarded(h, [&]() -> int {
    if (!e_coarse || !u_fine || level_index(h, L) < 1) fail(h, ST_EINVAL, "bad argument");
    Level& fine = h->levels[L];
    Level& coarse = h->levels[L - 1];
    copy<double>(h, coarse.v64.r, e_coarse, coarse.ndof);
    to_modal<double>(h, coarse, coarse.v64.r, (int64_t)coarse.N * h->q);
    to_modal<double>(h, fine, u_fine, (int64_t)fine.N * h->q);
    prolong_add<double>(h, L, coarse.v64.r, u_fine);
    from_modal<double>(h, fine, u_fine, (int64_t)fine.N * h->q);
    after_launch(h);
    return ST_OK;
  });
}

int st_coarsest_solve(st_handle* h, int adjoint, const double* f, double* u) {
  return guarded(h, [&]() -> int {
    if (!f || !u) fail(h, ST_EINVAL, "null pointer");
    Level& c = h->levels[0];
    const int64_t slabs = (int64_t)c.N * h->q;
    copy<double>(h, c.v64.f, f, c.ndof);
    to_modal<double>(h, c, c.v64.f, slabs);
    coarsest_modal<double>(h, adjoint != 0, u, c.v64.f, (const double*)nullptr);
    from_modal<double>(h, c, u, slabs);
    after_launch(h);
    return ST_OK;
  });
}

int st_profile_start(st_handle* h, int max_launches) {
  return guarded(h, [&]() -> int {
    if (max_launches < 1) fail(h, ST_EINVAL, "max_launches must be positive");
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
    h->ev_class.clear();
    h->ev_level.clear();
    h->lv_stats.assign((size_t)ST_K_COUNT * h->levels.size() * 4, 0.0);
    h->ev.resize(2 * (size_t)max_launches);
    for (auto& e : h->ev) check(h, cudaEventCreate(&e), "cudaEventCreate");
    for (int c = 0; c < ST_K_COUNT; ++c) {
      h->prof_launches[c] = 0;
      h->prof_bytes[c] = 0.0;
      h->prof_flops[c] = 0.0;
    }
    h->prof_dropped = 0;
    h->prof = true;
    return ST_OK;
  });
}

int st_profile_stop(st_handle* h, int* launches, double* ms, double* bytes, double* flops, int* dropped) {
  return guarded(h, [&]() -> int {
    if (!h->prof) fail(h, ST_EINVAL, "kernel timing was not started");
    h->prof = false;
    check(h, cudaStreamSynchronize(h->stream), "profile sync");
    double tot[ST_K_COUNT] = {0};
    for (size_t i = 0; i < h->ev_class.size(); ++i) {
      float t = 0.f;
      check(h, cudaEventElapsedTime(&t, h->ev[2 * i], h->ev[2 * i + 1]), "cudaEventElapsedTime");
      tot[h->ev_class[i]] += t;
      if (h->ev_level[i] >= 0)
        h->lv_stats[((size_t)h->ev_class[i] * h->levels.size() + h->ev_level[i]) * 4 + 1] += t;
    }
    for (int c = 0; c < ST_K_COUNT; ++c) {
      if (launches) launches[c] = h->prof_launches[c];
      if (ms) ms[c] = tot[c];
      if (bytes) bytes[c] = h->prof_bytes[c];
      if (flops) flops[c] = h->prof_flops[c];
    }
    if (dropped) *dropped = h->prof_dropped;
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
    h->ev_class.clear();
    h->ev_level.clear();
    return ST_OK;
  });
}

int st_profile_level(const st_handle* h, int cls, int L, int* launches, double* ms, double* bytes, double* flops) {
  if (!h || cls < 0 || cls >= ST_K_COUNT || L < 0 || L >= (int)h->levels.size() || h->lv_stats.empty())
    return ST_EINVAL;
  const size_t b = ((size_t)cls * h->levels.size() + L) * 4;
  if (launches) *launches = (int)h->lv_stats[b + 0];
  if (ms) *ms = h->lv_stats[b + 1];
  if (bytes) *bytes = h->lv_stats[b + 2];
  if (flops) *flops = h->lv_stats[b + 3];
  return ST_OK;
}

int st_transform(st_handle* h, int L, int inverse, const double* x, double* y, size_t slabs) {
  return guarded(h, [&]() -> int {
    if (!x || !y) fail(h, ST_EINVAL, "null pointer");
    Level& lv = h->levels[level_index(h, L)];
    if (slabs == 0) return ST_OK;
    const double sc = inverse ? 2.0 / (lv.n + 1) : 1.0;
    const int Nf = lv.n + 1;
    if (x == y || use_tc(h, lv) || (Nf >= 64 && Nf <= 512)) {
      dst_axes<double>(h, lv, x, y, y, (int64_t)slabs, sc);
    } else {   // the shared-memory FFT kernels work in place
      copy<double>(h, y, x, (int64_t)slabs * lv.Nx);
      dst_axes<double>(h, lv, y, (int64_t)slabs, sc);
    }
    after_launch(h);
    if (h->tcErr)
      check(h, cudaMemcpyAsync(h->hnorm + 1, h->tcErr, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "flag copy");
    check(h, cudaStreamSynchronize(h->stream), "transform sync");
    tc_check_flag(h);
    return ST_OK;
  });
}

int st_norm2(st_handle* h, const double* x, size_t n, double* out) {
  return guarded(h, [&]() -> int {
    if (!x || !out) fail(h, ST_EINVAL, "null pointer");
    *out = norm2<double>(h, x, (int64_t)n);
    return ST_OK;
  });
}

}  // extern "C"
