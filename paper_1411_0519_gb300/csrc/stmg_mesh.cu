// Space-time multigrid on uniformly refined simplicial meshes (include/stmg_mesh.h):
// host side -- refinement, P1 assembly in closed form, the hierarchy of
// Sections 2 and 4, the V-cycle with the inexact block inverse (one spatial
// V-cycle per time step), and the C ABI.  Kernels: stmg_mesh_kernels.cuh.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "stmg.h"
#include "stmg_host_time.h"
#include "stmg_kernels.cuh"
#include "stmg_mesh.h"
#include "stmg_mesh_kernels.cuh"

namespace {

using namespace stmg_host;

constexpr int kThreads = 256;
constexpr int kNormBlocks = 1024;
constexpr int kMaxQ = 4;
constexpr int kMaxDense = 1024;   // q * (interior vertices of the initial mesh)

// ------------------------------------------------------------------ host meshes
struct HMesh {
  int d = 0;
  std::vector<double> v;   // nv x d
  std::vector<int> c;      // nc x (d + 1)
  int nv() const { return (int)(v.size() / d); }
  int nc() const { return (int)(c.size() / (d + 1)); }
};

// One uniform refinement: every edge split at its midpoint; triangles into 4,
// tetrahedra into 8 (corner tetrahedra, inner octahedron cut along the diagonal
// between the midpoints of edges 02 and 13).  mid[k] = the edge whose midpoint
// is vertex nv + k of the result.
HMesh refine(const HMesh& m, std::vector<std::pair<int, int>>& mid) {
  HMesh r;
  r.d = m.d;
  r.v = m.v;
  mid.clear();
  std::unordered_map<uint64_t, int> at;
  auto midpoint = [&](int a, int b) {
    const int lo = std::min(a, b), hi = std::max(a, b);
    const uint64_t key = ((uint64_t)(uint32_t)lo << 32) | (uint32_t)hi;
    auto it = at.find(key);
    if (it != at.end()) return it->second;
    const int idx = (int)(r.v.size() / m.d);
    for (int a2 = 0; a2 < m.d; ++a2) r.v.push_back(0.5 * (m.v[(size_t)lo * m.d + a2] + m.v[(size_t)hi * m.d + a2]));
    at.emplace(key, idx);
    mid.emplace_back(lo, hi);
    return idx;
  };
  const int k = m.d + 1;
  for (int e = 0; e < m.nc(); ++e) {
    const int* c = &m.c[(size_t)e * k];
    if (m.d == 2) {
      const int v0 = c[0], v1 = c[1], v2 = c[2];
      const int m01 = midpoint(v0, v1), m12 = midpoint(v1, v2), m02 = midpoint(v0, v2);
      const int kids[4][3] = {{v0, m01, m02}, {v1, m12, m01}, {v2, m02, m12}, {m01, m12, m02}};
      for (auto& t : kids) r.c.insert(r.c.end(), t, t + 3);
    } else {
      const int x0 = c[0], x1 = c[1], x2 = c[2], x3 = c[3];
      const int x01 = midpoint(x0, x1), x02 = midpoint(x0, x2), x03 = midpoint(x0, x3);
      const int x12 = midpoint(x1, x2), x13 = midpoint(x1, x3), x23 = midpoint(x2, x3);
      const int kids[8][4] = {{x0, x01, x02, x03},   {x01, x1, x12, x13},  {x02, x12, x2, x23},
                              {x03, x13, x23, x3},   {x01, x02, x03, x13}, {x01, x02, x12, x13},
                              {x02, x03, x13, x23},  {x02, x12, x13, x23}};
      for (auto& t : kids) r.c.insert(r.c.end(), t, t + 4);
    }
  }
  return r;
}

double longest_edge(const HMesh& m) {
  double h2 = 0.0;
  const int k = m.d + 1;
  for (int e = 0; e < m.nc(); ++e)
    for (int a = 0; a < k; ++a)
      for (int b = a + 1; b < k; ++b) {
        double s = 0.0;
        for (int x = 0; x < m.d; ++x) {
          const double t = m.v[(size_t)m.c[(size_t)e * k + a] * m.d + x] - m.v[(size_t)m.c[(size_t)e * k + b] * m.d + x];
          s += t * t;
        }
        h2 = std::max(h2, s);
      }
  return std::sqrt(h2);
}

// Interior vertices (every coordinate strictly inside (0, 1)) ordered by z, y, x.
std::vector<int> interior_order(const HMesh& m, std::vector<int>& pos) {
  std::vector<int> idx;
  for (int i = 0; i < m.nv(); ++i) {
    bool in = true;
    for (int a = 0; a < m.d; ++a) {
      const double x = m.v[(size_t)i * m.d + a];
      if (!(x > 0.0 && x < 1.0)) in = false;
    }
    if (in) idx.push_back(i);
  }
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    for (int x = m.d - 1; x >= 0; --x) {
      const double pa = m.v[(size_t)a * m.d + x], pb = m.v[(size_t)b * m.d + x];
      if (pa != pb) return pa < pb;
    }
    return a < b;
  });
  pos.assign(m.nv(), -1);
  for (int i = 0; i < (int)idx.size(); ++i) pos[idx[i]] = i;
  return idx;
}

// Small dense inverse by Gauss-Jordan elimination with partial pivoting.
bool invert(std::vector<double>& a, int n) {
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + col]) > std::fabs(a[(size_t)piv * n + col])) piv = r;
    if (a[(size_t)piv * n + col] == 0.0) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)piv * n + k], a[(size_t)col * n + k]);
        std::swap(inv[(size_t)piv * n + k], inv[(size_t)col * n + k]);
      }
    const double p = 1.0 / a[(size_t)col * n + col];
    for (int k = 0; k < n; ++k) {
      a[(size_t)col * n + k] *= p;
      inv[(size_t)col * n + k] *= p;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = a[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)col * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)col * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

// ------------------------------------------------------------------ handle
struct SpaceLevel {          // one mesh of the refinement (device arrays + host copies)
  int Nx = 0, nnz = 0;
  double h = 0.0;
  std::vector<double> coords;       // Nx x d (host)
  std::vector<double> dM, dK;       // diagonals of M_h, K_h (host)
  std::vector<int> rp_h, ci_h;      // CSR (host, for the dense solve of the initial mesh)
  std::vector<double> mv_h, kv_h;
  int *rp = nullptr, *ci = nullptr;
  double *mv = nullptr, *kv = nullptr;
  int *p0 = nullptr, *p1 = nullptr;                   // parents on the next coarser mesh (level >= 1)
  int *ch_rp = nullptr, *ch_ci = nullptr;             // children on the next finer mesh (level < top)
  double* ch_w = nullptr;
};

struct MLevel {              // one space-time level
  int N = 0, l = 0, full = -1;
  double tau = 0.0, mu = 0.0;
  int64_t ndof = 0;
  double *u = nullptr, *f = nullptr, *r = nullptr;    // u, f: coarse levels only
  std::vector<double*> dinv;    // per mesh level k = 1..l: Nx_k q x q inverses of the node blocks (index k)
  double* a0inv = nullptr;      // dense inverse of A_tau on the initial mesh
  std::vector<double*> sb, sx, sy;   // spatial V-cycle buffers per mesh level k = 0..l
};

}  // namespace

struct stm_handle {
  int d = 0, p_t = 0, q = 0, N = 0;
  double T = 0.0;
  st_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<SpaceLevel> sp;    // 0 = initial mesh
  std::vector<MLevel> lv;        // 0 = coarsest
  HostTime tm{};
  std::vector<void*> allocs;
  size_t bytes = 0;
  double* partial = nullptr;
  double* dnorm = nullptr;
  double* hnorm = nullptr;
  double* feff = nullptr;        // f + IC of the finest level
  std::string err;
};

namespace {

struct Fail {
  int code;
};

void fail(stm_handle* h, int code, const std::string& msg) {
  h->err = msg;
  throw Fail{code};
}

void check(stm_handle* h, cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(h, ST_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

template <typename T>
T* dalloc(stm_handle* h, size_t count) {
  const size_t b = std::max<size_t>(count, 1) * sizeof(T);
  if (h->opt.max_workspace_bytes && h->bytes + b > h->opt.max_workspace_bytes)
    fail(h, ST_ENOMEM, "workspace limit exceeded");
  void* p = nullptr;
  if (cudaMalloc(&p, b) != cudaSuccess) {
    cudaGetLastError();
    fail(h, ST_ENOMEM, "cudaMalloc failed");
  }
  h->allocs.push_back(p);
  h->bytes += b;
  return static_cast<T*>(p);
}

template <typename T>
T* upload(stm_handle* h, const std::vector<T>& src) {
  T* d = dalloc<T>(h, src.size());
  if (!src.empty()) check(h, cudaMemcpy(d, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
  return d;
}

template <int Q>
stmm::MTime<Q> mtime(const HostTime& t) {
  stmm::MTime<Q> c{};
  for (int i = 0; i < Q * Q; ++i) {
    c.K[i] = t.K[i];
    c.R1[i] = t.R1[i];
    c.R2[i] = t.R2[i];
  }
  for (int i = 0; i < Q; ++i) {
    c.Mh[i] = t.Mh[i];
    c.st[i] = t.st[i];
    c.en[i] = t.en[i];
  }
  return c;
}

stmm::Csr csr(const SpaceLevel& s) { return stmm::Csr{s.rp, s.ci, s.mv, s.kv}; }
stmm::Parents parents(const SpaceLevel& s) { return stmm::Parents{s.p0, s.p1}; }
stmm::Children children(const SpaceLevel& s) { return stmm::Children{s.ch_rp, s.ch_ci, s.ch_w}; }

unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// grid over (vertices, steps) with the steps on the y axis in chunks of 65535
template <typename F>
void over_steps(int nodes, int steps, F&& launch) {
  for (int s0 = 0; s0 < steps; s0 += 65535) {
    dim3 grid(blocks_for(nodes), (unsigned)std::min(65535, steps - s0));
    launch(grid, s0);
  }
}

#define STM_Q(FN, ...)                                                 \
  do {                                                                 \
    switch (h->q) {                                                    \
      case 1: FN<1>(__VA_ARGS__); break;                               \
      case 2: FN<2>(__VA_ARGS__); break;                               \
      case 3: FN<3>(__VA_ARGS__); break;                               \
      case 4: FN<4>(__VA_ARGS__); break;                               \
      default: fail(h, ST_EINVAL, "p_t > 3");                          \
    }                                                                  \
  } while (0)

// ------------------------------------------------------------------ launches
template <int Q>
void l_residual(stm_handle* h, const MLevel& L, bool adj, const double* f, const double* u, double* r) {
  const SpaceLevel& s = h->sp[L.l];
  const auto tc = mtime<Q>(h->tm);
  over_steps(s.Nx, L.N, [&](dim3 g, int s0) {
    if (adj) stmm::k_mresidual<Q, true><<<g, kThreads, 0, h->stream>>>(f, u, r, csr(s), s.Nx, L.N, s0, L.tau, tc);
    else stmm::k_mresidual<Q, false><<<g, kThreads, 0, h->stream>>>(f, u, r, csr(s), s.Nx, L.N, s0, L.tau, tc);
  });
}

template <int Q>
void l_jacobi(stm_handle* h, const MLevel& L, int k, bool adj, bool zero, const double* b, const double* x,
              double* y) {
  const SpaceLevel& s = h->sp[k];
  const auto tc = mtime<Q>(h->tm);
  const double w = h->opt.omega_x;
  const double* D = L.dinv[k];
  over_steps(s.Nx, L.N, [&](dim3 g, int s0) {
#define STM_JAC(A, Z) \
  stmm::k_mjacobi<Q, A, Z><<<g, kThreads, 0, h->stream>>>(b, x, y, csr(s), s.Nx, L.N, s0, L.tau, w, D, tc)
    if (adj) { if (zero) STM_JAC(true, true); else STM_JAC(true, false); }
    else { if (zero) STM_JAC(false, true); else STM_JAC(false, false); }
#undef STM_JAC
  });
}

template <int Q>
void l_residual_jacobi0(stm_handle* h, const MLevel& L, bool adj, const double* f, const double* u, double* r,
                        double* x) {
  const SpaceLevel& s = h->sp[L.l];
  const auto tc = mtime<Q>(h->tm);
  const double* D = L.dinv[L.l];
  over_steps(s.Nx, L.N, [&](dim3 g, int s0) {
    if (adj)
      stmm::k_mresidual_jacobi0<Q, true><<<g, kThreads, 0, h->stream>>>(f, u, r, x, csr(s), s.Nx, L.N, s0, L.tau,
                                                                          h->opt.omega_x, D, tc);
    else
      stmm::k_mresidual_jacobi0<Q, false><<<g, kThreads, 0, h->stream>>>(f, u, r, x, csr(s), s.Nx, L.N, s0, L.tau,
                                                                           h->opt.omega_x, D, tc);
  });
}

template <int Q>
void l_jacobi_update(stm_handle* h, const MLevel& L, bool adj, const double* b, const double* x, double* u) {
  const SpaceLevel& s = h->sp[L.l];
  const auto tc = mtime<Q>(h->tm);
  const double* D = L.dinv[L.l];
  over_steps(s.Nx, L.N, [&](dim3 g, int s0) {
    if (adj)
      stmm::k_mjacobi_update<Q, true><<<g, kThreads, 0, h->stream>>>(b, x, u, csr(s), s.Nx, L.N, s0, L.tau,
                                                                       h->opt.omega_x, h->opt.omega, D, tc);
    else
      stmm::k_mjacobi_update<Q, false><<<g, kThreads, 0, h->stream>>>(b, x, u, csr(s), s.Nx, L.N, s0, L.tau,
                                                                        h->opt.omega_x, h->opt.omega, D, tc);
  });
}

template <int Q>
void l_space_residual(stm_handle* h, const MLevel& L, int k, bool adj, const double* b, const double* x, double* r) {
  const SpaceLevel& s = h->sp[k];
  const auto tc = mtime<Q>(h->tm);
  over_steps(s.Nx, L.N, [&](dim3 g, int s0) {
    if (adj) stmm::k_mspace_residual<Q, true><<<g, kThreads, 0, h->stream>>>(b, x, r, csr(s), s.Nx, L.N, s0, L.tau, tc);
    else stmm::k_mspace_residual<Q, false><<<g, kThreads, 0, h->stream>>>(b, x, r, csr(s), s.Nx, L.N, s0, L.tau, tc);
  });
}

template <int Q>
void l_restrict_space(stm_handle* h, const MLevel& L, int k, const double* r, double* bc) {
  const SpaceLevel& c = h->sp[k - 1];
  const SpaceLevel& f = h->sp[k];
  over_steps(c.Nx, L.N, [&](dim3 g, int s0) {
    stmm::k_mrestrict_space<Q><<<g, kThreads, 0, h->stream>>>(r, bc, children(c), c.Nx, f.Nx, L.N, s0);
  });
}

template <int Q>
void l_prolong_space_add(stm_handle* h, const MLevel& L, int k, const double* xc, double* x) {
  const SpaceLevel& c = h->sp[k - 1];
  const SpaceLevel& f = h->sp[k];
  over_steps(f.Nx, L.N, [&](dim3 g, int s0) {
    stmm::k_mprolong_space_add<Q><<<g, kThreads, 0, h->stream>>>(xc, x, parents(f), c.Nx, f.Nx, L.N, s0);
  });
}

void l_dense(stm_handle* h, const MLevel& L, bool adj, const double* b, double* y) {
  const int n = h->q * h->sp[0].Nx;
  over_steps(n, L.N, [&](dim3 g, int s0) {
    stmm::k_mdense_apply<<<g, kThreads, 0, h->stream>>>(b, y, L.a0inv, n, L.N, s0, adj);
  });
}

template <int Q>
void l_restrict(stm_handle* h, int Li, const double* r, double* fc) {
  const MLevel& F = h->lv[Li];
  const MLevel& C = h->lv[Li - 1];
  const SpaceLevel& cs = h->sp[C.l];
  const SpaceLevel& fs = h->sp[F.l];
  const auto tc = mtime<Q>(h->tm);
  over_steps(cs.Nx, C.N, [&](dim3 g, int m0) {
    if (F.l != C.l)
      stmm::k_mrestrict<Q, true><<<g, kThreads, 0, h->stream>>>(r, fc, children(cs), cs.Nx, fs.Nx, C.N, m0, tc);
    else
      stmm::k_mrestrict<Q, false><<<g, kThreads, 0, h->stream>>>(r, fc, children(cs), cs.Nx, fs.Nx, C.N, m0, tc);
  });
}

template <int Q>
void l_prolong(stm_handle* h, int Li, const double* ec, double* u) {
  const MLevel& F = h->lv[Li];
  const MLevel& C = h->lv[Li - 1];
  const SpaceLevel& cs = h->sp[C.l];
  const SpaceLevel& fs = h->sp[F.l];
  const auto tc = mtime<Q>(h->tm);
  over_steps(fs.Nx, C.N, [&](dim3 g, int m0) {
    if (F.l != C.l)
      stmm::k_mprolong<Q, true><<<g, kThreads, 0, h->stream>>>(ec, u, parents(fs), cs.Nx, fs.Nx, C.N, m0, tc);
    else
      stmm::k_mprolong<Q, false><<<g, kThreads, 0, h->stream>>>(ec, u, parents(fs), cs.Nx, fs.Nx, C.N, m0, tc);
  });
}

template <int Q>
void l_add_ic(stm_handle* h, const double* f, const double* u0, double* g) {
  const SpaceLevel& s = h->sp.back();
  const auto tc = mtime<Q>(h->tm);
  stmm::k_madd_ic<Q><<<blocks_for(s.Nx), kThreads, 0, h->stream>>>(f, u0, g, csr(s), s.Nx, tc);
}

template <int Q>
void l_ic_gradient(stm_handle* h, const double* lam, double* g) {
  const SpaceLevel& s = h->sp.back();
  const auto tc = mtime<Q>(h->tm);
  stmm::k_mic_gradient<Q><<<blocks_for(s.Nx), kThreads, 0, h->stream>>>(lam, g, csr(s), s.Nx, tc);
}

void copy(stm_handle* h, double* y, const double* x, int64_t n) {
  check(h, cudaMemcpyAsync(y, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream), "copy");
}
void zero(stm_handle* h, double* y, int64_t n) {
  check(h, cudaMemsetAsync(y, 0, sizeof(double) * n, h->stream), "memset");
}
void axpy(stm_handle* h, double* y, const double* x, double a, int64_t n) {
  stmg::k_axpy<double><<<(unsigned)std::min<int64_t>(blocks_for(n), 152 * 16), kThreads, 0, h->stream>>>(y, x, a, n);
}

double norm2(stm_handle* h, const double* x, int64_t n) {
  stmg::k_sumsq_partial<double><<<kNormBlocks, kThreads, 0, h->stream>>>(x, n, h->partial);
  stmg::k_sum_final<<<1, 1024, 0, h->stream>>>(h->partial, kNormBlocks, h->dnorm);
  check(h, cudaMemcpyAsync(h->hnorm, h->dnorm, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "norm copy");
  check(h, cudaStreamSynchronize(h->stream), "norm sync");
  return std::sqrt(*h->hnorm);
}

// ------------------------------------------------------------------ the cycle
// One spatial V-cycle on mesh levels k, k-1, ..., 0 for every time step of
// space-time level L (the inexact block inverse, Remark on the V-cycle
// approximation in space): x = D~^{-1} b from a zero guess.  Returns the buffer
// that holds the result (one of L.sx[k], L.sy[k]); b is not modified.
// x0_done: L.sx[k] already holds the first sweep omega_x D^{-1} b (fused into the
// residual pass).  update: instead of returning the result, the last sweep adds
// omega_t times it into `update` (the damped step of the smoother) and nullptr is
// returned.
const double* space_vcycle(stm_handle* h, MLevel& L, int k, bool adj, const double* b, bool x0_done = false,
                           double* update = nullptr) {
  if (k == 0) {
    if (update) {
      l_dense(h, L, adj, b, L.sx[0]);
      axpy(h, update, L.sx[0], h->opt.omega, L.ndof);
      return nullptr;
    }
    l_dense(h, L, adj, b, L.sx[0]);
    return L.sx[0];
  }
  double* x = L.sx[k];
  double* y = L.sy[k];
  const int nu = std::max(1, h->opt.nu_x);
  if (!x0_done) STM_Q(l_jacobi, h, L, k, adj, true, b, (const double*)nullptr, x);
  for (int i = 1; i < nu; ++i) {
    STM_Q(l_jacobi, h, L, k, adj, false, b, x, y);
    std::swap(x, y);
  }
  STM_Q(l_space_residual, h, L, k, adj, b, x, y);        // y = b - A x
  STM_Q(l_restrict_space, h, L, k, y, L.sb[k - 1]);
  const double* xc = space_vcycle(h, L, k - 1, adj, L.sb[k - 1]);
  STM_Q(l_prolong_space_add, h, L, k, xc, x);
  for (int i = 0; i < nu; ++i) {
    if (update != nullptr && i == nu - 1) {
      STM_Q(l_jacobi_update, h, L, adj, b, x, update);
      return nullptr;
    }
    STM_Q(l_jacobi, h, L, k, adj, false, b, x, y);
    std::swap(x, y);
  }
  return x;
}

// u <- u + omega D~^{-1} (f - L u), nu times (eq. chap4_smoother).  On a level
// whose mesh is refined, the residual pass also takes the first Jacobi sweep of
// the spatial V-cycle and the last sweep adds into u directly.
void smooth(stm_handle* h, int Li, bool adj, double* u, const double* f, int nu) {
  MLevel& L = h->lv[Li];
  for (int i = 0; i < nu; ++i) {
    if (L.l >= 1) {
      STM_Q(l_residual_jacobi0, h, L, adj, f, u, L.r, L.sx[L.l]);
      space_vcycle(h, L, L.l, adj, L.r, true, u);
    } else {
      STM_Q(l_residual, h, L, adj, f, u, L.r);
      const double* d = space_vcycle(h, L, L.l, adj, L.r);
      axpy(h, u, d, h->opt.omega, L.ndof);
    }
  }
}

// Exact solve on the coarsest level (one time step): A u = f by spatial
// V-cycles repeated until the residual stops decreasing below 1e-13 ||f||
// (one V-cycle is exact on the initial mesh).
void coarsest(stm_handle* h, bool adj, double* u, const double* f) {
  MLevel& L = h->lv[0];
  if (L.l == 0) {
    l_dense(h, L, adj, f, u);
    return;
  }
  zero(h, u, L.ndof);
  copy(h, L.r, f, L.ndof);
  const double f0 = norm2(h, f, L.ndof);
  if (f0 == 0.0) return;
  double prev = f0;
  for (int it = 0; it < 100; ++it) {
    const double* d = space_vcycle(h, L, L.l, adj, L.r);
    axpy(h, u, d, 1.0, L.ndof);
    STM_Q(l_space_residual, h, L, L.l, adj, f, u, L.r);
    const double rn = norm2(h, L.r, L.ndof);
    if (!std::isfinite(rn)) fail(h, ST_ENAN, "coarsest solve: residual not finite");
    if (rn <= 1e-15 * f0 || (rn <= 1e-13 * f0 && rn > 0.5 * prev)) break;
    prev = rn;
  }
}

void vcycle(stm_handle* h, int Li, bool adj, double* u, const double* f, bool u_zero) {
  if (Li == 0) {
    coarsest(h, adj, u, f);
    return;
  }
  MLevel& L = h->lv[Li];
  if (u_zero) zero(h, u, L.ndof);
  smooth(h, Li, adj, u, f, h->opt.nu1);
  STM_Q(l_residual, h, L, adj, f, u, L.r);
  MLevel& C = h->lv[Li - 1];
  STM_Q(l_restrict, h, Li, L.r, C.f);
  const int reps = (Li - 1 == 0) ? 1 : std::max(1, h->opt.gamma);
  for (int g = 0; g < reps; ++g) vcycle(h, Li - 1, adj, C.u, C.f, g == 0);
  STM_Q(l_prolong, h, Li, C.u, u);
  smooth(h, Li, adj, u, f, h->opt.nu2);
}

MLevel& finest(stm_handle* h) { return h->lv.back(); }

// f + IC on the finest level into the handle's copy (u0 may be null).
const double* with_ic(stm_handle* h, const double* f, const double* u0) {
  if (u0 == nullptr) return f;
  MLevel& F = finest(h);
  copy(h, h->feff, f, F.ndof);
  STM_Q(l_add_ic, h, f, u0, h->feff);
  return h->feff;
}

int solve_impl(stm_handle* h, bool adj, const double* f, double* u, bool given, int* iters, double* relres) {
  MLevel& F = finest(h);
  const int top = (int)h->lv.size() - 1;
  if (!given) zero(h, u, F.ndof);
  STM_Q(l_residual, h, F, adj, f, u, F.r);
  const double r0 = norm2(h, F.r, F.ndof);
  double rn = r0;
  int it = 0, status = ST_OK;
  if (!std::isfinite(r0)) status = ST_ENAN;
  while (status == ST_OK && r0 > 0.0 && rn > h->opt.rtol * r0) {
    if (it >= h->opt.maxit) { status = ST_ENOTCONV; h->err = "maxit reached"; break; }
    vcycle(h, top, adj, u, f, false);
    ++it;
    STM_Q(l_residual, h, F, adj, f, u, F.r);
    rn = norm2(h, F.r, F.ndof);
    if (!std::isfinite(rn)) { status = ST_ENAN; h->err = "residual norm is not finite"; break; }
    if (rn > 1e6 * r0) { status = ST_ENOTCONV; h->err = "residual grew by 1e6"; break; }
  }
  if (iters) *iters = it;
  if (relres) *relres = r0 > 0.0 ? rn / r0 : 0.0;
  return status;
}

template <typename Fn>
int guarded(stm_handle* h, Fn&& fn) {
  if (!h) return ST_EINVAL;
  try {
    h->err.clear();
    const int rc = fn();
    const cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->err = std::string("kernel launch: ") + cudaGetErrorString(e);
      return ST_ECUDA;
    }
    return rc;
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

int level_index(stm_handle* h, int L) {
  if (L < 0 || L >= (int)h->lv.size()) fail(h, ST_EINVAL, "level out of range");
  return L;
}

// ------------------------------------------------------------------ setup
const char* check_args(const st_simplex_mesh* m, int refinements, int p_t, int N, double T, const st_options& o) {
  if (!m || (m->dim != 2 && m->dim != 3)) return "dim must be 2 or 3";
  if (m->nverts < m->dim + 1 || m->ncells < 1 || !m->verts || !m->cells) return "empty mesh";
  for (int i = 0; i < m->ncells * (m->dim + 1); ++i)
    if (m->cells[i] < 0 || m->cells[i] >= m->nverts) return "cell vertex index out of range";
  for (int i = 0; i < m->nverts * m->dim; ++i)
    if (!(m->verts[i] >= 0.0 && m->verts[i] <= 1.0)) return "vertex outside the unit cube";
  if (refinements < 0 || refinements > 12) return "refinements must be 0 ... 12";
  if (p_t < 0 || p_t + 1 > kMaxQ) return "p_t must be 0 ... 3";
  if (N < 1 || N > 32768 || (N & (N - 1))) return "N must be a power of 2 up to 32768";
  if (!(T > 0.0)) return "T must be positive";
  if (o.precision != ST_FP64) return "precision must be ST_FP64";
  if (o.smoother != ST_SMOOTH_VCYCLE) return "smoother must be ST_SMOOTH_VCYCLE";
  if (o.coarsest_steps != 1) return "coarsest_steps must be 1";
  if (o.nu1 < 0 || o.nu2 < 0 || o.nu_x < 1 || o.maxit < 0 || !(o.rtol >= 0.0) || o.gamma < 1 || o.gamma > 2)
    return "invalid smoothing / cycle options";
  return nullptr;
}

void build(stm_handle* h, const st_simplex_mesh* m0, int refinements) {
  const int d = h->d, k = d + 1, q = h->q;
  HMesh mesh;
  mesh.d = d;
  mesh.v.assign(m0->verts, m0->verts + (size_t)m0->nverts * d);
  mesh.c.assign(m0->cells, m0->cells + (size_t)m0->ncells * k);
  std::vector<int> prev_pos;
  for (int lvl = 0; lvl <= refinements; ++lvl) {
    std::vector<std::pair<int, int>> mid;
    if (lvl > 0) mesh = refine(mesh, mid);
    SpaceLevel s;
    std::vector<int> pos;
    const std::vector<int> order = interior_order(mesh, pos);
    s.Nx = (int)order.size();
    s.h = longest_edge(mesh);
    if (s.Nx == 0) fail(h, ST_EINVAL, "a mesh level has no interior vertex");
    s.coords.resize((size_t)s.Nx * d);
    for (int i = 0; i < s.Nx; ++i)
      for (int a = 0; a < d; ++a) s.coords[(size_t)i * d + a] = mesh.v[(size_t)order[i] * d + a];
    // P1 element matrices in closed form: mass |T| (1 + delta_ab) / ((d+1)(d+2)),
    // stiffness |T| grad l_a . grad l_b with the barycentric gradients from J^{-1}
    struct Trip { int r, c; double m, kk; };
    std::vector<Trip> trips;
    trips.reserve((size_t)mesh.nc() * k * k);
    const double fact = (d == 2) ? 2.0 : 6.0;
    for (int e = 0; e < mesh.nc(); ++e) {
      const int* c = &mesh.c[(size_t)e * k];
      double J[9], Ji[9];
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) J[a * d + b] = mesh.v[(size_t)c[b + 1] * d + a] - mesh.v[(size_t)c[0] * d + a];
      double det;
      if (d == 2) {
        det = J[0] * J[3] - J[1] * J[2];
        Ji[0] = J[3] / det; Ji[1] = -J[1] / det; Ji[2] = -J[2] / det; Ji[3] = J[0] / det;
      } else {
        det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
        Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det; Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
        Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det; Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
        Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det; Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
        Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det; Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
        Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
      }
      if (det == 0.0) fail(h, ST_EINVAL, "degenerate cell");
      const double vol = std::fabs(det) / fact;
      double g[4][3];   // grad of lambda_b (b >= 1) = row b-1 of J^{-1}; lambda_0 = 1 - sum
      for (int b = 1; b < k; ++b)
        for (int a = 0; a < d; ++a) g[b][a] = Ji[(b - 1) * d + a];
      for (int a = 0; a < d; ++a) {
        g[0][a] = 0.0;
        for (int b = 1; b < k; ++b) g[0][a] -= g[b][a];
      }
      for (int a = 0; a < k; ++a) {
        const int ia = pos[c[a]];
        if (ia < 0) continue;
        for (int b = 0; b < k; ++b) {
          const int ib = pos[c[b]];
          if (ib < 0) continue;
          double dot = 0.0;
          for (int x = 0; x < d; ++x) dot += g[a][x] * g[b][x];
          trips.push_back({ia, ib, vol * (a == b ? 2.0 : 1.0) / ((d + 1) * (d + 2)), vol * dot});
        }
      }
    }
    std::sort(trips.begin(), trips.end(), [](const Trip& x, const Trip& y) { return x.r != y.r ? x.r < y.r : x.c < y.c; });
    s.rp_h.assign(s.Nx + 1, 0);
    for (size_t i = 0; i < trips.size();) {
      size_t j = i;
      double mv = 0.0, kv = 0.0;
      while (j < trips.size() && trips[j].r == trips[i].r && trips[j].c == trips[i].c) {
        mv += trips[j].m;
        kv += trips[j].kk;
        ++j;
      }
      s.ci_h.push_back(trips[i].c);
      s.mv_h.push_back(mv);
      s.kv_h.push_back(kv);
      s.rp_h[trips[i].r + 1]++;
      i = j;
    }
    for (int i = 0; i < s.Nx; ++i) s.rp_h[i + 1] += s.rp_h[i];
    s.nnz = (int)s.ci_h.size();
    s.dM.assign(s.Nx, 0.0);
    s.dK.assign(s.Nx, 0.0);
    for (int i = 0; i < s.Nx; ++i)
      for (int e = s.rp_h[i]; e < s.rp_h[i + 1]; ++e)
        if (s.ci_h[e] == i) {
          s.dM[i] = s.mv_h[e];
          s.dK[i] = s.kv_h[e];
        }
    s.rp = upload(h, s.rp_h);
    s.ci = upload(h, s.ci_h);
    s.mv = upload(h, s.mv_h);
    s.kv = upload(h, s.kv_h);
    if (lvl > 0) {
      // parents of every interior vertex on the previous mesh
      SpaceLevel& c = h->sp.back();
      const int ncv = mesh.nv() - (int)mid.size();   // vertices carried over keep their indices
      std::vector<int> p0(s.Nx), p1(s.Nx);
      std::vector<std::vector<std::pair<int, double>>> kids(c.Nx);
      for (int i = 0; i < s.Nx; ++i) {
        const int v = order[i];
        if (v < ncv) {
          p0[i] = prev_pos[v];
          p1[i] = -2;
          if (p0[i] >= 0) kids[p0[i]].push_back({i, 1.0});
        } else {
          const auto& e = mid[v - ncv];
          p0[i] = prev_pos[e.first];
          p1[i] = prev_pos[e.second];
          if (p0[i] >= 0) kids[p0[i]].push_back({i, 0.5});
          if (p1[i] >= 0) kids[p1[i]].push_back({i, 0.5});
        }
      }
      std::vector<int> crp(c.Nx + 1, 0), cci;
      std::vector<double> cw;
      for (int j = 0; j < c.Nx; ++j) {
        std::sort(kids[j].begin(), kids[j].end());
        for (auto& kw : kids[j]) {
          cci.push_back(kw.first);
          cw.push_back(kw.second);
        }
        crp[j + 1] = (int)cci.size();
      }
      s.p0 = upload(h, p0);
      s.p1 = upload(h, p1);
      c.ch_rp = upload(h, crp);
      c.ch_ci = upload(h, cci);
      c.ch_w = upload(h, cw);
    }
    prev_pos = pos;
    h->sp.push_back(std::move(s));
  }
  if ((int64_t)q * h->sp[0].Nx > kMaxDense) fail(h, ST_EINVAL, "the initial mesh has too many interior vertices");

  // space-time levels by the rule of Section 4, finest first
  struct P { int N, l, full; double tau, mu; };
  std::vector<P> plan;
  const double ms = mu_star(h->p_t);
  int Nl = h->N, l = refinements;
  double tau = h->T / h->N;
  for (;;) {
    const double hl = h->sp[l].h;
    P p{Nl, l, -1, tau, tau / (hl * hl)};
    if (Nl <= 1) { plan.push_back(p); break; }
    bool full;
    if (h->opt.coarsening == ST_SEMI) full = false;
    else if (h->opt.coarsening == ST_FULL) full = l >= 1;
    else full = p.mu >= ms * (1.0 - 1e-12) && l >= 1;
    plan.push_back(p);
    Nl /= 2;
    tau *= 2.0;
    if (full) --l;
    plan.back().full = full ? 1 : 0;   // how this level is coarsened
  }
  // API levels: 0 = coarsest; level L stores how it was obtained from L + 1
  const int nl = (int)plan.size();
  h->lv.resize(nl);
  for (int i = 0; i < nl; ++i) {
    const P& p = plan[nl - 1 - i];
    MLevel& L = h->lv[i];
    L.N = p.N;
    L.l = p.l;
    L.tau = p.tau;
    L.mu = p.mu;
    L.full = (i == nl - 1) ? -1 : plan[nl - 2 - i].full;
    L.ndof = (int64_t)p.N * q * h->sp[p.l].Nx;
  }
  // workspace and per-level tables
  for (int i = 0; i < nl; ++i) {
    MLevel& L = h->lv[i];
    const bool top = i == nl - 1;
    if (!top) {
      L.u = dalloc<double>(h, L.ndof);
      L.f = dalloc<double>(h, L.ndof);
    }
    L.r = dalloc<double>(h, L.ndof);
    L.sb.assign(L.l + 1, nullptr);
    L.sx.assign(L.l + 1, nullptr);
    L.sy.assign(L.l + 1, nullptr);
    L.dinv.assign(L.l + 1, nullptr);
    for (int kk = 0; kk <= L.l; ++kk) {
      const int64_t n = (int64_t)L.N * q * h->sp[kk].Nx;
      L.sx[kk] = dalloc<double>(h, n);
      if (kk >= 1) L.sy[kk] = dalloc<double>(h, n);
      if (kk < L.l) L.sb[kk] = dalloc<double>(h, n);
      if (kk >= 1) {   // node blocks D_j = (M_h)_jj K_tau + (K_h)_jj M_tau, inverted
        const SpaceLevel& s = h->sp[kk];
        std::vector<double> tab((size_t)s.Nx * q * q);
        std::vector<double> D(q * q);
        for (int j = 0; j < s.Nx; ++j) {
          for (int a = 0; a < q; ++a)
            for (int b = 0; b < q; ++b)
              D[a * q + b] = s.dM[j] * h->tm.K[a * q + b] + (a == b ? s.dK[j] * L.tau * h->tm.Mh[a] : 0.0);
          if (!invert(D, q)) fail(h, ST_EINVAL, "singular node block");
          std::copy(D.begin(), D.end(), tab.begin() + (size_t)j * q * q);
        }
        L.dinv[kk] = upload(h, tab);
      }
    }
    {   // dense inverse of A_tau = K_tau (x) M_0 + M_tau (x) K_0 on the initial mesh
      const SpaceLevel& s0 = h->sp[0];
      const int n0 = s0.Nx, n = q * n0;
      std::vector<double> A((size_t)n * n, 0.0);
      for (int j = 0; j < n0; ++j)
        for (int e = s0.rp_h[j]; e < s0.rp_h[j + 1]; ++e) {
          const int c = s0.ci_h[e];
          for (int a = 0; a < q; ++a)
            for (int b = 0; b < q; ++b)
              A[(size_t)(a * n0 + j) * n + b * n0 + c] +=
                  h->tm.K[a * q + b] * s0.mv_h[e] + (a == b ? L.tau * h->tm.Mh[a] * s0.kv_h[e] : 0.0);
        }
      if (!invert(A, n)) fail(h, ST_EINVAL, "singular block on the initial mesh");
      L.a0inv = upload(h, A);
    }
  }
  h->partial = dalloc<double>(h, kNormBlocks);
  h->dnorm = dalloc<double>(h, 1);
  check(h, cudaMallocHost(&h->hnorm, sizeof(double)), "cudaMallocHost");
  h->feff = dalloc<double>(h, h->lv.back().ndof);
}

}  // namespace

// =========================================================================== C ABI
extern "C" {

int stm_setup(const st_simplex_mesh* mesh0, int refinements, int p_t, int N, double T, const st_options* opt,
              void* cuda_stream, stm_handle** out) {
  if (!out) return ST_EINVAL;
  *out = nullptr;
  st_options o;
  if (opt) o = *opt;
  else {
    st_default_options(&o);
    o.smoother = ST_SMOOTH_VCYCLE;
  }
  if (const char* why = check_args(mesh0, refinements, p_t, N, T, o)) {
    (void)why;
    return ST_EINVAL;
  }
  stm_handle* h = new (std::nothrow) stm_handle();
  if (!h) return ST_ENOMEM;
  h->d = mesh0->dim;
  h->p_t = p_t;
  h->q = p_t + 1;
  h->N = N;
  h->T = T;
  h->opt = o;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->tm = make_time(p_t);
  int rc = ST_OK;
  try {
    build(h, mesh0, refinements);
  } catch (const Fail& e) {
    rc = e.code;
  } catch (const std::bad_alloc&) {
    rc = ST_ENOMEM;
  } catch (...) {
    rc = ST_ECUDA;
  }
  if (rc != ST_OK) {
    stm_destroy(h);
    return rc;
  }
  *out = h;
  return ST_OK;
}

void stm_destroy(stm_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (void* p : h->allocs) cudaFree(p);
  if (h->hnorm) cudaFreeHost(h->hnorm);
  delete h;
}

const char* stm_last_error(const stm_handle* h) { return h ? h->err.c_str() : "null handle"; }

size_t stm_ndof(const stm_handle* h) { return h ? (size_t)h->lv.back().ndof : 0; }

int stm_num_levels(const stm_handle* h) { return h ? (int)h->lv.size() : 0; }

int stm_nodes(const stm_handle* h, int space_level, int* count, double* coords) {
  if (!h || space_level < 0 || space_level >= (int)h->sp.size()) return ST_EINVAL;
  const SpaceLevel& s = h->sp[space_level];
  if (count) *count = s.Nx;
  if (coords) std::memcpy(coords, s.coords.data(), s.coords.size() * sizeof(double));
  return ST_OK;
}

int stm_level_info(const stm_handle* h, int L, int* N_L, int* space_level, double* mu_L, int* full) {
  if (!h || L < 0 || L >= (int)h->lv.size()) return ST_EINVAL;
  const MLevel& v = h->lv[L];
  if (N_L) *N_L = v.N;
  if (space_level) *space_level = v.l;
  if (mu_L) *mu_L = v.mu;
  if (full) *full = v.full;
  return ST_OK;
}

int stm_residual(stm_handle* h, const double* f, const double* u0_ic, const double* u, double* r) {
  return guarded(h, [&]() -> int {
    if (!f || !u || !r) fail(h, ST_EINVAL, "null pointer");
    const double* g = with_ic(h, f, u0_ic);
    STM_Q(l_residual, h, finest(h), false, g, u, r);
    return ST_OK;
  });
}

int stm_vcycle(stm_handle* h, double* u, const double* f, const double* u0_ic) {
  return guarded(h, [&]() -> int {
    if (!f || !u) fail(h, ST_EINVAL, "null pointer");
    const double* g = with_ic(h, f, u0_ic);
    vcycle(h, (int)h->lv.size() - 1, false, u, g, false);
    return ST_OK;
  });
}

int stm_solve(stm_handle* h, const double* f, const double* u0_ic, double* u, int flags, int* iters, double* relres) {
  return guarded(h, [&]() -> int {
    if (!f || !u) fail(h, ST_EINVAL, "null pointer");
    const double* g = with_ic(h, f, u0_ic);
    return solve_impl(h, false, g, u, (flags & ST_INIT_GIVEN) != 0, iters, relres);
  });
}

int stm_adjoint_solve(stm_handle* h, const double* g, double* lambda, double* grad_u0, int* iters, double* relres) {
  return guarded(h, [&]() -> int {
    if (!g || !lambda) fail(h, ST_EINVAL, "null pointer");
    const int rc = solve_impl(h, true, g, lambda, false, iters, relres);
    if (grad_u0) STM_Q(l_ic_gradient, h, lambda, grad_u0);
    return rc;
  });
}

int stm_level_residual(stm_handle* h, int L, int adjoint, const double* f, const double* u, double* r) {
  return guarded(h, [&]() -> int {
    if (!f || !u || !r) fail(h, ST_EINVAL, "null pointer");
    STM_Q(l_residual, h, h->lv[level_index(h, L)], adjoint != 0, f, u, r);
    return ST_OK;
  });
}

int stm_level_block_solve(stm_handle* h, int L, int adjoint, const double* r, double* d) {
  return guarded(h, [&]() -> int {
    if (!r || !d) fail(h, ST_EINVAL, "null pointer");
    MLevel& lv = h->lv[level_index(h, L)];
    const double* x = space_vcycle(h, lv, lv.l, adjoint != 0, r);
    copy(h, d, x, lv.ndof);
    return ST_OK;
  });
}

int stm_level_smooth(stm_handle* h, int L, int adjoint, int nu, const double* f, double* u) {
  return guarded(h, [&]() -> int {
    if (!f || !u || nu < 0) fail(h, ST_EINVAL, "invalid argument");
    smooth(h, level_index(h, L), adjoint != 0, u, f, nu);
    return ST_OK;
  });
}

int stm_level_restrict(stm_handle* h, int L, const double* r_fine, double* f_coarse) {
  return guarded(h, [&]() -> int {
    if (!r_fine || !f_coarse || level_index(h, L) < 1) fail(h, ST_EINVAL, "invalid argument");
    STM_Q(l_restrict, h, L, r_fine, f_coarse);
    return ST_OK;
  });
}

int stm_level_prolong(stm_handle* h, int L, const double* e_coarse, double* u_fine) {
  return guarded(h, [&]() -> int {
    if (!e_coarse || !u_fine || level_index(h, L) < 1) fail(h, ST_EINVAL, "invalid argument");
    STM_Q(l_prolong, h, L, e_coarse, u_fine);
    return ST_OK;
  });
}

int stm_coarsest_solve(stm_handle* h, int adjoint, const double* f, double* u) {
  return guarded(h, [&]() -> int {
    if (!f || !u) fail(h, ST_EINVAL, "null pointer");
    coarsest(h, adjoint != 0, u, f);
    return ST_OK;
  });
}

}  // extern "C"
