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
  int ell_w = 0;                                      // the rows in slot-major padded form (stmm::Ell)
  int* ell_ci = nullptr;
  double *ell_mv = nullptr, *ell_kv = nullptr;
  float *ell_mv32 = nullptr, *ell_kv32 = nullptr;     // mixed form: the entries rounded to FP32
  int *p0 = nullptr, *p1 = nullptr;                   // parents on the next coarser mesh (level >= 1)
  int *ch_rp = nullptr, *ch_ci = nullptr;             // children on the next finer mesh (level < top)
  double* ch_w = nullptr;
  float* ch_w32 = nullptr;
};

template <typename T>
struct Bufs {                // the vectors and tables of one space-time level in one precision
  T *u = nullptr, *f = nullptr, *r = nullptr;   // FP64: u, f on coarse levels only; FP32: every level
  std::vector<T*> dinv;      // per mesh level k = 1..l: Nx_k q x q inverses of the node blocks (index k)
  T* a0inv = nullptr;        // dense inverse of A_tau on the initial mesh
  std::vector<T*> sb, sx, sy;   // spatial V-cycle buffers per mesh level k = 0..l
};

struct MLevel {              // one space-time level
  int N = 0, l = 0, full = -1;
  double tau = 0.0, mu = 0.0;
  int64_t ndof = 0;
  Bufs<double> d;            // FP64
  Bufs<float> s;             // FP32 (mixed form)
};

template <typename T> Bufs<T>& bufs(MLevel& L);
template <> Bufs<double>& bufs<double>(MLevel& L) { return L.d; }
template <> Bufs<float>& bufs<float>(MLevel& L) { return L.s; }

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

// FP64 host values uploaded rounded to T
template <typename T>
T* upload_as(stm_handle* h, const std::vector<double>& src) {
  std::vector<T> v(src.begin(), src.end());
  return upload(h, v);
}

bool mixed(const stm_handle* h) { return h->opt.precision == ST_MIXED; }

template <typename T, int Q>
stmm::MTime<T, Q> mtime(const HostTime& t) {
  stmm::MTime<T, Q> c{};
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

template <typename T> stmm::Csr<T> csr(const SpaceLevel& s);
template <> stmm::Csr<double> csr<double>(const SpaceLevel& s) { return {s.rp, s.ci, s.mv, s.kv}; }
template <typename T> stmm::Ell<T> ell(const SpaceLevel& s);
template <> stmm::Ell<double> ell<double>(const SpaceLevel& s) { return {s.ell_w, s.ell_ci, s.ell_mv, s.ell_kv}; }
template <> stmm::Ell<float> ell<float>(const SpaceLevel& s) { return {s.ell_w, s.ell_ci, s.ell_mv32, s.ell_kv32}; }
template <typename T> stmm::Children<T> children(const SpaceLevel& s);
template <> stmm::Children<double> children<double>(const SpaceLevel& s) { return {s.ch_rp, s.ch_ci, s.ch_w}; }
template <> stmm::Children<float> children<float>(const SpaceLevel& s) { return {s.ch_rp, s.ch_ci, s.ch_w32}; }
stmm::Parents parents(const SpaceLevel& s) { return stmm::Parents{s.p0, s.p1}; }

unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// grid over (vertices, steps) with the steps on the y axis in chunks of 65535
template <typename F>
void over_steps(int nodes, int steps, F&& launch) {
  for (int s0 = 0; s0 < steps; s0 += 65535) {
    dim3 grid(blocks_for(nodes), (unsigned)std::min(65535, steps - s0));
    launch(grid, s0);
  }
}

// the same for kernels that take stmm::kMSteps consecutive steps per thread
template <typename F>
void over_step_blocks(int nodes, int steps, F&& launch) {
  constexpr int TS = stmm::kMSteps;
  const int nblk = (steps + TS - 1) / TS;
  for (int b0 = 0; b0 < nblk; b0 += 65535) {
    dim3 grid(blocks_for(nodes), (unsigned)std::min(65535, nblk - b0));
    launch(grid, b0 * TS);
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

#define STM_TQ(T, FN, ...)                                             \
  do {                                                                 \
    switch (h->q) {                                                    \
      case 1: FN<T, 1>(__VA_ARGS__); break;                            \
      case 2: FN<T, 2>(__VA_ARGS__); break;                            \
      case 3: FN<T, 3>(__VA_ARGS__); break;                            \
      case 4: FN<T, 4>(__VA_ARGS__); break;                            \
      default: fail(h, ST_EINVAL, "p_t > 3");                          \
    }                                                                  \
  } while (0)

// ------------------------------------------------------------------ launches
template <typename T, int Q>
void l_residual(stm_handle* h, const MLevel& L, bool adj, const T* f, const T* u, T* r) {
  const SpaceLevel& s = h->sp[L.l];
  const auto tc = mtime<T, Q>(h->tm);
  over_step_blocks(s.Nx, L.N, [&](dim3 g, int s0) {
    if (adj)
      stmm::k_mresidual<T, Q, true><<<g, kThreads, 0, h->stream>>>(f, u, r, ell<T>(s), s.Nx, L.N, s0, (T)L.tau, tc);
    else
      stmm::k_mresidual<T, Q, false><<<g, kThreads, 0, h->stream>>>(f, u, r, ell<T>(s), s.Nx, L.N, s0, (T)L.tau, tc);
  });
}

template <typename T, int Q>
void l_jacobi(stm_handle* h, MLevel& L, int k, bool adj, bool zero, const T* b, const T* x, T* y) {
  const SpaceLevel& s = h->sp[k];
  const auto tc = mtime<T, Q>(h->tm);
  const T w = (T)h->opt.omega_x;
  const T* D = bufs<T>(L).dinv[k];
  over_step_blocks(s.Nx, L.N, [&](dim3 g, int s0) {
#define STM_JAC(A, Z)                                                                                        \
  stmm::k_mjacobi<T, Q, A, Z><<<g, kThreads, 0, h->stream>>>(b, x, y, ell<T>(s), s.Nx, L.N, s0, (T)L.tau, w, D, \
                                                              tc)
    if (adj) { if (zero) STM_JAC(true, true); else STM_JAC(true, false); }
    else { if (zero) STM_JAC(false, true); else STM_JAC(false, false); }
#undef STM_JAC
  });
}

template <typename T, int Q>
void l_residual_jacobi0(stm_handle* h, MLevel& L, bool adj, const T* f, const T* u, T* r, T* x) {
  const SpaceLevel& s = h->sp[L.l];
  const auto tc = mtime<T, Q>(h->tm);
  const T* D = bufs<T>(L).dinv[L.l];
  over_step_blocks(s.Nx, L.N, [&](dim3 g, int s0) {
    if (adj)
      stmm::k_mresidual_jacobi0<T, Q, true><<<g, kThreads, 0, h->stream>>>(
          f, u, r, x, ell<T>(s), s.Nx, L.N, s0, (T)L.tau, (T)h->opt.omega_x, D, tc);
    else
      stmm::k_mresidual_jacobi0<T, Q, false><<<g, kThreads, 0, h->stream>>>(
          f, u, r, x, ell<T>(s), s.Nx, L.N, s0, (T)L.tau, (T)h->opt.omega_x, D, tc);
  });
}

template <typename T, int Q>
void l_jacobi_update(stm_handle* h, MLevel& L, bool adj, const T* b, const T* x, T* u) {
  const SpaceLevel& s = h->sp[L.l];
  const auto tc = mtime<T, Q>(h->tm);
  const T* D = bufs<T>(L).dinv[L.l];
  over_step_blocks(s.Nx, L.N, [&](dim3 g, int s0) {
    if (adj)
      stmm::k_mjacobi_update<T, Q, true><<<g, kThreads, 0, h->stream>>>(
          b, x, u, ell<T>(s), s.Nx, L.N, s0, (T)L.tau, (T)h->opt.omega_x, (T)h->opt.omega, D, tc);
    else
      stmm::k_mjacobi_update<T, Q, false><<<g, kThreads, 0, h->stream>>>(
          b, x, u, ell<T>(s), s.Nx, L.N, s0, (T)L.tau, (T)h->opt.omega_x, (T)h->opt.omega, D, tc);
  });
}

template <typename T, int Q>
void l_space_residual(stm_handle* h, const MLevel& L, int k, bool adj, const T* b, const T* x, T* r) {
  const SpaceLevel& s = h->sp[k];
  const auto tc = mtime<T, Q>(h->tm);
  over_step_blocks(s.Nx, L.N, [&](dim3 g, int s0) {
    if (adj)
      stmm::k_mspace_residual<T, Q, true><<<g, kThreads, 0, h->stream>>>(b, x, r, ell<T>(s), s.Nx, L.N, s0,
                                                                           (T)L.tau, tc);
    else
      stmm::k_mspace_residual<T, Q, false><<<g, kThreads, 0, h->stream>>>(b, x, r, ell<T>(s), s.Nx, L.N, s0,
                                                                            (T)L.tau, tc);
  });
}

template <typename T, int Q>
void l_restrict_space(stm_handle* h, const MLevel& L, int k, const T* r, T* bc) {
  const SpaceLevel& c = h->sp[k - 1];
  const SpaceLevel& f = h->sp[k];
  over_steps(c.Nx, L.N, [&](dim3 g, int s0) {
    stmm::k_mrestrict_space<T, Q><<<g, kThreads, 0, h->stream>>>(r, bc, children<T>(c), c.Nx, f.Nx, L.N, s0);
  });
}

template <typename T, int Q>
void l_prolong_space_add(stm_handle* h, const MLevel& L, int k, const T* xc, T* x) {
  const SpaceLevel& c = h->sp[k - 1];
  const SpaceLevel& f = h->sp[k];
  over_steps(f.Nx, L.N, [&](dim3 g, int s0) {
    stmm::k_mprolong_space_add<T, Q><<<g, kThreads, 0, h->stream>>>(xc, x, parents(f), c.Nx, f.Nx, L.N, s0);
  });
}

template <typename T>
void l_dense(stm_handle* h, MLevel& L, bool adj, const T* b, T* y) {
  const int n = h->q * h->sp[0].Nx;
  const T* ainv = bufs<T>(L).a0inv;
  over_steps(n, L.N, [&](dim3 g, int s0) {
    stmm::k_mdense_apply<T><<<g, kThreads, 0, h->stream>>>(b, y, ainv, n, L.N, s0, adj);
  });
}

template <typename T, int Q>
void l_restrict(stm_handle* h, int Li, const T* r, T* fc) {
  const MLevel& F = h->lv[Li];
  const MLevel& C = h->lv[Li - 1];
  const SpaceLevel& cs = h->sp[C.l];
  const SpaceLevel& fs = h->sp[F.l];
  const auto tc = mtime<T, Q>(h->tm);
  over_steps(cs.Nx, C.N, [&](dim3 g, int m0) {
    if (F.l != C.l)
      stmm::k_mrestrict<T, Q, true><<<g, kThreads, 0, h->stream>>>(r, fc, children<T>(cs), cs.Nx, fs.Nx, C.N, m0,
                                                                     tc);
    else
      stmm::k_mrestrict<T, Q, false><<<g, kThreads, 0, h->stream>>>(r, fc, children<T>(cs), cs.Nx, fs.Nx, C.N, m0,
                                                                      tc);
  });
}

template <typename T, int Q>
void l_prolong(stm_handle* h, int Li, const T* ec, T* u) {
  const MLevel& F = h->lv[Li];
  const MLevel& C = h->lv[Li - 1];
  const SpaceLevel& cs = h->sp[C.l];
  const SpaceLevel& fs = h->sp[F.l];
  const auto tc = mtime<T, Q>(h->tm);
  over_steps(fs.Nx, C.N, [&](dim3 g, int m0) {
    if (F.l != C.l)
      stmm::k_mprolong<T, Q, true><<<g, kThreads, 0, h->stream>>>(ec, u, parents(fs), cs.Nx, fs.Nx, C.N, m0, tc);
    else
      stmm::k_mprolong<T, Q, false><<<g, kThreads, 0, h->stream>>>(ec, u, parents(fs), cs.Nx, fs.Nx, C.N, m0, tc);
  });
}

template <int Q>
void l_add_ic(stm_handle* h, const double* f, const double* u0, double* g) {
  const SpaceLevel& s = h->sp.back();
  const auto tc = mtime<double, Q>(h->tm);
  stmm::k_madd_ic<Q><<<blocks_for(s.Nx), kThreads, 0, h->stream>>>(f, u0, g, csr<double>(s), s.Nx, tc);
}

template <int Q>
void l_ic_gradient(stm_handle* h, const double* lam, double* g) {
  const SpaceLevel& s = h->sp.back();
  const auto tc = mtime<double, Q>(h->tm);
  stmm::k_mic_gradient<Q><<<blocks_for(s.Nx), kThreads, 0, h->stream>>>(lam, g, csr<double>(s), s.Nx, tc);
}

template <typename T>
void copy(stm_handle* h, T* y, const T* x, int64_t n) {
  check(h, cudaMemcpyAsync(y, x, sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream), "copy");
}
template <typename T>
void zero(stm_handle* h, T* y, int64_t n) {
  check(h, cudaMemsetAsync(y, 0, sizeof(T) * n, h->stream), "memset");
}
template <typename T>
void axpy(stm_handle* h, T* y, const T* x, T a, int64_t n) {
  stmg::k_axpy<T><<<(unsigned)std::min<int64_t>(blocks_for(n), 152 * 16), kThreads, 0, h->stream>>>(y, x, a, n);
}
unsigned vec_grid(int64_t n) { return (unsigned)std::min<int64_t>(blocks_for(n), 152 * 16); }

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
// that holds the result (one of the level's sx[k], sy[k]); b is not modified.
// x0_done: sx[k] already holds the first sweep omega_x D^{-1} b (fused into the
// residual pass).  update: instead of returning the result, the last sweep adds
// omega_t times it into `update` (the damped step of the smoother) and nullptr is
// returned.
template <typename T>
const T* space_vcycle(stm_handle* h, MLevel& L, int k, bool adj, const T* b, bool x0_done = false,
                      T* update = nullptr) {
  Bufs<T>& B = bufs<T>(L);
  if (k == 0) {
    l_dense<T>(h, L, adj, b, B.sx[0]);
    if (update) {
      axpy<T>(h, update, B.sx[0], (T)h->opt.omega, L.ndof);
      return nullptr;
    }
    return B.sx[0];
  }
  T* x = B.sx[k];
  T* y = B.sy[k];
  const int nu = std::max(1, h->opt.nu_x);
  if (!x0_done) STM_TQ(T, l_jacobi, h, L, k, adj, true, b, (const T*)nullptr, x);
  for (int i = 1; i < nu; ++i) {
    STM_TQ(T, l_jacobi, h, L, k, adj, false, b, x, y);
    std::swap(x, y);
  }
  STM_TQ(T, l_space_residual, h, L, k, adj, b, x, y);        // y = b - A x
  STM_TQ(T, l_restrict_space, h, L, k, y, B.sb[k - 1]);
  const T* xc = space_vcycle<T>(h, L, k - 1, adj, B.sb[k - 1]);
  STM_TQ(T, l_prolong_space_add, h, L, k, xc, x);
  for (int i = 0; i < nu; ++i) {
    if (update != nullptr && i == nu - 1) {
      STM_TQ(T, l_jacobi_update, h, L, adj, b, x, update);
      return nullptr;
    }
    STM_TQ(T, l_jacobi, h, L, k, adj, false, b, x, y);
    std::swap(x, y);
  }
  return x;
}

// u <- u + omega D~^{-1} (f - L u), nu times (eq. chap4_smoother).  On a level
// whose mesh is refined, the residual pass also takes the first Jacobi sweep of
// the spatial V-cycle and the last sweep adds into u directly.
template <typename T>
void smooth(stm_handle* h, int Li, bool adj, T* u, const T* f, int nu) {
  MLevel& L = h->lv[Li];
  Bufs<T>& B = bufs<T>(L);
  for (int i = 0; i < nu; ++i) {
    if (L.l >= 1) {
      STM_TQ(T, l_residual_jacobi0, h, L, adj, f, u, B.r, B.sx[L.l]);
      space_vcycle<T>(h, L, L.l, adj, (const T*)B.r, true, u);
    } else {
      STM_TQ(T, l_residual, h, L, adj, f, u, B.r);
      const T* d = space_vcycle<T>(h, L, L.l, adj, (const T*)B.r);
      axpy<T>(h, u, d, (T)h->opt.omega, L.ndof);
    }
  }
}

// Exact solve on the coarsest level (one time step) in FP64: A u = f by spatial
// V-cycles repeated until the residual stops decreasing below 1e-13 ||f||
// (one V-cycle is exact when the level's mesh is the initial one).
void coarsest64(stm_handle* h, bool adj, double* u, const double* f) {
  MLevel& L = h->lv[0];
  if (L.l == 0) {
    l_dense<double>(h, L, adj, f, u);
    return;
  }
  zero<double>(h, u, L.ndof);
  copy<double>(h, L.d.r, f, L.ndof);
  const double f0 = norm2(h, f, L.ndof);
  if (f0 == 0.0) return;
  double prev = f0;
  for (int it = 0; it < 100; ++it) {
    const double* d = space_vcycle<double>(h, L, L.l, adj, L.d.r);
    axpy<double>(h, u, d, 1.0, L.ndof);
    STM_TQ(double, l_space_residual, h, L, L.l, adj, f, u, L.d.r);
    const double rn = norm2(h, L.d.r, L.ndof);
    if (!std::isfinite(rn)) fail(h, ST_ENAN, "coarsest solve: residual not finite");
    if (rn <= 1e-15 * f0 || (rn <= 1e-13 * f0 && rn > 0.5 * prev)) break;
    prev = rn;
  }
}

// The coarsest solve of the FP32 cycles runs in FP64 (the FP64 buffers of level 0).
template <typename T>
void coarsest(stm_handle* h, bool adj, T* u, const T* f);
template <>
void coarsest<double>(stm_handle* h, bool adj, double* u, const double* f) {
  coarsest64(h, adj, u, f);
}
template <>
void coarsest<float>(stm_handle* h, bool adj, float* u, const float* f) {
  MLevel& L = h->lv[0];
  stmg::k_cast_up<<<vec_grid(L.ndof), kThreads, 0, h->stream>>>(L.d.f, f, L.ndof);
  coarsest64(h, adj, L.d.u, L.d.f);
  stmg::k_cast_down<<<vec_grid(L.ndof), kThreads, 0, h->stream>>>(u, L.d.u, 1.0, L.ndof);
}

template <typename T>
void vcycle(stm_handle* h, int Li, bool adj, T* u, const T* f, bool u_zero) {
  if (Li == 0) {
    coarsest<T>(h, adj, u, f);
    return;
  }
  MLevel& L = h->lv[Li];
  if (u_zero) zero<T>(h, u, L.ndof);
  smooth<T>(h, Li, adj, u, f, h->opt.nu1);
  Bufs<T>& B = bufs<T>(L);
  STM_TQ(T, l_residual, h, L, adj, f, (const T*)u, B.r);
  MLevel& C = h->lv[Li - 1];
  Bufs<T>& CB = bufs<T>(C);
  STM_TQ(T, l_restrict, h, Li, (const T*)B.r, CB.f);
  const int reps = (Li - 1 == 0) ? 1 : std::max(1, h->opt.gamma);
  for (int g = 0; g < reps; ++g) vcycle<T>(h, Li - 1, adj, CB.u, (const T*)CB.f, g == 0);
  STM_TQ(T, l_prolong, h, Li, (const T*)CB.u, u);
  smooth<T>(h, Li, adj, u, f, h->opt.nu2);
}

MLevel& finest(stm_handle* h) { return h->lv.back(); }

// f + IC on the finest level into the handle's copy (u0 may be null).
const double* with_ic(stm_handle* h, const double* f, const double* u0) {
  if (u0 == nullptr) return f;
  MLevel& F = finest(h);
  copy<double>(h, h->feff, f, F.ndof);
  STM_Q(l_add_ic, h, f, u0, h->feff);
  return h->feff;
}

// One refinement step of the mixed form: given the FP64 residual r (norm s > 0)
// of the finest level, inner_cycles FP32 cycles on L e = r / s from e = 0, then
// u += s e in FP64.
void mixed_step(stm_handle* h, bool adj, double* u, const double* r, double s) {
  MLevel& F = finest(h);
  const int top = (int)h->lv.size() - 1;
  stmg::k_cast_down<<<vec_grid(F.ndof), kThreads, 0, h->stream>>>(F.s.f, r, 1.0 / s, F.ndof);
  for (int c = 0; c < std::max(1, h->opt.inner_cycles); ++c) vcycle<float>(h, top, adj, F.s.u, F.s.f, c == 0);
  stmg::k_axpy_up<<<vec_grid(F.ndof), kThreads, 0, h->stream>>>(u, F.s.u, s, F.ndof);
}

int solve_impl(stm_handle* h, bool adj, const double* f, double* u, bool given, int* iters, double* relres) {
  MLevel& F = finest(h);
  const int top = (int)h->lv.size() - 1;
  if (!given) zero<double>(h, u, F.ndof);
  STM_TQ(double, l_residual, h, F, adj, f, (const double*)u, F.d.r);
  const double r0 = norm2(h, F.d.r, F.ndof);
  double rn = r0;
  int it = 0, status = ST_OK;
  if (!std::isfinite(r0)) status = ST_ENAN;
  while (status == ST_OK && r0 > 0.0 && rn > h->opt.rtol * r0) {
    if (it >= h->opt.maxit) { status = ST_ENOTCONV; h->err = "maxit reached"; break; }
    if (mixed(h)) mixed_step(h, adj, u, F.d.r, rn);
    else vcycle<double>(h, top, adj, u, f, false);
    ++it;
    STM_TQ(double, l_residual, h, F, adj, f, (const double*)u, F.d.r);
    rn = norm2(h, F.d.r, F.ndof);
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
  if (o.precision != ST_FP64 && o.precision != ST_MIXED) return "precision must be ST_FP64 or ST_MIXED";
  if (o.inner_cycles < 0) return "inner_cycles must be >= 0";
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
    {   // slot-major padded rows (stmm::Ell)
      int w = 0;
      for (int i = 0; i < s.Nx; ++i) w = std::max(w, s.rp_h[i + 1] - s.rp_h[i]);
      s.ell_w = w;
      std::vector<int> eci((size_t)w * s.Nx);
      std::vector<double> emv((size_t)w * s.Nx, 0.0), ekv((size_t)w * s.Nx, 0.0);
      for (int i = 0; i < s.Nx; ++i)
        for (int k = 0; k < w; ++k) {
          const int e = s.rp_h[i] + k;
          const size_t o = (size_t)k * s.Nx + i;
          if (e < s.rp_h[i + 1]) {
            eci[o] = s.ci_h[e];
            emv[o] = s.mv_h[e];
            ekv[o] = s.kv_h[e];
          } else {
            eci[o] = i;
          }
        }
      s.ell_ci = upload(h, eci);
      s.ell_mv = upload(h, emv);
      s.ell_kv = upload(h, ekv);
      if (mixed(h)) {
        s.ell_mv32 = upload_as<float>(h, emv);
        s.ell_kv32 = upload_as<float>(h, ekv);
      }
    }
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
      if (mixed(h)) c.ch_w32 = upload_as<float>(h, cw);
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
  // workspace and per-level tables (FP64 always; the mixed form adds FP32 copies)
  const bool mx = mixed(h);
  for (int i = 0; i < nl; ++i) {
    MLevel& L = h->lv[i];
    const bool top = i == nl - 1;
    if (!top || i == 0) {   // level 0 keeps FP64 u, f for the FP64 coarsest solve of the FP32 cycles
      L.d.u = dalloc<double>(h, L.ndof);
      L.d.f = dalloc<double>(h, L.ndof);
    }
    L.d.r = dalloc<double>(h, L.ndof);
    if (mx) {
      L.s.u = dalloc<float>(h, L.ndof);
      L.s.f = dalloc<float>(h, L.ndof);
      L.s.r = dalloc<float>(h, L.ndof);
    }
    for (Bufs<double>* B : {&L.d}) {
      B->sb.assign(L.l + 1, nullptr);
      B->sx.assign(L.l + 1, nullptr);
      B->sy.assign(L.l + 1, nullptr);
      B->dinv.assign(L.l + 1, nullptr);
    }
    L.s.sb.assign(L.l + 1, nullptr);
    L.s.sx.assign(L.l + 1, nullptr);
    L.s.sy.assign(L.l + 1, nullptr);
    L.s.dinv.assign(L.l + 1, nullptr);
    for (int kk = 0; kk <= L.l; ++kk) {
      const int64_t n = (int64_t)L.N * q * h->sp[kk].Nx;
      L.d.sx[kk] = dalloc<double>(h, n);
      if (kk >= 1) L.d.sy[kk] = dalloc<double>(h, n);
      if (kk < L.l) L.d.sb[kk] = dalloc<double>(h, n);
      if (mx) {
        L.s.sx[kk] = dalloc<float>(h, n);
        if (kk >= 1) L.s.sy[kk] = dalloc<float>(h, n);
        if (kk < L.l) L.s.sb[kk] = dalloc<float>(h, n);
      }
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
        L.d.dinv[kk] = upload(h, tab);
        if (mx) L.s.dinv[kk] = upload_as<float>(h, tab);
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
      L.d.a0inv = upload(h, A);
      if (mx) L.s.a0inv = upload_as<float>(h, A);
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
    STM_TQ(double, l_residual, h, finest(h), false, g, u, r);
    return ST_OK;
  });
}

int stm_vcycle(stm_handle* h, double* u, const double* f, const double* u0_ic) {
  return guarded(h, [&]() -> int {
    if (!f || !u) fail(h, ST_EINVAL, "null pointer");
    const double* g = with_ic(h, f, u0_ic);
    if (mixed(h)) {   // one refinement step
      MLevel& F = finest(h);
      STM_TQ(double, l_residual, h, F, false, g, (const double*)u, F.d.r);
      const double rn = norm2(h, F.d.r, F.ndof);
      if (!std::isfinite(rn)) fail(h, ST_ENAN, "residual norm is not finite");
      if (rn > 0.0) mixed_step(h, false, u, F.d.r, rn);
      return ST_OK;
    }
    vcycle<double>(h, (int)h->lv.size() - 1, false, u, g, false);
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
    STM_TQ(double, l_residual, h, h->lv[level_index(h, L)], adjoint != 0, f, u, r);
    return ST_OK;
  });
}

int stm_level_block_solve(stm_handle* h, int L, int adjoint, const double* r, double* d) {
  return guarded(h, [&]() -> int {
    if (!r || !d) fail(h, ST_EINVAL, "null pointer");
    MLevel& lv = h->lv[level_index(h, L)];
    const double* x = space_vcycle<double>(h, lv, lv.l, adjoint != 0, r);
    copy<double>(h, d, x, lv.ndof);
    return ST_OK;
  });
}

int stm_level_smooth(stm_handle* h, int L, int adjoint, int nu, const double* f, double* u) {
  return guarded(h, [&]() -> int {
    if (!f || !u || nu < 0) fail(h, ST_EINVAL, "invalid argument");
    smooth<double>(h, level_index(h, L), adjoint != 0, u, f, nu);
    return ST_OK;
  });
}

int stm_level_restrict(stm_handle* h, int L, const double* r_fine, double* f_coarse) {
  return guarded(h, [&]() -> int {
    if (!r_fine || !f_coarse || level_index(h, L) < 1) fail(h, ST_EINVAL, "invalid argument");
    STM_TQ(double, l_restrict, h, L, r_fine, f_coarse);
    return ST_OK;
  });
}

int stm_level_prolong(stm_handle* h, int L, const double* e_coarse, double* u_fine) {
  return guarded(h, [&]() -> int {
    if (!e_coarse || !u_fine || level_index(h, L) < 1) fail(h, ST_EINVAL, "invalid argument");
    STM_TQ(double, l_prolong, h, L, e_coarse, u_fine);
    return ST_OK;
  });
}

int stm_coarsest_solve(stm_handle* h, int adjoint, const double* f, double* u) {
  return guarded(h, [&]() -> int {
    if (!f || !u) fail(h, ST_EINVAL, "null pointer");
    coarsest<double>(h, adjoint != 0, u, f);
    return ST_OK;
  });
}

}  // extern "C"
