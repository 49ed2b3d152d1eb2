// Allocation-free l2 norm.
//
// Some callers cannot allocate device memory: an application that hands
// all of a GPU's memory to its own allocator at start-up and forbids later
// cudaMalloc, or a code path that must not take the implicit device
// synchronisation that cudaMalloc / cudaFree may perform.  For them
// st_norm2_noalloc computes the l2 norm that st_norm2 computes, without a
// handle (creating one allocates) and with its partial sums in a fixed
// file-scope device array instead of handle workspace.  Its sum of squares is
// deterministic in its own fixed order -- one partial per contiguous chunk of
// kNoallocChunk elements, then one block adds the partials -- which is not the
// order of st_norm2 (a fixed grid-stride split), so the two agree to rounding.
//
// Limits and sharing rules (also stated in include/stmg.h):
//  * the scratch holds kNoallocPartials FP64 partial sums (128 KB per GPU that
//    loads this library, held until the process exits); each partial covers a
//    fixed chunk of kNoallocChunk elements, so at most
//    kNoallocPartials * kNoallocChunk = 2^30 elements per call;
//  * every call shares the one array; calls whose kernels overlap on the GPU
//    (different streams, no ordering between them) race on it;
//  * stage 1 writes every partial that stage 2 reads, so nothing has to be
//    cleared between calls;
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture;
//  * a CUDA error that is already pending on the calling thread (from earlier,
//    unrelated work) is neither cleared nor attributed to a launch here: the
//    call returns ST_ECUDA before launching anything and leaves the error for
//    the caller's own check; launch failures of its own kernels are read with
//    cudaPeekAtLastError, which does not clear them either.
#include <atomic>
#include <cstdint>
#include <mutex>

#include "stmg.h"

namespace {

constexpr int kNoallocPartials = 16384;               // 128 KB of FP64
constexpr int64_t kNoallocChunk = int64_t(1) << 16;   // elements per partial
static_assert((int64_t)kNoallocPartials * kNoallocChunk == (int64_t)ST_NOALLOC_MAX_ELEMENTS,
              "header limit and scratch size disagree");
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoallocPartials];

// Stage 1: block b sums the squares of elements [b*chunk, min((b+1)*chunk, n)),
// fixed thread ranges and a fixed reduction tree, into partial[b].
__global__ void k_noalloc_sumsq(const double* __restrict__ x, int64_t n, double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const int64_t begin = (int64_t)blockIdx.x * kNoallocChunk;
  const int64_t end = begin + kNoallocChunk < n ? begin + kNoallocChunk : n;
  double acc = 0.0;
  for (int64_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
    const double v = x[i];
    acc += v * v;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    acc = lane < (kThreads / 32) ? red[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) partial[blockIdx.x] = acc;
  }
}

// Stage 2: one block adds the partials in a fixed order and writes the root.
__global__ void k_noalloc_finish(const double* __restrict__ partial, int np, double* __restrict__ out) {
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
    if (lane == 0) out[0] = sqrt(acc);
  }
}

// Device address of g_noalloc_partials, looked up once per device.
std::atomic<double*> g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ST_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return ST_EINVAL;
  double* p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (p == nullptr) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    p = g_scratch_addr[dev].load(std::memory_order_relaxed);
    if (p == nullptr) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_noalloc_partials) != cudaSuccess || addr == nullptr) {
        cudaGetLastError();
        return ST_ECUDA;
      }
      p = static_cast<double*>(addr);
      g_scratch_addr[dev].store(p, std::memory_order_release);
    }
  }
  *out = p;
  return ST_OK;
}

}  // namespace

extern "C" int st_norm2_noalloc(const double* x, size_t n, double* out, void* cuda_stream) {
  if (x == nullptr || out == nullptr) return ST_EINVAL;
  if (n > (size_t)ST_NOALLOC_MAX_ELEMENTS) return ST_EINVAL;   // beyond the scratch capacity
  if (cudaPeekAtLastError() != cudaSuccess) return ST_ECUDA;   // an earlier error, left pending for its owner
  double* scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != ST_OK) return rc;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const int np = n == 0 ? 1 : (int)((n + kNoallocChunk - 1) / kNoallocChunk);
  k_noalloc_sumsq<<<np, kThreads, 0, stream>>>(x, (int64_t)n, scratch);
  if (cudaPeekAtLastError() != cudaSuccess) return ST_ECUDA;
  k_noalloc_finish<<<1, 1024, 0, stream>>>(scratch, np, out);
  return cudaPeekAtLastError() == cudaSuccess ? ST_OK : ST_ECUDA;
}
