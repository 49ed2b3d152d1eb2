// Sine transform (DST-I) of FP64 lines on the tcgen05 tensor cores.
//
// The exact block inverse of Section 3.1 diagonalises the spatial operators with the
// discrete sine transform y_k = sum_{j=1..n} x_j sin(pi j k / Nf), Nf = n + 1.  Here it is
// a dense product with the sine matrix S, computed exactly in integer arithmetic on the
// FP16 tensor cores (a digit-splitting scheme in the manner of Ozaki):
//
//  * each line's values are scaled by the line's largest exponent Er to 56-bit integers
//    F = |x| 2^(1078 - Er) and cut into eight 7-bit digits d_0 .. d_7 (most significant first);
//  * S / 2 is cut into eight balanced base-128 digits e_0 .. e_7 in [-64, 64];
//  * every digit is an FP16 integer, and the products d_s e_t with s + t = g are summed over
//    K (Nf <= 256 terms) into accumulator g = 0 .. 7 in FP32 tensor memory.  The bound
//    |C_g| <= 255 * 127 * 64 * (g + 1) < 2^24 keeps every partial sum an exact integer;
//  * the epilogue forms W = sum_g C_g 2^(7 (7 - g)) exactly in integers and rounds
//    W 2^(Er - 1084 + out_exp) once to FP64.
// Dropped pairs (s + t >= 8) and the 56-bit truncation of x keep the error near 2^-53 of
// the line's scale (measured below 5e-16 of sqrt(Nf / 2) ||x||_2).
//
// Work split: a split pass (k_split_planes) reads 16 lines per CTA through shared memory, finds each
// line's largest exponent and writes the FP16 digit planes of every value once, in the exact layout of
// one pipeline stage of the tensor kernel (32 KB per 128 lines x 16 K); the tensor kernel k_dst_tc is
// persistent (one CTA per SM) and warp-specialised:
//   warp 0     brings each chunk's data planes and sine planes with two bulk copies (48 KB) into a
//              3-stage ring;
//   warp 1     issues 12 tcgen05.mma per chunk: for digit s, the sine planes t = t0 .. t0 + 3
//              are adjacent along N, so one M = 128, N = 64 cnt MMA feeds accumulators
//              s + t0 .. s + t0 + cnt - 1 (N <= 256);
//   warps 2 .. 8 (Nf = 256) or 16 (Nf <= 128) epilogue warps drain the eight accumulators (TMEM,
//              512 columns) into the exact integer of each output in shared memory, release TMEM to
//              the next tile's MMAs, then round to FP64 and store.
// Every wait on an mbarrier is bounded: on time-out the kernel raises *err, drains its own
// tensor-core and bulk-copy work and returns.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace stmg_tc {

constexpr int BM = 128;                  // lines per tile (MMA M, TMEM lanes)
constexpr int BNP = 64;                  // output frequencies per tile (N of one sine digit plane)
constexpr int BK = 16;                   // K of one pipeline stage (one MMA K-step)
constexpr int NSL = 8;                   // base-128 digits per operand
constexpr int A_PLANE = BM * BK * 2;     // 4 KB: one FP16 data digit plane of a chunk
constexpr int B_PLANE = BNP * BK * 2;    // 2 KB: one FP16 sine digit plane of a chunk
constexpr int A_STAGE = NSL * A_PLANE;   // 32 KB
constexpr int B_STAGE = NSL * B_PLANE;   // 16 KB (the sine table stores this per (N tile, chunk))
constexpr int NST = 3;                   // pipeline stages
constexpr int TMA_WARP = 0;              // bulk copies of the stages
constexpr int MMA_WARP = 1;              // MMA issuer
constexpr int EPI0 = 2;                  // epilogue warps from 2 on: NE / 4 per TMEM lane quadrant (warp % 4)
constexpr int NEPI = 8;                  // epilogue warps for Nf = 256 (the MMAs of a tile hide their work)
constexpr int NEPI_SHORT = 16;           // for Nf <= 128: 4 or 8 K-chunks per tile, the epilogue sets the pace
constexpr int NTHREADS = (EPI0 + NEPI) * 32;
__host__ __device__ constexpr int threads_for(int ne) { return (EPI0 + ne) * 32; }
constexpr int TS_BYTES = 4 * BNP * 32 * 10;   // staged exact sums of a tile: 64 columns x 128 lines x (8 + 2) B
constexpr int kMaxNf = 256;              // Nf <= 256 keeps every accumulator below 2^24
constexpr int kMinNf = 64;
constexpr uint32_t kWaitLimit = 1u << 24;
constexpr int kZeroExp = -1100;          // exponent assigned to zero (below every FP64 exponent)

struct Smem {
  static constexpr int a_off = 0;
  static constexpr int b_off = a_off + NST * A_STAGE;
  static constexpr int ts_off = b_off + NST * B_STAGE;   // per warp: int64 high parts, then uint16 remainders
  static constexpr int bar_off = ts_off + TS_BYTES;
  static constexpr int nbars = 2 * NST + 3;   // full[NST], empty[NST], accf, acce, drain
  static constexpr int misc_off = bar_off + nbars * 8;
  static constexpr int bytes = misc_off + 16 + 1024;   // + slack for 1024-byte alignment of the base
};

// Bytes of the digit planes of the split pass for nlines lines of Nf - 1 values (16 per value).
inline size_t plane_bytes_for(int64_t nlines, int Nf) { return (size_t)((nlines + BM - 1) / BM * BM) * (size_t)Nf * 16; }

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major, no swizzle: 8 x 16-byte core matrices, LBO 128 B
// (next core matrix along K), SBO 256 B (next group of 8 rows).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: FP16 A and B (K-major), FP32 accumulator, M = 128, N.
__device__ __forceinline__ uint32_t idesc_n(uint32_t N) {
  return (1u << 4) | ((N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}

// Bounded wait: false once the limit is reached (raises the abort flag and *err) or another role aborted.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err, int code) {
  for (uint32_t i = 0;; ++i) {
    if (try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u && *abort_flag) return false;
    if (i > kWaitLimit) {
      *abort_flag = 1;
      atomicExch(err, code);
      return false;
    }
  }
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(addr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ uint32_t hfma2(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Exponent of the leading bit of x on the biased scale of normal numbers: the exponent field
// for normal x, 1 - (leading zeros of the 52-bit fraction) for subnormal x, kZeroExp for zero.
__device__ __forceinline__ int exp_of(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  const int E = (int)(b >> 52);
  if (E) return E;
  if (b == 0ull) return kZeroExp;
  return (63 - __clzll((long long)b)) - 51;
}

// F = |x| 2^(1078 - Er) truncated to an integer (F < 2^56 since Er >= exp_of(x)), as its
// 28-bit halves f2 = F >> 28 and f1 = F mod 2^28.  Subnormal x are read with exponent 1 and
// no implicit bit (exact); a line whose maximum is subnormal has Er <= 0 and shifts left.
__device__ __forceinline__ void split28(double x, int Er, uint32_t& f2, uint32_t& f1) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = ((b & 0xfffffffffffffull) | (E ? (1ull << 52) : 0ull)) << 3;
  const int sh = Er - (E ? E : 1);
  const unsigned long long F = sh >= 0 ? (m >> (sh < 63 ? sh : 63)) : (m << (-sh < 63 ? -sh : 63));
  f2 = (uint32_t)(F >> 28);
  f1 = (uint32_t)F & 0x0fffffffu;
}

// The FP16 digit s of two values a, b as one word (a low, b high): the 7-bit fields of their fixed-point
// halves at bit pos, as FP16 1024 + d, then sign and offset in one f16x2 fma: +-(1024 + d) -+ 1024.
__device__ __forceinline__ uint32_t digit_pair(uint32_t ha, uint32_t hb, int pos, uint32_t sgn2, uint32_t nm2) {
  const uint32_t w = ((ha >> pos) & 0x7fu) | (((hb >> pos) & 0x7fu) << 16) | 0x64006400u;
  return hfma2(w, sgn2, nm2);
}

constexpr int SPLIT_LINES = 16;          // lines per CTA of the split pass
constexpr int SPLIT_ROW = kMaxNf + 1;    // shared-memory row of one line (odd: no bank conflicts)

// Split pass: digit planes of lines L0 .. L0 + 15 (L0 = 16 blockIdx.x) of the padded line blocks.
// Line L: x_j at in[L n + j - 1] (ROWS) or in[(L / inner) n inner + (j - 1) inner + L % inner];
// x_0 and lines >= nlines are zero.  lineE[L] = largest exp_of over line L (L < nlines).
// P: per (line block b, K chunk c) one stage of 8 planes x 4 KB; plane s holds digit s of
// (row, k) at byte ((row / 8) 2 + (k / 8) % 2) 128 + (row % 8) 16 + (k % 8) 2 (K-major core
// matrices).  256 threads; 64 <= Nf = n + 1 <= 256.
template <bool ROWS>
__global__ void __launch_bounds__(256) k_split_planes(const double* __restrict__ in, int n, int64_t nlines,
                                                      int64_t inner, int nch, int* __restrict__ lineE,
                                                      uint4* __restrict__ P) {
  __shared__ double xs[SPLIT_LINES * SPLIT_ROW];
  __shared__ int es[SPLIT_LINES];
  const int Nf = n + 1;
  const int64_t L0 = (int64_t)blockIdx.x * SPLIT_LINES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (ROWS) {   // warp w loads lines 2w, 2w + 1: 32 consecutive values per instruction
    double v[2][kMaxNf / 32];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t L = L0 + 2 * warp + h;
#pragma unroll
      for (int i = 0; i < kMaxNf / 32; ++i) {
        const int j = 32 * i + lane;   // x_(j + 1)
        v[h][i] = (L < nlines && j < n) ? in[L * n + j] : 0.0;
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double* row = xs + (2 * warp + h) * SPLIT_ROW;
#pragma unroll
      for (int i = 0; i < kMaxNf / 32; ++i)
        if (32 * i + lane < n) row[32 * i + lane + 1] = v[h][i];
      if (lane == 0) row[0] = 0.0;
    }
  } else {      // thread (line r, offset jj): 16 consecutive lines x 2 positions per warp instruction
    const int r = tid & 15, jj = tid >> 4;
    const int64_t L = L0 + r;
    const bool live = L < nlines;
    const double* p = live ? in + (L / inner) * n * inner + (L % inner) : in;
    double v[kMaxNf / 16];
#pragma unroll
    for (int i = 0; i < kMaxNf / 16; ++i) {
      const int j = jj + 16 * i;   // x_(j + 1)
      v[i] = (live && j < n) ? p[(int64_t)j * inner] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < kMaxNf / 16; ++i)
      if (jj + 16 * i < n) xs[r * SPLIT_ROW + jj + 16 * i + 1] = v[i];
    if (jj == 0) xs[r * SPLIT_ROW] = 0.0;
  }
  __syncthreads();
  for (int r = 2 * warp; r < 2 * warp + 2; ++r) {   // 8 warps, 2 lines each
    int e = kZeroExp;
    for (int k = lane; k < Nf; k += 32) e = max(e, exp_of(xs[r * SPLIT_ROW + k]));
#pragma unroll
    for (int o = 16; o; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (lane == 0) {
      es[r] = e;
      if (L0 + r < nlines) lineE[L0 + r] = e;
    }
  }
  __syncthreads();
  // lane -> (row r, K group kg): lanes 0-7 rows 0-7 kg 0, 8-15 rows 0-7 kg 1, 16-31 rows 8-15;
  // the 32 lanes' 16-byte pieces of one plane are then 512 contiguous bytes
  const int r = (lane & 7) + 8 * (lane >> 4), kg = (lane >> 3) & 1;
  const int Er = es[r];
  const int64_t b = L0 / BM;
  const int m = (int)((L0 % BM) / SPLIT_LINES);
  for (int c = warp; c < nch; c += 8) {
    const double* xr = xs + r * SPLIT_ROW + 16 * c + 8 * kg;
    uint32_t w[NSL][4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const double xa = xr[2 * p], xb = xr[2 * p + 1];
      uint32_t a2, a1, b2, b1;
      split28(xa, Er, a2, a1);
      split28(xb, Er, b2, b1);
      const uint32_t sbits = (((uint32_t)__double2hiint(xa) >> 31) << 15) | (((uint32_t)__double2hiint(xb) >> 31) << 31);
      const uint32_t sgn2 = 0x3c003c00u | sbits, nm2 = 0xe400e400u ^ sbits;   // (+-1, +-1), (-+1024, -+1024)
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        w[s][p] = digit_pair(a2, b2, 21 - 7 * s, sgn2, nm2);
        w[4 + s][p] = digit_pair(a1, b1, 21 - 7 * s, sgn2, nm2);
      }
    }
    uint4* stage = P + ((b * nch + c) * (A_STAGE / 16)) + 32 * m + lane;
#pragma unroll
    for (int s = 0; s < NSL; ++s) stage[s * (A_PLANE / 16)] = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
  }
}

// value = W 2^e0 rounded to nearest even, any W (subnormal and overflowing results included).
__device__ __noinline__ double assemble128(__int128 W, int e0) {
  if (W == 0) return 0.0;
  const bool neg = W < 0;
  const unsigned __int128 M = neg ? (unsigned __int128)(-W) : (unsigned __int128)W;
  const unsigned long long mh = (unsigned long long)(M >> 64), ml = (unsigned long long)M;
  const int p = mh ? 127 - __clzll((long long)mh) : 63 - __clzll((long long)ml);
  int sh = p - 52;                      // quantum exponent relative to M's unit: 53 significant bits,
  const int qmin = -1074 - e0;          // but no finer than 2^-1074
  if (sh < qmin) sh = qmin;
  unsigned long long q;
  if (sh <= 0) {
    q = ml << (-sh);
  } else if (sh >= 128) {
    q = 0;
  } else {
    q = (unsigned long long)(M >> sh);
    const unsigned __int128 rem = M - ((unsigned __int128)q << sh);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  if (q >> 53) { q >>= 1; ++sh; }
  const long long ef = (long long)sh + e0 + 1074;   // exponent field of q 2^(sh + e0) with q < 2^53
  unsigned long long bits;
  if (ef + (long long)(q >> 52) >= 2047) bits = 0x7ff0000000000000ull;
  else bits = q + ((unsigned long long)ef << 52);
  if (neg) bits |= 0x8000000000000000ull;
  return __longlong_as_double((long long)bits);
}

// value = (Vp 2^14 + r) 2^e0 rounded to nearest even, |Vp| < 2^58, 0 <= r < 2^14, branch-free for
// results in the normal range; slow = true when the result is subnormal or overflows (use assemble128).
__device__ __forceinline__ double assemble_vr(long long Vp, uint32_t r, int e0, bool& slow) {
  const bool neg = Vp < 0;
  const unsigned long long A = neg ? (unsigned long long)(-Vp) - (r ? 1ull : 0ull) : (unsigned long long)Vp;
  const uint32_t B = neg ? (r ? 16384u - r : 0u) : r;   // |W| = A 2^14 + B = (hw, lw) as 128 bits
  const unsigned long long lw = (A << 14) | B, hw = A >> 50;
  const int p = A ? 77 - __clzll((long long)A) : (B ? 31 - __clz((int)B) : 0);   // leading bit of |W|
  const int be = p + e0 + 1023;
  const int sh = p - 52;                                                      // in [-52, 19]
  const int shp = sh > 0 ? sh : 0, shn = sh < 0 ? -sh : 0;
  unsigned long long q = (lw >> shp) | (shp ? (hw << (64 - shp)) : 0ull);
  q <<= shn;
  const unsigned long long mask = shp ? ((1ull << shp) - 1ull) : 0ull;
  const unsigned long long rem = lw & mask, half = shp ? (1ull << (shp - 1)) : 1ull;
  q += (shp && (rem > half || (rem == half && (q & 1ull)))) ? 1ull : 0ull;
  const int carry = (int)(q >> 53);
  q >>= carry;
  const int e = be + carry;
  slow = (be <= 0) || (e >= 2047);
  const unsigned long long bits =
      ((A | B) == 0ull) ? 0ull
                        : ((q & 0xfffffffffffffull) | ((unsigned long long)e << 52) | (neg ? 0x8000000000000000ull : 0ull));
  return __longlong_as_double((long long)bits);
}

// y_k = 2^out_exp sum_{j=1..n} x_j sin(pi j k / Nf), k = 1 .. n, Nf = n + 1 = 16 nch = 64 ntn
// (64 <= Nf <= 256), for every line, from the digit planes P and line exponents lineE of the split
// pass.  Output line L: y_k at out[L n + k - 1] (ROWS) or out[(L / inner) n inner + (k - 1) inner
// + L % inner].  sdig: FP16 digits of S / 2, B_STAGE bytes per (N tile, K chunk).  Launch with
// threads_for(NE) threads (NE = 8 or 16 epilogue warps), Smem::bytes of dynamic shared memory and at
// most one CTA per SM.
template <bool ROWS, int NE>
__global__ void __launch_bounds__(threads_for(NE), 1)
k_dst_tc(const uint8_t* __restrict__ P, double* __restrict__ out, int n, int64_t nlines, int64_t inner,
         const int* __restrict__ lineE, const uint8_t* __restrict__ sdig, int nch, int ntn, int out_exp,
         int* __restrict__ err) {
  using SL = Smem;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = su32(smem_raw);
  const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
  unsigned char* sm = smem_raw + pad;
  const uint32_t sbase = raw + pad;
  const uint32_t bars = sbase + SL::bar_off;
  auto full = [&](int s) { return bars + 8u * (uint32_t)s; };            // both bulk copies landed
  auto empty = [&](int s) { return bars + 8u * (uint32_t)(NST + s); };   // the stage's MMAs completed
  const uint32_t accf = bars + 8u * (uint32_t)(2 * NST), acce = accf + 8u, drain = accf + 16u;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + SL::misc_off);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + SL::misc_off + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nrb = (nlines + BM - 1) / BM;
  const int64_t ntiles = nrb * ntn;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(su32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < NST; ++s) {
      bar_init(full(s), 1);
      bar_init(empty(s), 1);
    }
    bar_init(accf, 1);
    bar_init(acce, NE);
    bar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = *tslot;

  if (warp == TMA_WARP) {
    // ---- bulk copies: the chunk's data planes (split pass) and sine planes ----
    if (lane == 0) {
      uint32_t it = 0;
      for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t b = t / ntn;
        const int nt = (int)(t % ntn);
        bool alive = true;
        for (int c = 0; c < nch; ++c, ++it) {
          const int st = (int)(it % NST);
          if (!wait_bar(empty(st), ((it / NST) & 1u) ^ 1u, abort_flag, err, 1)) { alive = false; break; }
          bar_expect_tx(full(st), A_STAGE + B_STAGE);
          bulk_g2s(sbase + SL::a_off + st * A_STAGE, P + ((size_t)b * nch + c) * A_STAGE, A_STAGE, full(st));
          bulk_g2s(sbase + SL::b_off + st * B_STAGE, sdig + ((size_t)nt * nch + c) * B_STAGE, B_STAGE, full(st));
        }
        if (!alive) break;
      }
      // drain: wait for the copies still in flight before the CTA exits
      const uint32_t first = it > (uint32_t)NST ? it - NST : 0u;
      for (uint32_t k = first; k < it; ++k) {
        const int st = (int)(k % NST);
        uint32_t i = 0;
        while (!try_wait(full(st), (k / NST) & 1u) && ++i < kWaitLimit) {}
      }
    }
  } else if (warp == MMA_WARP) {
    // ---- MMA issuer ----
    if (lane == 0) {
      uint32_t idn[5];
#pragma unroll
      for (int c = 1; c <= 4; ++c) idn[c] = idesc_n(64u * c);
      uint32_t it = 0, ti = 0;
      bool alive = true, issued = false;
      for (int64_t t = blockIdx.x; t < ntiles && alive; t += gridDim.x, ++ti) {
        if (!wait_bar(acce, (ti & 1u) ^ 1u, abort_flag, err, 2)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int c = 0; c < nch; ++c, ++it) {
          const int st = (int)(it % NST);
          const uint32_t par = (it / NST) & 1u;
          if (!wait_bar(full(st), par, abort_flag, err, 3)) {
            alive = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = sbase + SL::a_off + st * A_STAGE, b0 = sbase + SL::b_off + st * B_STAGE;
#pragma unroll
          for (int s = 0; s < NSL; ++s) {
#pragma unroll
            for (int t0 = 0; t0 < NSL; t0 += 4) {
              if (s + t0 < NSL) {
                const int cnt = (NSL - s - t0) < 4 ? (NSL - s - t0) : 4;
                mma_f16(tbase + (uint32_t)(BNP * (s + t0)), sdesc(a0 + s * A_PLANE), sdesc(b0 + t0 * B_PLANE),
                        idn[cnt], (c == 0 && s == 0) ? 0u : 1u);
              }
            }
          }
          issued = true;
          mma_commit(empty(st));
        }
        if (!alive) break;
        mma_commit(accf);
      }
      if (issued) {   // every MMA of this thread has completed before TMEM is released
        mma_commit(drain);
        uint32_t i = 0;
        while (!try_wait(drain, 0u) && ++i < kWaitLimit) {}
      }
    }
  } else {
    // ---- epilogue ----
    // Phase 1 (TMEM held): group sums -> the exact W = sum_g C_g 2^(7 (7 - g)) = Vp 2^14 + r (C_0, C_1 < 2^22
    // by magic-number addition, C_2 .. C_7 < 2^24 by conversion; pairs C_g 2^7 + C_(g+1)
    // < 2^31 in int32, then 64-bit) staged in shared memory; then TMEM goes to the next tile's MMAs.
    // Phase 2: FP64 rounding and stores.
    const int q = warp & 3;                   // TMEM lane quadrant of this warp
    constexpr int EC = 4 * BNP / NE;          // tile columns per epilogue warp (32 or 16)
    constexpr int TSW = EC * 32 * 10;         // its staging bytes
    const int cq = (warp - EPI0) >> 2;        // columns [EC cq, EC cq + EC) of the tile
    long long* tsv = reinterpret_cast<long long*>(sm + SL::ts_off + (warp - EPI0) * TSW);   // [column][lane]
    uint16_t* tsr = reinterpret_cast<uint16_t*>(sm + SL::ts_off + (warp - EPI0) * TSW + EC * 32 * 8);
    uint32_t ti = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++ti) {
      const int64_t b = t / ntn;
      const int nt = (int)(t % ntn);
      bool ok = true;
      if (lane == 0) ok = wait_bar(accf, ti & 1u, abort_flag, err, 5);
      if (__shfl_sync(0xffffffffu, ok ? 1 : 0, 0) == 0) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t tl = tbase + ((uint32_t)(32 * q) << 16);
#pragma unroll 1
      for (int cb = 0; cb < EC / 8; ++cb) {   // 8 columns at a time
        const uint32_t col = (uint32_t)(EC * cq + 8 * cb);
        uint32_t v[NSL][8];   // all eight group sums of 8 columns, one wait
#pragma unroll
        for (int g = 0; g < NSL; ++g) tmem_ld8(tl + (uint32_t)(BNP * g) + col, v[g]);
        tmem_wait_ld();
        uint32_t tp[4][8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint32_t b0 = __float_as_uint(__uint_as_float(v[0][c]) + 12582912.0f);
          const uint32_t b1 = __float_as_uint(__uint_as_float(v[1][c]) + 12582912.0f);
          tp[0][c] = b0 * 128u + b1 - 129u * 0x4b400000u;
#pragma unroll
          for (int g = 2; g < NSL; g += 2)
            tp[g >> 1][c] = (uint32_t)(__float2int_rn(__uint_as_float(v[g][c])) * 128 +
                                       __float2int_rn(__uint_as_float(v[g + 1][c])));
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int t67 = (int)tp[3][c];
          const long long V = (((long long)(int)tp[0][c] << 14) + (int)tp[1][c]) * 16384ll + (int)tp[2][c];
          tsv[(8 * cb + c) * 32 + lane] = V + (long long)(t67 >> 14);   // floor division: remainder below
          tsr[(8 * cb + c) * 32 + lane] = (uint16_t)((uint32_t)t67 & 0x3fffu);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) bar_arrive(acce);
      const int64_t L = b * BM + 32 * q + lane;
      const int Er = L < nlines ? lineE[L] : kZeroExp;
      const int e0 = Er - 1084 + out_exp;
      int64_t obase = 0;
      if (L < nlines) obase = ROWS ? L * n : (L / inner) * n * inner + (L % inner);
      const int64_t ostride = ROWS ? 1 : inner;
      const int k0 = nt * BNP + EC * cq;   // frequency of column 0 of this warp
#pragma unroll 4
      for (int c = 0; c < EC; ++c) {
        const long long Vp = tsv[c * 32 + lane];
        const uint32_t r = tsr[c * 32 + lane];
        bool slow;
        double y = assemble_vr(Vp, r, e0, slow);
        if (slow || Er >= 2047)
          y = Er >= 2047 ? __longlong_as_double(0x7ff8000000000000ll)
                         : assemble128(((__int128)Vp << 14) + (__int128)r, e0);
        const int k = k0 + c;
        if (L < nlines && k >= 1 && k <= n) out[obase + (int64_t)(k - 1) * ostride] = y;
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tbase));
}

}  // namespace stmg_tc
