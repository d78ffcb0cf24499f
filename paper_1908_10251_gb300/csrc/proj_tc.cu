// Float64-accurate coarse projections on the 5th-generation tensor cores
// (tcgen05, sm_103a): b' = Q^T b, c' = Q^T c for all pairs (the only dense
// contraction of a correction step) and u_H = Q g.
//
// tcgen05 has no float64 kind, so the product is emulated exactly in digit
// planes (error-free slicing, Ozaki, Ogita, Oishi and Rump 2012):
//   A[i][j] = 2^ea_i * sum_s 2^(-7 (s+1)) A_s[i][j] + (|.| < 2^(ea_i - 56)),
//   B[j][n] = 2^eb_n * sum_t 2^(-7 (t+1)) B_t[j][n] + (|.| < 2^(eb_n - 56)),
// s, t = 0..7, with integer digits |A_s|, |B_t| <= 127 (exact in bf16): the
// base-128 digits of floor(|x| 2^56), x = A / 2^ea or B / 2^eb, carrying the
// sign of x.  Each digit product A_s B_t over a chunk of 32 inner indices is a
// bf16 x bf16 -> f32 tcgen05 MMA with integer entries; all products of one
// weight 2^(-7 d) (d = s + t + 2 <= 9; lighter ones lie below the slicing
// error) share one TMEM accumulator, whose sum stays below 8 * 32 * 127^2 <
// 2^24, so float32 holds it exactly.  The accumulators are folded exactly into
// two int64 sums per output, H (d <= 5) and L (d >= 6), value =
// (H 2^28 + L) 2^(ea_i + eb_n - 63), and added across the inner-dimension
// chunks with integer atomics (exact, so the result does not depend on their
// order).  The last CTA of an output tile rounds once to float64, writes the
// tile and clears the sums for the next call.  The result differs from the
// exact product by about 2^-56 K max|A_i.| max|B_.n|, i.e. it is as accurate
// as a float64 dot product.
//
// GB300 runs float64 at 1/64 of the float32 rate, so everything around the
// MMAs is integer work: B's exponents come from its bit fields, its digits from
// shifts of its significands.  Grid: (16-column tiles) x (128-row tiles) x
// (32-wide chunks of the inner dimension); 128 threads, one per TMEM lane /
// output row.  A's digit planes are split once at setup, stored in the
// canonical K-major no-swizzle operand layout, and the chunk's planes are
// brought into shared memory by bulk asynchronous copies (cp.async.bulk,
// completion on an mbarrier) while the threads form B's digit planes.  One
// elected thread issues the MMAs.  Every wait is bounded: on a timeout the CTA
// counts an error, waits (bounded) for what it has in flight and adds nothing.
#include "common.cuh"
#include "kernels.cuh"

#include <cmath>
#include <cstring>

namespace pasm {
namespace {

constexpr int kM = 128;          // rows per tile (TMEM lanes)
constexpr int kN = 16;           // output columns per tile (MMA N)
constexpr int kKC = 32;          // inner-dimension chunk per CTA
constexpr int kThreads = 128;
constexpr int kDigitBits = 7, kDigits = 8;   // 56 bits per operand
constexpr int kGroups = kDigits;             // weights d = 2 .. S + 1
constexpr uint32_t kTmemCols = 128;          // kGroups x kN
constexpr int kAPlaneBytes = (kKC / 8) * 2048;           // one digit plane of a 128 x 32 A chunk
constexpr int kBPlaneBytes = (kKC / 8) * (kN / 8) * 128;  // one digit plane of a 16 x 32 B chunk
constexpr int kSmem = kDigits * (kAPlaneBytes + kBPlaneBytes) + 1024;
constexpr int kWaitLimit = 1 << 22;
static_assert(kGroups * kN <= (int)kTmemCols, "accumulators must fit in TMEM");
static_assert((uint64_t)kGroups * kKC * 127 * 127 < (1u << 24), "group sums must be exact in float32");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// element (row, k) at (row % 8) * 16 + (row / 8) * SBO + (k / 8) * LBO + (k % 8) * 2 bytes.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Bounded wait for phase `parity` of an mbarrier (at most `limit` polls); true when it completed.
__device__ __forceinline__ bool wait_parity(uint32_t mbar, uint32_t parity, int limit) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
  }
  return done != 0;
}

// bf16 bit pattern of a small integer (|q| <= 255 is exact in bf16, so the
// upper half of its float32 encoding is the bf16 encoding).
__device__ __forceinline__ uint32_t bf16_bits_of_int(int q) { return __float_as_uint((float)q) >> 16; }

// Column n (< ncols) of the two stacked K x ldk inputs.
__device__ __forceinline__ const double* bcol(const double* B0, const double* B1, int ldk, int n) {
  return n < ldk ? B0 + n : B1 + (n - ldk);
}

__device__ __forceinline__ uint64_t ld_bits(const double* p) { return (uint64_t)__double_as_longlong(__ldg(p)); }

__device__ __forceinline__ void red_add(unsigned long long* p, long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"((unsigned long long)v) : "memory");
}

// Exponent e with |v| < 2^e for a finite nonzero v, from its bit fields.
__device__ __forceinline__ int bound_exponent(uint64_t bits) {
  const int ex = (int)((bits >> 52) & 0x7FF);
  return (ex > 0 ? ex : 1) - 1022;
}

// floor(|v| / 2^e * 2^T) for |v| < 2^e, T <= 62, from the significand of v.
__device__ __forceinline__ uint64_t scaled_magnitude(uint64_t bits, int e, int T) {
  const int ex = (int)((bits >> 52) & 0x7FF);
  const uint64_t mant = (bits & ((1ull << 52) - 1)) | (ex > 0 ? (1ull << 52) : 0ull);
  const int sh = (ex > 0 ? ex : 1) - 1075 - e + T;  // |v| = mant 2^(ex - 1075)
  if (sh >= 0) return mant << sh;
  return -sh < 64 ? (mant >> -sh) : 0ull;
}

// Round a signed 128-bit integer to float64 (to nearest, once) times 2^k.
__device__ __forceinline__ double i128_to_double_scaled(__int128 a, int k) {
  if (a == 0) return 0.0;
  const bool neg = a < 0;
  const unsigned __int128 u = neg ? (unsigned __int128)(-a) : (unsigned __int128)a;
  const uint64_t hi = (uint64_t)(u >> 64);
  double d;
  if (hi == 0) {
    d = (double)(uint64_t)u;
  } else {
    const int drop = 64 - __clzll((long long)hi);              // bits below the top 64
    const unsigned __int128 lowmask = (((unsigned __int128)1) << drop) - 1;
    uint64_t top = (uint64_t)(u >> drop);
    if ((u & lowmask) != 0) top |= 1ull;                       // sticky bit keeps the rounding exact
    d = (double)top;
    k += drop;
  }
  d = ldexp(d, k);
  return neg ? -d : d;
}

// Digit products A_s B_t (0-based digits) of weight 2^(-7 (s + t + 2)) with
// s + t + 2 <= S + 1, ordered by weight; products of one weight d share the
// accumulator of group d - 2.
struct DigitPlan {
  static constexpr int npairs = kDigits * (kDigits + 1) / 2;
  int s[npairs] = {}, t[npairs] = {}, first[npairs] = {};
  constexpr DigitPlan() {
    int p = 0;
    for (int d = 2; d <= kDigits + 1; ++d)
      for (int ss = 0; ss + 1 < d; ++ss) {
        s[p] = ss;
        t[p] = d - 2 - ss;
        first[p] = ss == 0 ? 1 : 0;
        ++p;
      }
  }
};

__global__ void __launch_bounds__(kThreads)
    k_proj_tc(int m, int K, int Kpad, const uint16_t* __restrict__ planes, const int* __restrict__ rexp,
              const double* __restrict__ B0, const double* __restrict__ B1, double* __restrict__ C0,
              double* __restrict__ C1, int ldk, int ncols, unsigned long long* __restrict__ hl,
              unsigned int* __restrict__ tickets, int* __restrict__ err, int wait_limit, int skip_mma) {
  constexpr DigitPlan P{};
  constexpr int S = kDigits, T = kDigitBits * kDigits;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;                                          // S x [4 kc8][16 row groups][8][8] bf16
  uint8_t* sB = smem + S * kAPlaneBytes;                       // S x [4 kc8][2 col groups][8][8] bf16
  int* cexp = reinterpret_cast<int*>(sB + S * kBPlaneBytes);  // [kN]
  int* cbad = cexp + kN;                                       // [kN]
  int* red = cbad + kN;                                        // [kThreads]
  int* flag = red + kThreads;                                  // [0] a wait gave up, [1] CTA finishes the tile
  uint64_t* mbar = reinterpret_cast<uint64_t*>(flag + 2);      // [0] copies, [1] MMAs
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * kN, mt = blockIdx.y, ch = blockIdx.z;
  const int kc0 = ch * kKC, kw = min(kKC, Kpad - kc0);
  const uint32_t bar_load = smem_u32(mbar), bar_mma = smem_u32(mbar + 1);

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_load));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_mma));
    asm volatile("fence.mbarrier_init.release.cluster;");
    flag[0] = 0;
    flag[1] = 0;
    // this chunk of A's digit planes: one bulk copy per plane
    const uint32_t bytes = (uint32_t)(S * (kw / 8) * 2048);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_load), "r"(bytes) : "memory");
    for (int s = 0; s < S; ++s) {
      const uint16_t* src = planes + ((size_t)(mt * S + s) * (Kpad / 8) + kc0 / 8) * 1024;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(sA + s * kAPlaneBytes)),
          "l"(src), "r"((uint32_t)((kw / 8) * 2048)), "r"(bar_load)
          : "memory");
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // column exponents over the whole inner dimension, from the bit fields:
  // |B[j][n]| < 2^cexp[n]; a NaN/Inf marks the column.  Loads use clamped
  // indices (always valid addresses) so that each batch is issued at once.
  {
    const int col = tid % kN, part = tid / kN;
    constexpr int kParts = kThreads / kN;
    const bool cv = n0 + col < ncols;
    const double* cp = bcol(B0, B1, ldk, cv ? n0 + col : 0);
    int emax = -100000;
    bool bad = false;
    for (int j0 = part; j0 < K; j0 += 8 * kParts) {
      uint64_t bits[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) bits[q] = ld_bits(cp + (size_t)min(j0 + q * kParts, K - 1) * ldk);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (!cv || j0 + q * kParts >= K) continue;
        if (((bits[q] >> 52) & 0x7FF) == 0x7FF) bad = true;
        else if ((bits[q] << 1) != 0) emax = max(emax, bound_exponent(bits[q]));
      }
    }
    red[tid] = bad ? 0x7FFFFFFF : emax;
  }
  __syncthreads();
  if (tid < kN) {
    int emax = -100000;
    bool bad = false;
    for (int p = 0; p < kThreads / kN; ++p) {
      const int v = red[p * kN + tid];
      if (v == 0x7FFFFFFF) bad = true;
      else emax = max(emax, v);
    }
    cexp[tid] = (bad || emax == -100000) ? 0 : emax;
    cbad[tid] = bad ? 1 : 0;
  }
  __syncthreads();
  // B's digit planes for this chunk: item (kc8, n) slices 8 consecutive entries of column n
  const uint64_t dmask = (1ull << kDigitBits) - 1;
  for (int it = tid; it < (kw / 8) * kN; it += kThreads) {
    const int n = it % kN, kc8 = it / kN;
    const int e = cexp[n];
    const bool cv = n0 + n < ncols && !cbad[n];
    const double* cp = bcol(B0, B1, ldk, n0 + n < ncols ? n0 + n : 0);
    uint64_t raw[8], mag[8];
    uint32_t neg = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) raw[q] = ld_bits(cp + (size_t)min(kc0 + kc8 * 8 + q, K - 1) * ldk);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint64_t bits = (cv && kc0 + kc8 * 8 + q < K) ? raw[q] : 0ull;
      mag[q] = (bits << 1) ? scaled_magnitude(bits, e, T) : 0ull;
      neg |= (uint32_t)(bits >> 63) << q;
    }
    const int off = kc8 * (kN / 8) * 128 + (n / 8) * 128 + (n % 8) * 16;
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const int sh = T - kDigitBits * (t + 1);
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        int d0 = (int)((mag[q] >> sh) & dmask), d1 = (int)((mag[q + 1] >> sh) & dmask);
        if (neg >> q & 1u) d0 = -d0;
        if (neg >> (q + 1) & 1u) d1 = -d1;
        w[q / 2] = bf16_bits_of_int(d0) | (bf16_bits_of_int(d1) << 16);
      }
      *reinterpret_cast<uint4*>(sB + t * kBPlaneBytes + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    bool ok = wait_parity(bar_load, 0, wait_limit);
    // skip_mma (a test of the timeout path): no MMA is issued and nothing arrives on bar_mma, so
    // its wait runs out with nothing in flight
    if (ok && skip_mma) {
      ok = wait_parity(bar_mma, 0, wait_limit);
    } else if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t idesc =
          (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      constexpr uint32_t bsb = (uint32_t)((kN / 8) * 128);
#pragma unroll
      for (int kk = 0; kk < kKC / 16; ++kk) {
        if (kk * 16 >= kw) break;
        const uint64_t ad = sdesc(a0 + (uint32_t)(kk * 2 * 2048), 2048, 128);
        const uint64_t bd = sdesc(b0 + (uint32_t)(kk * 2 * bsb), bsb, 128);
#pragma unroll
        for (int p = 0; p < P.npairs; ++p) {
          const uint32_t acc = (kk == 0 && P.first[p]) ? 0u : 1u;
          mma_bf16(tmem + (uint32_t)((P.s[p] + P.t[p]) * kN), ad + (uint64_t)((P.s[p] * kAPlaneBytes) >> 4),
                   bd + (uint64_t)((P.t[p] * kBPlaneBytes) >> 4), idesc, acc);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_mma));
      ok = wait_parity(bar_mma, 0, wait_limit);
      if (!ok) wait_parity(bar_mma, 0, kWaitLimit);  // MMAs still reading shared memory
    } else {
      wait_parity(bar_load, 0, kWaitLimit);  // copies still in flight
    }
    if (!ok) {
      atomicAdd(err, 1);
      flag[0] = 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const int i = mt * kM + warp * 32 + lane;
  if (!flag[0]) {
    // fold the weight groups of this row exactly: H (d <= 5), L (d >= 6)
    long long H[kN], L[kN];
#pragma unroll
    for (int n = 0; n < kN; ++n) H[n] = L[n] = 0;
    const uint32_t lanebase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
      float v[16];
      tmem_ld16(lanebase + (uint32_t)(g * kN), v);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      const int d = g + 2;
#pragma unroll
      for (int n = 0; n < kN; ++n) {
        const long long x = (long long)__float2int_rn(v[n]);
        if (d <= 5) H[n] += x << (kDigitBits * (5 - d));
        else L[n] += x << (kDigitBits * (9 - d));
      }
    }
    if (i < m) {
#pragma unroll
      for (int n = 0; n < kN; ++n) {
        const int col = n0 + n;
        if (col >= ncols) continue;
        unsigned long long* q = hl + ((size_t)i * ncols + col) * 2;
        red_add(q, H[n]);
        red_add(q + 1, L[n]);
      }
    }
  }
  // the last CTA of this output tile rounds, writes and clears
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned int prev = atomicAdd(&tickets[blockIdx.y * gridDim.x + blockIdx.x], 1u);
    flag[1] = prev == gridDim.z - 1 ? 1 : 0;
  }
  __syncthreads();
  if (flag[1]) {
    __threadfence();
    if (i < m) {
      const int kbase = rexp[i] - kDigitBits * (S + 1);
      unsigned long long* row = hl + (size_t)i * ncols * 2;
      long long h[kN], l[kN];
#pragma unroll
      for (int n = 0; n < kN; ++n) {
        const int col = min(n0 + n, ncols - 1);
        h[n] = (long long)__ldcg(row + col * 2);
        l[n] = (long long)__ldcg(row + col * 2 + 1);
      }
#pragma unroll
      for (int n = 0; n < kN; ++n) {
        const int col = n0 + n;
        if (col >= ncols) continue;
        row[col * 2] = 0ull;
        row[col * 2 + 1] = 0ull;
        const double r = cbad[n] ? __longlong_as_double(0x7ff8000000000000LL)
                                 : i128_to_double_scaled(((__int128)h[n] << 28) + (__int128)l[n], kbase + cexp[n]);
        if (col < ldk) C0[(size_t)i * ldk + col] = r;
        else C1[(size_t)i * ldk + (col - ldk)] = r;
      }
    }
    if (tid == 0) tickets[blockIdx.y * gridDim.x + blockIdx.x] = 0u;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

bool proj_plan(int K, ProjPlan& p) {
  p = ProjPlan{};
  if (K < 1 || K > (1 << 22)) return false;  // keeps the int64 sums over all chunks exact
  p.beta = kDigitBits;
  p.S = kDigits;
  return true;
}

void proj_split_host(const double* A, int m, int K, const ProjPlan& plan, int& Kpad, int& mtiles,
                     std::vector<uint16_t>& planes, std::vector<int>& rexp) {
  Kpad = (K + 15) / 16 * 16;
  mtiles = (m + kM - 1) / kM;
  const int S = plan.S, kc8n = Kpad / 8;
  planes.assign((size_t)mtiles * S * kc8n * 1024, 0);
  rexp.assign((size_t)m, 0);
  const double two_beta = std::ldexp(1.0, plan.beta);
  for (int i = 0; i < m; ++i) {
    double mx = 0.0;
    for (int j = 0; j < K; ++j) mx = std::fmax(mx, std::fabs(A[(size_t)i * K + j]));
    int e = 0;
    if (mx > 0.0) std::frexp(mx, &e);
    rexp[(size_t)i] = e;
    const int mt = i / kM, rg = (i % kM) / 8, r8 = i % 8;
    for (int j = 0; j < K; ++j) {
      double x = std::ldexp(A[(size_t)i * K + j], -e);
      for (int s = 0; s < S; ++s) {
        const double y = x * two_beta;
        const double q = std::trunc(y);
        x = y - q;
        const float qf = (float)q;
        uint32_t bits;
        std::memcpy(&bits, &qf, 4);
        const size_t off = ((((size_t)(mt * S + s) * kc8n + j / 8) * 16 + rg) * 8 + r8) * 8 + j % 8;
        planes[off] = (uint16_t)(bits >> 16);
      }
    }
  }
}

size_t proj_scratch_words(int m, int ncols_max) { return (size_t)m * ncols_max * 2; }
size_t proj_tickets(int m, int ncols_max) { return (size_t)((m + kM - 1) / kM) * ((ncols_max + kN - 1) / kN); }

cudaError_t proj_tc_prepare() { return allow_dynamic_smem((const void*)k_proj_tc, (size_t)kSmem); }

void proj_tc(const Launch& L, const SplitMat& A, const double* B0, const double* B1, double* C0, double* C1,
             int ldk, int ncols, unsigned long long* hl, unsigned int* tickets, int* err, int wait_limit,
             int skip_mma) {
  dim3 grid((ncols + kN - 1) / kN, A.mtiles, (A.Kpad + kKC - 1) / kKC);
  const double m = A.m, K = A.K, n = ncols;
  L.begin(KC_PROJ, (m * K + K * n + m * n) * 8.0, 2.0 * m * K * n);
  k_proj_tc<<<grid, kThreads, kSmem, L.s>>>(A.m, A.K, A.Kpad, A.planes, A.rexp, B0, B1, C0, C1, ldk, ncols, hl,
                                            tickets, err, wait_limit > 0 ? wait_limit : kWaitLimit, skip_mma);
  L.bump();
}

}  // namespace pasm
