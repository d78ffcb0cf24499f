// Float64-accuracy kernels of the mixed-precision path in double-float
// arithmetic (ff.cuh): the outer residuals of the defect correction
// (Algorithm 1 step 1), the bordering products (the bordered matrix form of
// Section 3.1), the transfer chains and the update.  Vectors that are gathered
// through a sparse matrix are kept as (hi, lo) float pairs ("ff", 8 bytes per
// entry like float64): the multigrid iterate u~, its products A u~ and M u~,
// the intermediate levels of the transfer chains, and the state U itself
// between steps (its float64 form is rebuilt when read).  Matrix values are
// split once at setup; a matrix whose values are all float32 skips the
// low-part products.  The coarse vectors and the eigenvalues stay float64.
// Results carry about 2^-46 relative to the sum of the magnitudes of their
// terms (float64: 2^-53), far below what the float32 V-cycles of the mixed
// path resolve.
#include "common.cuh"
#include "ff.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace pasm {
namespace {

constexpr int kBlock = 256;
// The residual and transfer kernels are held to 64 registers (four 256-thread
// blocks per SM): the extra warps hide more gather latency than the few
// spilled values cost (outer_rhs 0.64 -> 0.59 ms, outer_res 0.34 -> 0.28,
// spmm 0.52 -> 0.48 at h = 1/1024, k = 64).  The bordering and update kernels
// were slower that way and keep the compiler's choice.
constexpr int kMinBlocksGather = 4;

struct Geo {
  int tpr, ch;
};
// Row groups as in the float64 kernels: 16-byte chunks of 2 columns; pref as
// in the float64 geometry (chunks per thread chosen by the autotuner).
Geo geometry_ff(int ldk, int pref) {
  const int chunks = ldk / 2;
  Geo g;
  if (chunks <= 32) { g.tpr = chunks; g.ch = 1; }
  else { g.tpr = 32; g.ch = chunks / 32; }
  if ((pref == 1 || pref == 2 || pref == 4 || pref == 8) && chunks % pref == 0 && chunks / pref <= 32) {
    g.tpr = chunks / pref;
    g.ch = pref;
  }
  return g;
}

// Row blocks one thread block walks (1 or 4, chosen by the autotuner; 1 when untuned).
static int ff_rows(const Launch& L) { return L.rpt > 0 ? L.rpt : 1; }

#define PASM_FF_DISPATCH(ch, ...)                          \
  switch (ch) {                                            \
    case 1: { constexpr int CH = 1; __VA_ARGS__; } break;  \
    case 2: { constexpr int CH = 2; __VA_ARGS__; } break;  \
    case 4: { constexpr int CH = 4; __VA_ARGS__; } break;  \
    case 8: { constexpr int CH = 8; __VA_ARGS__; } break;  \
    default: break;                                        \
  }

// Two consecutive entries (columns col, col + 1) of row i of a block vector,
// as (hi, lo) pairs: from float pairs directly, from float64 by splitting.
template <bool FF>
__device__ __forceinline__ void load_pair(const double* __restrict__ X, size_t off, float (&h)[2], float (&l)[2]) {
  if (FF) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(X + off));
    h[0] = t.x; l[0] = t.y; h[1] = t.z; l[1] = t.w;
  } else {
    const double2 t = __ldg(reinterpret_cast<const double2*>(X + off));
    ff_split(t.x, h[0], l[0]);
    ff_split(t.y, h[1], l[1]);
  }
}

// acc += a_p X[ci_p, cols] for the N entries p .. p+N-1: index and value loads,
// then the N row gathers, then the double-float products.
template <int CH, int N, bool FFIN, bool EX>
__device__ __forceinline__ void gather_group_ff(const int* __restrict__ ci, const float2* __restrict__ av,
                                                const double* __restrict__ X, int p, int lane, int tpr, int ldk,
                                                float (&hi)[CH][2], float (&lo)[CH][2]) {
  int j[N];
  float2 a[N];
#pragma unroll
  for (int u = 0; u < N; ++u) {
    j[u] = __ldg(ci + p + u);
    a[u] = __ldg(av + p + u);
  }
  float xh[N][CH][2], xl[N][CH][2];
#pragma unroll
  for (int u = 0; u < N; ++u)
#pragma unroll
    for (int c = 0; c < CH; ++c) load_pair<FFIN>(X, (size_t)j[u] * ldk + (c * tpr + lane) * 2, xh[u][c], xl[u][c]);
#pragma unroll
  for (int u = 0; u < N; ++u)
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        if (EX) ff_mac_exact(hi[c][v], lo[c][v], a[u].x, xh[u][c][v], xl[u][c][v]);
        else ff_mac(hi[c][v], lo[c][v], a[u].x, a[u].y, xh[u][c][v], xl[u][c][v]);
      }
}

// One row of S X in double-float (groups of 4 entries, then an exact remainder group);
// EX: S's values are float32 (no low parts).
template <int CH, bool FFIN, bool EX = false>
__device__ __forceinline__ void gather_row_ff(const int* __restrict__ rp, const int* __restrict__ ci,
                                              const float2* __restrict__ av, const double* __restrict__ X, int row,
                                              int lane, int tpr, int ldk, float (&hi)[CH][2], float (&lo)[CH][2]) {
#pragma unroll
  for (int c = 0; c < CH; ++c) hi[c][0] = hi[c][1] = lo[c][0] = lo[c][1] = 0.f;
  int p = __ldg(rp + row);
  const int p1 = __ldg(rp + row + 1);
  for (; p + 4 <= p1; p += 4) gather_group_ff<CH, 4, FFIN, EX>(ci, av, X, p, lane, tpr, ldk, hi, lo);
  const int rem = p1 - p;
  if (rem == 3) gather_group_ff<CH, 3, FFIN, EX>(ci, av, X, p, lane, tpr, ldk, hi, lo);
  else if (rem == 2) gather_group_ff<CH, 2, FFIN, EX>(ci, av, X, p, lane, tpr, ldk, hi, lo);
  else if (rem == 1) gather_group_ff<CH, 1, FFIN, EX>(ci, av, X, p, lane, tpr, ldk, hi, lo);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    ff_norm(hi[c][0], lo[c][0]);
    ff_norm(hi[c][1], lo[c][1]);
  }
}

// A X and M X together over M's pattern (am: A's and M's split values per
// entry, a = 0 where A has no entry): one gather of each row of X serves both
// products.  Each accumulator sees the same terms in the same order as the
// separate gathers (A's entries in M's column order).
template <int CH, int N, bool FFIN, bool AEX>
__device__ __forceinline__ void gather_group_am(const int* __restrict__ ci, const float4* __restrict__ am,
                                                const double* __restrict__ X, int p, int lane, int tpr, int ldk,
                                                float (&ah)[CH][2], float (&al)[CH][2], float (&mh)[CH][2],
                                                float (&ml)[CH][2]) {
  int j[N];
  float4 w[N];
#pragma unroll
  for (int u = 0; u < N; ++u) {
    j[u] = __ldg(ci + p + u);
    w[u] = __ldg(am + p + u);
  }
  float xh[N][CH][2], xl[N][CH][2];
#pragma unroll
  for (int u = 0; u < N; ++u)
#pragma unroll
    for (int c = 0; c < CH; ++c) load_pair<FFIN>(X, (size_t)j[u] * ldk + (c * tpr + lane) * 2, xh[u][c], xl[u][c]);
#pragma unroll
  for (int u = 0; u < N; ++u) {
    const bool has_a = w[u].x != 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        ff_mac(mh[c][v], ml[c][v], w[u].z, w[u].w, xh[u][c][v], xl[u][c][v]);
        if (has_a) {
          if (AEX) ff_mac_exact(ah[c][v], al[c][v], w[u].x, xh[u][c][v], xl[u][c][v]);
          else ff_mac(ah[c][v], al[c][v], w[u].x, w[u].y, xh[u][c][v], xl[u][c][v]);
        }
      }
  }
}

template <int CH, bool FFIN, bool AEX>
__device__ __forceinline__ void gather_row_am(const int* __restrict__ rp, const int* __restrict__ ci,
                                              const float4* __restrict__ am, const double* __restrict__ X, int row,
                                              int lane, int tpr, int ldk, float (&ah)[CH][2], float (&al)[CH][2],
                                              float (&mh)[CH][2], float (&ml)[CH][2]) {
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < 2; ++v) ah[c][v] = al[c][v] = mh[c][v] = ml[c][v] = 0.f;
  int p = __ldg(rp + row);
  const int p1 = __ldg(rp + row + 1);
  for (; p + 4 <= p1; p += 4) gather_group_am<CH, 4, FFIN, AEX>(ci, am, X, p, lane, tpr, ldk, ah, al, mh, ml);
  const int rem = p1 - p;
  if (rem == 3) gather_group_am<CH, 3, FFIN, AEX>(ci, am, X, p, lane, tpr, ldk, ah, al, mh, ml);
  else if (rem == 2) gather_group_am<CH, 2, FFIN, AEX>(ci, am, X, p, lane, tpr, ldk, ah, al, mh, ml);
  else if (rem == 1) gather_group_am<CH, 1, FFIN, AEX>(ci, am, X, p, lane, tpr, ldk, ah, al, mh, ml);
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      ff_norm(ah[c][v], al[c][v]);
      ff_norm(mh[c][v], ml[c][v]);
    }
}

// Store two entries as float pairs or, rounded, as float64.
template <bool FF>
__device__ __forceinline__ void store_pair(double* __restrict__ out, size_t off, const float (&h)[2],
                                           const float (&l)[2]) {
  if (FF) *reinterpret_cast<float4*>(out + off) = make_float4(h[0], l[0], h[1], l[1]);
  else *reinterpret_cast<double2*>(out + off) = make_double2(ff_to_double(h[0], l[0]), ff_to_double(h[1], l[1]));
}

// Fd = lam .* (M U) stored as (hi, lo) float pairs, R = Fd - A U as float32
// (U given as float pairs).
template <int CH, bool AEX>
__global__ void __launch_bounds__(kBlock, kMinBlocksGather)
    k_outer_rhs_res_ff(int n, const int* __restrict__ arp, const int* __restrict__ aci, const float2* __restrict__ aval,
                       const int* __restrict__ mrp, const int* __restrict__ mci, const float2* __restrict__ mval,
                       const double* __restrict__ lam, const double* __restrict__ U, float2* __restrict__ Fd,
                       float* __restrict__ R, int ldk, int tpr, int rpt) {
  // the eigenvalues as (hi, lo) pairs, split once per block rather than once per entry
  extern __shared__ float2 lsp[];  // [ldk]
  for (int t = threadIdx.x; t < ldk; t += blockDim.x) ff_split(__ldg(lam + t), lsp[t].x, lsp[t].y);
  __syncthreads();
  const int rpb = kBlock / tpr;
  const int lane = threadIdx.x % tpr;
  for (int rr = 0; rr < rpt; ++rr) {
  const int row = (blockIdx.x * rpt + rr) * rpb + threadIdx.x / tpr;
  if (row >= n) return;
  float muh[CH][2], mul[CH][2], auh[CH][2], aul[CH][2];
  // two separate gathers: the one-gather form (as in the bordering kernel) needs more registers
  // than the four blocks per SM this kernel runs at, and was slower (0.57 -> 0.63 ms)
  gather_row_ff<CH, true>(mrp, mci, mval, U, row, lane, tpr, ldk, muh, mul);
  gather_row_ff<CH, true, AEX>(arp, aci, aval, U, row, lane, tpr, ldk, auh, aul);
  const size_t base = (size_t)row * ldk;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * tpr + lane) * 2;
    float f[2][2], r[2];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const float2 l = lsp[col + v];
      ff_mul(l.x, l.y, muh[c][v], mul[c][v], f[v][0], f[v][1]);
      r[v] = __fadd_rn(__fsub_rn(f[v][0], auh[c][v]), __fsub_rn(f[v][1], aul[c][v]));
    }
    *reinterpret_cast<float4*>(Fd + base + col) = make_float4(f[0][0], f[0][1], f[1][0], f[1][1]);
    *reinterpret_cast<float2*>(R + base + col) = make_float2(r[0], r[1]);
  }
  }
}

// R = Fd - A X as float32 (Fd and X as float pairs).
template <int CH, bool AEX>
__global__ void __launch_bounds__(kBlock, kMinBlocksGather)
    k_outer_res_ff(int n, const int* __restrict__ arp, const int* __restrict__ aci, const float2* __restrict__ aval,
                   const float2* __restrict__ Fd, const double* __restrict__ X, float* __restrict__ R, int ldk,
                   int tpr, int rpt) {
  const int rpb = kBlock / tpr;
  const int lane = threadIdx.x % tpr;
  for (int rr = 0; rr < rpt; ++rr) {
  const int row = (blockIdx.x * rpt + rr) * rpb + threadIdx.x / tpr;
  if (row >= n) return;
  float axh[CH][2], axl[CH][2];
  gather_row_ff<CH, true, AEX>(arp, aci, aval, X, row, lane, tpr, ldk, axh, axl);
  const size_t base = (size_t)row * ldk;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * tpr + lane) * 2;
    const float4 f = __ldg(reinterpret_cast<const float4*>(Fd + base + col));
    const float r0 = __fadd_rn(__fsub_rn(f.x, axh[c][0]), __fsub_rn(f.y, axl[c][0]));
    const float r1 = __fadd_rn(__fsub_rn(f.z, axh[c][1]), __fsub_rn(f.w, axl[c][1]));
    *reinterpret_cast<float2*>(R + base + col) = make_float2(r0, r1);
  }
  }
}

// YA = A X, YM = M X (X, YA, YM as float pairs) and per-block partial sums of
// X .* YA, X .* YM (double-float per thread, float64 across the block).
template <int CH, bool AEX, bool MERGED>
__global__ void __launch_bounds__(kBlock)
    k_border_ff(int n, const int* __restrict__ arp, const int* __restrict__ aci, const float2* __restrict__ aval,
                const int* __restrict__ mrp, const int* __restrict__ mci, const float2* __restrict__ mval,
                const double* __restrict__ X, double* __restrict__ YA, double* __restrict__ YM,
                double* __restrict__ partials, int ldk, int tpr, const float4* __restrict__ am) {
  extern __shared__ double red[];  // [rpb][2][ldk]
  const int rpb = kBlock / tpr;
  const int grp = threadIdx.x / tpr;
  const int lane = threadIdx.x % tpr;
  float sAh[CH][2], sAl[CH][2], sMh[CH][2], sMl[CH][2];
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < 2; ++v) sAh[c][v] = sAl[c][v] = sMh[c][v] = sMl[c][v] = 0.f;
  for (int row = blockIdx.x * rpb + grp; row < n; row += gridDim.x * rpb) {
    float yah[CH][2], yal[CH][2], ymh[CH][2], yml[CH][2];
    if (MERGED) {
      gather_row_am<CH, true, AEX>(mrp, mci, am, X, row, lane, tpr, ldk, yah, yal, ymh, yml);
    } else {
      gather_row_ff<CH, true, AEX>(arp, aci, aval, X, row, lane, tpr, ldk, yah, yal);
      gather_row_ff<CH, true>(mrp, mci, mval, X, row, lane, tpr, ldk, ymh, yml);
    }
    const size_t base = (size_t)row * ldk;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const size_t off = base + (c * tpr + lane) * 2;
      float xh[2], xl[2];
      load_pair<true>(X, off, xh, xl);
      store_pair<true>(YA, off, yah[c], yal[c]);
      store_pair<true>(YM, off, ymh[c], yml[c]);
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        ff_mac(sAh[c][v], sAl[c][v], xh[v], xl[v], yah[c][v], yal[c][v]);
        ff_mac(sMh[c][v], sMl[c][v], xh[v], xl[v], ymh[c][v], yml[c][v]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * tpr + lane) * 2;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      red[(grp * 2 + 0) * ldk + col + v] = ff_to_double(sAh[c][v], sAl[c][v]);
      red[(grp * 2 + 1) * ldk + col + v] = ff_to_double(sMh[c][v], sMl[c][v]);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * ldk; t += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < rpb; ++r) s += red[r * 2 * ldk + t];
    partials[(size_t)blockIdx.x * 2 * ldk + t] = s;
  }
}

// out = S X; FFIN / FFOUT: X / out as float pairs (else float64).
template <int CH, bool FFIN, bool FFOUT, bool EX>
__global__ void __launch_bounds__(kBlock, kMinBlocksGather) k_spmm_ff(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                     const float2* __restrict__ av, const double* __restrict__ X,
                                                     double* __restrict__ out, int ldk, int tpr, int rpt) {
  const int rpb = kBlock / tpr;
  const int lane = threadIdx.x % tpr;
  for (int rr = 0; rr < rpt; ++rr) {
  const int row = (blockIdx.x * rpt + rr) * rpb + threadIdx.x / tpr;
  if (row >= n) return;
  float yh[CH][2], yl[CH][2];
  gather_row_ff<CH, FFIN, EX>(rp, ci, av, X, row, lane, tpr, ldk, yh, yl);
  const size_t base = (size_t)row * ldk;
#pragma unroll
  for (int c = 0; c < CH; ++c) store_pair<FFOUT>(out, base + (c * tpr + lane) * 2, yh[c], yl[c]);
  }
}

// outA = S XA and outM = S XM together (the two restriction chains of the bordering products): one
// load of S's indices and values serves both; each product sees the same terms in the same order
// as two separate k_spmm_ff launches.
template <int CH, int N, bool FFIN, bool EX>
__device__ __forceinline__ void gather_group_ff2(const int* __restrict__ ci, const float2* __restrict__ av,
                                                 const double* __restrict__ XA, const double* __restrict__ XM,
                                                 int p, int lane, int tpr, int ldk, float (&ah)[CH][2],
                                                 float (&al)[CH][2], float (&mh)[CH][2], float (&ml)[CH][2]) {
  int j[N];
  float2 a[N];
#pragma unroll
  for (int u = 0; u < N; ++u) {
    j[u] = __ldg(ci + p + u);
    a[u] = __ldg(av + p + u);
  }
  float xh[N][CH][2], xl[N][CH][2], yh[N][CH][2], yl[N][CH][2];
#pragma unroll
  for (int u = 0; u < N; ++u)
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const size_t off = (size_t)j[u] * ldk + (c * tpr + lane) * 2;
      load_pair<FFIN>(XA, off, xh[u][c], xl[u][c]);
      load_pair<FFIN>(XM, off, yh[u][c], yl[u][c]);
    }
#pragma unroll
  for (int u = 0; u < N; ++u)
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        if (EX) {
          ff_mac_exact(ah[c][v], al[c][v], a[u].x, xh[u][c][v], xl[u][c][v]);
          ff_mac_exact(mh[c][v], ml[c][v], a[u].x, yh[u][c][v], yl[u][c][v]);
        } else {
          ff_mac(ah[c][v], al[c][v], a[u].x, a[u].y, xh[u][c][v], xl[u][c][v]);
          ff_mac(mh[c][v], ml[c][v], a[u].x, a[u].y, yh[u][c][v], yl[u][c][v]);
        }
      }
}

template <int CH, bool FFIN, bool FFOUT, bool EX>
__global__ void __launch_bounds__(kBlock, kMinBlocksGather) k_spmm2_ff(int n, const int* __restrict__ rp,
                                                                     const int* __restrict__ ci,
                                                                     const float2* __restrict__ av,
                                                                     const double* __restrict__ XA,
                                                                     const double* __restrict__ XM,
                                                                     double* __restrict__ outA,
                                                                     double* __restrict__ outM, int ldk, int tpr,
                                                                     int rpt) {
  const int rpb = kBlock / tpr;
  const int lane = threadIdx.x % tpr;
  for (int rr = 0; rr < rpt; ++rr) {
    const int row = (blockIdx.x * rpt + rr) * rpb + threadIdx.x / tpr;
    if (row >= n) return;
    float ah[CH][2], al[CH][2], mh[CH][2], ml[CH][2];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < 2; ++v) ah[c][v] = al[c][v] = mh[c][v] = ml[c][v] = 0.f;
    int p = __ldg(rp + row);
    const int p1 = __ldg(rp + row + 1);
    for (; p + 4 <= p1; p += 4) gather_group_ff2<CH, 4, FFIN, EX>(ci, av, XA, XM, p, lane, tpr, ldk, ah, al, mh, ml);
    const int rem = p1 - p;
    if (rem == 3) gather_group_ff2<CH, 3, FFIN, EX>(ci, av, XA, XM, p, lane, tpr, ldk, ah, al, mh, ml);
    else if (rem == 2) gather_group_ff2<CH, 2, FFIN, EX>(ci, av, XA, XM, p, lane, tpr, ldk, ah, al, mh, ml);
    else if (rem == 1) gather_group_ff2<CH, 1, FFIN, EX>(ci, av, XA, XM, p, lane, tpr, ldk, ah, al, mh, ml);
    const size_t base = (size_t)row * ldk;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        ff_norm(ah[c][v], al[c][v]);
        ff_norm(mh[c][v], ml[c][v]);
      }
      store_pair<FFOUT>(outA, base + (c * tpr + lane) * 2, ah[c], al[c]);
      store_pair<FFOUT>(outM, base + (c * tpr + lane) * 2, mh[c], ml[c]);
    }
  }
}

// X = B + E with E float32, X as float pairs; B as float pairs (may alias X)
// or float64.
template <bool BFF>
__global__ void k_axpy_ff(int64_t total, const double* B, const float* __restrict__ E, double* X) {
  const int64_t np = total / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    float bh[2], bl[2];
    load_pair<BFF>(B, 2 * i, bh, bl);
    const float2 e = __ldg(reinterpret_cast<const float2*>(E + 2 * i));
    const float ev[2] = {e.x, e.y};
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      float h = bh[v], l = bl[v];
      ff_mac(h, l, ev[v], 0.f, 1.f, 0.f);
      ff_norm(h, l);
      bh[v] = h;
      bl[v] = l;
    }
    store_pair<true>(X, 2 * i, bh, bl);
  }
}

// Elementwise format conversions of block vectors.
// in may equal out: each thread reads its two entries before writing them.
__global__ void k_to_ff(int64_t total, const double* in, double* out) {
  const int64_t np = total / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    float h[2], l[2];
    load_pair<false>(in, 2 * i, h, l);
    store_pair<true>(out, 2 * i, h, l);
  }
}
__global__ void k_from_ff(int64_t total, const double* __restrict__ in, double* __restrict__ out) {
  const int64_t np = total / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    float h[2], l[2];
    load_pair<true>(in, 2 * i, h, l);
    store_pair<false>(out, 2 * i, h, l);
  }
}

// U[row][c] = upd[c] ? alpha[c] X[row][c] + (P W)[row][c] : U[row][c], X as
// float pairs, W as float pairs (WFF) or float64; identity: P W = W.  Entries
// of frozen pairs are neither read nor written.  With U null the state is the
// pair array Usplit alone (the finest-level state of the mixed-precision step;
// its float64 copy is made on demand), else U is written in float64 and, if
// Usplit is given, also split into pairs.
template <int CH, bool WFF, bool EX>
__global__ void __launch_bounds__(kBlock)
    k_update_ff(int n, const int* __restrict__ rp, const int* __restrict__ ci, const float2* __restrict__ pv,
                const double* __restrict__ W, const double* __restrict__ X, const double* __restrict__ alpha,
                const int* __restrict__ upd, double* __restrict__ U, double* __restrict__ Usplit, int ldk, int tpr,
                int identity, int rpt) {
  extern __shared__ float2 asp[];  // [ldk]: alpha as (hi, lo) pairs, split once per block
  for (int t = threadIdx.x; t < ldk; t += blockDim.x) ff_split(__ldg(alpha + t), asp[t].x, asp[t].y);
  __syncthreads();
  const int rpb = kBlock / tpr;
  const int lane = threadIdx.x % tpr;
  for (int rr = 0; rr < rpt; ++rr) {
  const int row = (blockIdx.x * rpt + rr) * rpb + threadIdx.x / tpr;
  if (row >= n) return;
  float wh[CH][2], wl[CH][2];
  const size_t base = (size_t)row * ldk;
  if (identity) {
#pragma unroll
    for (int c = 0; c < CH; ++c) load_pair<WFF>(W, base + (c * tpr + lane) * 2, wh[c], wl[c]);
  } else {
    gather_row_ff<CH, WFF, EX>(rp, ci, pv, W, row, lane, tpr, ldk, wh, wl);
  }
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * tpr + lane) * 2;
    const size_t off = base + col;
    const int u0 = upd[col], u1 = upd[col + 1];
    if (!u0 && !u1) continue;  // both pairs frozen: U and its split copy stay as they are
    float xh[2], xl[2];
    load_pair<true>(X, off, xh, xl);
    float h[2], l[2];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const float2 a = asp[col + v];
      h[v] = wh[c][v];
      l[v] = wl[c][v];
      ff_mac(h[v], l[v], a.x, a.y, xh[v], xl[v]);
      ff_norm(h[v], l[v]);
    }
    if (!U) {  // the state lives in pairs only: write the updated pairs, keep the frozen one
      if (!(u0 && u1)) {
        float oh[2], ol[2];
        load_pair<true>(Usplit, off, oh, ol);
        if (!u0) { h[0] = oh[0]; l[0] = ol[0]; }
        if (!u1) { h[1] = oh[1]; l[1] = ol[1]; }
      }
      store_pair<true>(Usplit, off, h, l);
      continue;
    }
    double2 u;
    if (!(u0 && u1)) u = *reinterpret_cast<const double2*>(U + off);
    if (u0) u.x = ff_to_double(h[0], l[0]);
    if (u1) u.y = ff_to_double(h[1], l[1]);
    *reinterpret_cast<double2*>(U + off) = u;
    if (Usplit) {  // the (hi, lo) copy of U the next step's gathers read
      float uh[2], ul[2];
      ff_split(u.x, uh[0], ul[0]);
      ff_split(u.y, uh[1], ul[1]);
      store_pair<true>(Usplit, off, uh, ul);
    }
  }
  }
}

}  // namespace

void outer_rhs_residual_ff(const Launch& L, const DCsr& A, const DCsr& M, const double* lam, const double* U,
                           double* Fd, float* R, int ldk) {
  const Geo g = geometry_ff(ldk, L.geo);
  const int rpb = kBlock / g.tpr, rpt = ff_rows(L);
  const int grid = (A.n_rows + rpb * rpt - 1) / (rpb * rpt);
  {
    const double n = A.n_rows, nnz = (double)(A.nnz + M.nnz);
    L.rows(A.n_rows);
    L.begin(KC_OUTER_RHS, nnz * 12.0 + 2 * (n + 1) * 4.0 + n * ldk * (16.0 + 4.0), 2.0 * nnz * ldk + 2.0 * n * ldk);
  }
#define PASM_FF_RHS(AEX)                                                                      \
  PASM_FF_DISPATCH(g.ch, k_outer_rhs_res_ff<CH, AEX><<<grid, kBlock, ldk * sizeof(float2), L.s>>>( \
                             A.n_rows, A.rp, A.ci, A.vff, M.rp, M.ci, M.vff, lam, U,            \
                             reinterpret_cast<float2*>(Fd), R, ldk, g.tpr, rpt))
  if (A.exact32) { PASM_FF_RHS(true); } else { PASM_FF_RHS(false); }
#undef PASM_FF_RHS
  L.bump();
}

void outer_residual_ff(const Launch& L, const DCsr& A, const double* Fd, const double* X, float* R, int ldk) {
  const Geo g = geometry_ff(ldk, L.geo);
  const int rpb = kBlock / g.tpr, rpt = ff_rows(L);
  const int grid = (A.n_rows + rpb * rpt - 1) / (rpb * rpt);
  {
    const double n = A.n_rows, nnz = (double)A.nnz;
    L.rows(A.n_rows);
    L.begin(KC_OUTER_RES, nnz * 12.0 + (n + 1) * 4.0 + n * ldk * (16.0 + 4.0), 2.0 * nnz * ldk + n * ldk);
  }
  if (A.exact32) {
    PASM_FF_DISPATCH(g.ch, k_outer_res_ff<CH, true><<<grid, kBlock, 0, L.s>>>(
                               A.n_rows, A.rp, A.ci, A.vff, reinterpret_cast<const float2*>(Fd), X, R, ldk, g.tpr, rpt));
  } else {
    PASM_FF_DISPATCH(g.ch, k_outer_res_ff<CH, false><<<grid, kBlock, 0, L.s>>>(
                               A.n_rows, A.rp, A.ci, A.vff, reinterpret_cast<const float2*>(Fd), X, R, ldk, g.tpr, rpt));
  }
  L.bump();
}

int border_products_ff(const Launch& L, const DCsr& A, const DCsr& M, const double* X, double* YA, double* YM,
                       double* partials, int ldk, int max_blocks) {
  Geo g = geometry_ff(ldk, L.geo);
  // the per-block reduction buffer (rows per block x 2 x ldk doubles) stays within the
  // default 48 KB of dynamic shared memory; a tile shape that needs more is not used
  if ((size_t)(kBlock / g.tpr) * 2 * ldk * sizeof(double) > 48 * 1024) g = geometry_ff(ldk, 0);
  const int rpb = kBlock / g.tpr;
  int grid = std::min((A.n_rows + rpb - 1) / rpb, max_blocks);
  if (grid < 1) grid = 1;
  const size_t smem = (size_t)rpb * 2 * ldk * sizeof(double);
  {
    const double n = A.n_rows, nnz = (double)(A.nnz + M.nnz);
    L.rows(A.n_rows);
    L.begin(KC_BORDER, nnz * 12.0 + 2 * (n + 1) * 4.0 + 3.0 * n * ldk * 8.0, 2.0 * nnz * ldk + 4.0 * n * ldk);
  }
#define PASM_FF_BORDER(AEX, MG)                                                                \
  PASM_FF_DISPATCH(g.ch, k_border_ff<CH, AEX, MG><<<grid, kBlock, smem, L.s>>>(                 \
                             A.n_rows, A.rp, A.ci, A.vff, M.rp, M.ci, M.vff, X, YA, YM, partials, ldk, g.tpr, M.am))
  if (M.am) {
    if (A.exact32) { PASM_FF_BORDER(true, true); } else { PASM_FF_BORDER(false, true); }
  } else {
    if (A.exact32) { PASM_FF_BORDER(true, false); } else { PASM_FF_BORDER(false, false); }
  }
#undef PASM_FF_BORDER
  L.bump();
  return grid;
}

void spmm_ff(const Launch& L, const DCsr& S, const double* X, bool x_ff, double* out, bool out_ff, int ldk) {
  if (S.n_rows == 0) return;
  const Geo g = geometry_ff(ldk, L.geo);
  const int rpb = kBlock / g.tpr, rpt = ff_rows(L);
  const int grid = (S.n_rows + rpb * rpt - 1) / (rpb * rpt);
  {
    const double rows = S.n_rows, cols = S.n_cols, nnz = (double)S.nnz;
    L.rows(S.n_rows);
    L.begin(KC_SPMM, nnz * 12.0 + (rows + 1) * 4.0 + cols * ldk * 8.0 + rows * ldk * 8.0, 2.0 * nnz * ldk);
  }
#define PASM_FF_SPMM(FI, FO)                                                                                   \
  if (S.exact32) {                                                                                             \
    PASM_FF_DISPATCH(g.ch, k_spmm_ff<CH, FI, FO, true><<<grid, kBlock, 0, L.s>>>(S.n_rows, S.rp, S.ci, S.vff, X, \
                                                                                  out, ldk, g.tpr, rpt));           \
  } else {                                                                                                     \
    PASM_FF_DISPATCH(g.ch, k_spmm_ff<CH, FI, FO, false><<<grid, kBlock, 0, L.s>>>(S.n_rows, S.rp, S.ci, S.vff, \
                                                                                   X, out, ldk, g.tpr, rpt));       \
  }
  if (x_ff && out_ff) { PASM_FF_SPMM(true, true); }
  else if (x_ff) { PASM_FF_SPMM(true, false); }
  else if (out_ff) { PASM_FF_SPMM(false, true); }
  else { PASM_FF_SPMM(false, false); }
#undef PASM_FF_SPMM
  L.bump();
}

void spmm2_ff(const Launch& L, const DCsr& S, const double* XA, const double* XM, bool x_ff, double* outA,
              double* outM, bool out_ff, int ldk) {
  if (S.n_rows == 0) return;
  const Geo g = geometry_ff(ldk, L.geo);
  const int rpb = kBlock / g.tpr, rpt = ff_rows(L);
  const int grid = (S.n_rows + rpb * rpt - 1) / (rpb * rpt);
  {
    const double rows = S.n_rows, cols = S.n_cols, nnz = (double)S.nnz;
    L.rows(S.n_rows);
    L.begin(KC_SPMM, nnz * 12.0 + (rows + 1) * 4.0 + 2.0 * (cols + rows) * ldk * 8.0, 4.0 * nnz * ldk);
  }
#define PASM_FF_SPMM2(FI, FO)                                                                                    \
  if (S.exact32) {                                                                                               \
    PASM_FF_DISPATCH(g.ch, k_spmm2_ff<CH, FI, FO, true><<<grid, kBlock, 0, L.s>>>(S.n_rows, S.rp, S.ci, S.vff, XA,  \
                                                                                   XM, outA, outM, ldk, g.tpr, rpt)); \
  } else {                                                                                                       \
    PASM_FF_DISPATCH(g.ch, k_spmm2_ff<CH, FI, FO, false><<<grid, kBlock, 0, L.s>>>(S.n_rows, S.rp, S.ci, S.vff, XA, \
                                                                                    XM, outA, outM, ldk, g.tpr, rpt)); \
  }
  if (x_ff && out_ff) { PASM_FF_SPMM2(true, true); }
  else if (x_ff) { PASM_FF_SPMM2(true, false); }
  else if (out_ff) { PASM_FF_SPMM2(false, true); }
  else { PASM_FF_SPMM2(false, false); }
#undef PASM_FF_SPMM2
  L.bump();
}

static int stream_grid(int64_t total) { return (int)std::min<int64_t>((total / 2 + kBlock - 1) / kBlock, 152 * 16); }

void axpy_ff(const Launch& L, int n, const double* B, bool b_ff, const float* E, double* X, int ldk) {
  const int64_t total = (int64_t)n * ldk;
  L.begin(KC_AXPY, (double)total * (16.0 + 4.0), (double)total);
  if (b_ff) k_axpy_ff<true><<<stream_grid(total), kBlock, 0, L.s>>>(total, B, E, X);
  else k_axpy_ff<false><<<stream_grid(total), kBlock, 0, L.s>>>(total, B, E, X);
  L.bump();
}

void to_ff(const Launch& L, int64_t total, const double* in, double* out) {
  L.begin(KC_CAST, (double)total * 16.0, 0.0);
  k_to_ff<<<stream_grid(total), kBlock, 0, L.s>>>(total, in, out);
  L.bump();
}

void from_ff(const Launch& L, int64_t total, const double* in, double* out) {
  L.begin(KC_CAST, (double)total * 16.0, (double)total);
  k_from_ff<<<stream_grid(total), kBlock, 0, L.s>>>(total, in, out);
  L.bump();
}

void update_pairs_ff(const Launch& L, const DCsr* P, int n, const double* W, bool w_ff, const double* X,
                     const double* alpha, const int* upd, double* U, double* Usplit, int ldk) {
  const Geo g = geometry_ff(ldk, L.geo);
  const int rpb = kBlock / g.tpr, rpt = ff_rows(L);
  const int grid = (n + rpb * rpt - 1) / (rpb * rpt);
  const int identity = P ? 0 : 1;
  {
    const double nn = n, nnz = P ? (double)P->nnz : 0.0, cols = P ? (double)P->n_cols : nn;
    L.begin(KC_UPDATE, nnz * 12.0 + (nn + 1) * 4.0 + cols * ldk * 8.0 + 3.0 * nn * ldk * 8.0,
            2.0 * nnz * ldk + 2.0 * nn * ldk);
  }
  const int* rp = P ? P->rp : nullptr;
  const int* ci = P ? P->ci : nullptr;
  const float2* pv = P ? P->vff : nullptr;
  const bool ex = P ? P->exact32 : true;
#define PASM_FF_UPD(WF, EXV)                                                                                  \
  PASM_FF_DISPATCH(g.ch, k_update_ff<CH, WF, EXV><<<grid, kBlock, ldk * sizeof(float2), L.s>>>(                \
                             n, rp, ci, pv, W, X, alpha, upd, U,                                                \
                                                                           Usplit, ldk, g.tpr, identity, rpt))
  if (w_ff) {
    if (ex) { PASM_FF_UPD(true, true); } else { PASM_FF_UPD(true, false); }
  } else {
    if (ex) { PASM_FF_UPD(false, true); } else { PASM_FF_UPD(false, false); }
  }
#undef PASM_FF_UPD
  L.bump();
}

}  // namespace pasm
