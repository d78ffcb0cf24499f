// Device kernels of the PASM correction step on sm_103a.
//
// Block vectors are n x ldk row-major (ldk = k rounded up to a power of two
// >= 4), so a gathered column index of a CSR row yields ldk contiguous values
// and every matrix entry is reused ldk times (all pairs of Algorithm 1 share
// the same matrices; Section 3.2 runs them independently).  A "row group" of
// tpr threads owns one row, each thread CH chunks of one 16-byte vector.
#include "common.cuh"
#include "ff.cuh"
#include "kernels.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>

namespace pasm {

static constexpr int kBlock = 256;

struct Geo {
  int tpr, ch;
};
// Row-group geometry for ldk columns of T: chunks = ldk / (16 / sizeof(T))
// 16-byte chunks per row, tpr threads per row, ch chunks per thread.  The
// default is the fewest chunks per thread with tpr <= 32; pref (1, 2, 4, 8;
// chosen by the autotuner) is taken when it divides the row with tpr <= 32.
template <typename T>
static Geo geometry(int ldk, int pref = 0) {
  const int V = Vec16<T>::N;
  int chunks = ldk / V;
  Geo g;
  if (chunks <= 32) { g.tpr = chunks; g.ch = 1; }
  else { g.tpr = 32; g.ch = chunks / 32; }
  if ((pref == 1 || pref == 2 || pref == 4 || pref == 8) && chunks % pref == 0 && chunks / pref <= 32) {
    g.tpr = chunks / pref;
    g.ch = pref;
  }
  return g;
}

#define PASM_DISPATCH_CH(ch, ...)                          \
  switch (ch) {                                            \
    case 1: { constexpr int CH = 1; __VA_ARGS__; } break;  \
    case 2: { constexpr int CH = 2; __VA_ARGS__; } break;  \
    case 4: { constexpr int CH = 4; __VA_ARGS__; } break;  \
    case 8: { constexpr int CH = 8; __VA_ARGS__; } break;  \
    default: break;                                        \
  }

// acc += a_p * X[ci_p, cols] for the N entries p .. p+N-1 (all valid): the N
// index/value loads first, then the N row gathers, then the FMAs, so N
// gathers are in flight at once.  With dscale, a_p is scaled by
// omega * dscale[ci_p].
template <typename T, int CH, int N>
__device__ __forceinline__ void gather_group(const int* __restrict__ ci, const T* __restrict__ av,
                                             const T* __restrict__ dscale, T omega, const T* __restrict__ X, int p,
                                             int lane, int tpr, int ldk, T (&acc)[CH][Vec16<T>::N]) {
  constexpr int V = Vec16<T>::N;
  int j[N];
  T a[N];
#pragma unroll
  for (int u = 0; u < N; ++u) {
    j[u] = __ldg(ci + p + u);
    a[u] = __ldg(av + p + u);
  }
  if (dscale) {
#pragma unroll
    for (int u = 0; u < N; ++u) a[u] *= omega * __ldg(dscale + j[u]);
  }
  T x[N][CH][V];
#pragma unroll
  for (int u = 0; u < N; ++u)
#pragma unroll
    for (int c = 0; c < CH; ++c) ldg16<T>(X + (size_t)j[u] * ldk + (c * tpr + lane) * V, x[u][c]);
#pragma unroll
  for (int u = 0; u < N; ++u)
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[c][v] = fma(a[u], x[u][c][v], acc[c][v]);
}

// acc += sum_{p0 <= p < p1} a_p * X[ci_p, cols]: full groups of 4 entries, then
// an exact group of the remaining 1-3 (no padded loads, no wasted FMAs).
template <typename T, int CH>
__device__ __forceinline__ void gather_rows(const int* __restrict__ ci, const T* __restrict__ av,
                                            const T* __restrict__ dscale, T omega, const T* __restrict__ X, int p0,
                                            int p1, int lane, int tpr, int ldk, T (&acc)[CH][Vec16<T>::N]) {
  int p = p0;
  for (; p + 4 <= p1; p += 4) gather_group<T, CH, 4>(ci, av, dscale, omega, X, p, lane, tpr, ldk, acc);
  const int rem = p1 - p;
  if (rem == 3) gather_group<T, CH, 3>(ci, av, dscale, omega, X, p, lane, tpr, ldk, acc);
  else if (rem == 2) gather_group<T, CH, 2>(ci, av, dscale, omega, X, p, lane, tpr, ldk, acc);
  else if (rem == 1) gather_group<T, CH, 1>(ci, av, dscale, omega, X, p, lane, tpr, ldk, acc);
}

// ----------------------------------------------------------------------------------------------
// Row blocks per block: a block may walk `rpt` consecutive row blocks, so that fewer blocks are
// launched and the neighbour rows one row block gathers are still in L1 for the next.  The
// autotuner picks 1 or 4 per level and kernel kind; untuned launches take 1.  Float32 kernels only:
// for the float64 ones (bound by the float64 pipe) the count is the constant 1 on both sides.
template <typename T> struct RowBlocks { __host__ __device__ static constexpr int of(int) { return 1; } };
template <> struct RowBlocks<float> { __host__ __device__ static constexpr int of(int r) { return r; } };
template <typename T>
static int rows_per_block(const Launch& L) { return RowBlocks<T>::of(L.rpt > 0 ? L.rpt : 1); }

// Float32 row operations: registers capped so that 2048 threads fit an SM (one chunk per thread)
// or 1024 (two chunks); wider chunks and float64 keep the compiler's choice.
template <typename T, int CH> struct RowMinBlocks { static constexpr int v = 0; };  // 0: no minimum (compiler default)
template <> struct RowMinBlocks<float, 1> { static constexpr int v = 8; };
template <> struct RowMinBlocks<float, 2> { static constexpr int v = 4; };

// Generic row operation (Jacobi sweep, residual, SpMM, SpMM + add).
template <typename T, int CH, int OP>
__global__ void __launch_bounds__(kBlock, (RowMinBlocks<T, CH>::v)) k_rowop(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                   const T* __restrict__ av, const T* __restrict__ X,
                                                   const T* Y, const T* Z, const T* __restrict__ dinv, T omega,
                                                   T* out, int ldk, int tpr, int rpt) {
  constexpr int V = Vec16<T>::N;
  const int rpb = kBlock / tpr;
  const int lane = threadIdx.x % tpr;
  for (int rr = 0; rr < RowBlocks<T>::of(rpt); ++rr) {
  const int row = (blockIdx.x * RowBlocks<T>::of(rpt) + rr) * rpb + threadIdx.x / tpr;
  if (row >= n) return;
  T acc[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[c][v] = T(0);
  // row-aligned operands first: their loads overlap the gather's round trips
  const size_t base = (size_t)row * ldk;
  T y[CH][V], z[CH][V];
  T w = T(0);
  if (OP != OP_SPMM) {
#pragma unroll
    for (int c = 0; c < CH; ++c) Vec16<T>::load(Y + base + (c * tpr + lane) * V, y[c]);
  }
  if (OP == OP_JACOBI) {
    w = omega * dinv[row];
#pragma unroll
    for (int c = 0; c < CH; ++c) Vec16<T>::load(Z + base + (c * tpr + lane) * V, z[c]);
  }
  gather_rows<T, CH>(ci, av, nullptr, T(0), X, rp[row], rp[row + 1], lane, tpr, ldk, acc);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const size_t off = base + (c * tpr + lane) * V;
    T r[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if (OP == OP_JACOBI) r[v] = fma(w, y[c][v] - acc[c][v], z[c][v]);
      else if (OP == OP_RESID) r[v] = y[c][v] - acc[c][v];
      else if (OP == OP_SPMM) r[v] = acc[c][v];
      else r[v] = y[c][v] + acc[c][v];
    }
    Vec16<T>::store(out + off, r);
  }
  }
}

template <typename T>
void rowop(const Launch& L, RowOp op, const DCsr& S, const T* X, const T* Y, const T* Z, const T* dinv, T omega,
           T* out, int ldk) {
  if (S.n_rows == 0) return;
  Geo g = geometry<T>(ldk, L.geo);
  const int rpb = kBlock / g.tpr;
  const int rpt = rows_per_block<T>(L);
  const int grid = (S.n_rows + rpb * rpt - 1) / (rpb * rpt);
  const T* av = vals<T>(S);
  {
    const double sz = sizeof(T), rows = S.n_rows, cols = S.n_cols, nnz = (double)S.nnz;
    double bytes = nnz * (4.0 + sz) + (rows + 1) * 4.0 + cols * ldk * sz + rows * ldk * sz;
    double flops = 2.0 * nnz * ldk;
    int cls = KC_SPMM;
    if (op == OP_JACOBI) { bytes += rows * ldk * sz + rows * sz; flops += 3.0 * rows * ldk; cls = KC_JACOBI; }
    else if (op == OP_RESID) { bytes += rows * ldk * sz; flops += rows * ldk; cls = KC_RESID; }
    else if (op == OP_SPMM_ADD) { bytes += rows * ldk * sz; flops += rows * ldk; cls = KC_PROLONG; }
    L.rows(S.n_rows);
    L.begin(cls, bytes, flops);
  }
  PASM_DISPATCH_CH(g.ch,
    switch (op) {
      case OP_JACOBI: k_rowop<T, CH, OP_JACOBI><<<grid, kBlock, 0, L.s>>>(S.n_rows, S.rp, S.ci, av, X, Y, Z, dinv, omega, out, ldk, g.tpr, rpt); break;
      case OP_RESID: k_rowop<T, CH, OP_RESID><<<grid, kBlock, 0, L.s>>>(S.n_rows, S.rp, S.ci, av, X, Y, Z, dinv, omega, out, ldk, g.tpr, rpt); break;
      case OP_SPMM: k_rowop<T, CH, OP_SPMM><<<grid, kBlock, 0, L.s>>>(S.n_rows, S.rp, S.ci, av, X, Y, Z, dinv, omega, out, ldk, g.tpr, rpt); break;
      case OP_SPMM_ADD: k_rowop<T, CH, OP_SPMM_ADD><<<grid, kBlock, 0, L.s>>>(S.n_rows, S.rp, S.ci, av, X, Y, Z, dinv, omega, out, ldk, g.tpr, rpt); break;
    });
  L.bump();
}
template void rowop<double>(const Launch&, RowOp, const DCsr&, const double*, const double*, const double*,
                            const double*, double, double*, int);
template void rowop<float>(const Launch&, RowOp, const DCsr&, const float*, const float*, const float*,
                           const float*, float, float*, int);

// ----------------------------------------------------------------------------------------------
// Prolongate-and-correct fused with the first post-smoothing sweep (float32 cycles):
//   out = xn + omega D^{-1} (F - A xn),  xn = X + P Ec,
// with xn formed on the fly for the row and each neighbour the sweep gathers (Ec, the coarse
// correction, is a quarter of the rows and stays in L2), so the corrected iterate is never written
// and read back.  Every product and sum is taken in the order of the unfused pair (the
// prolongation's row sum of P Ec, then X + it; the sweep's row sum over A in CSR order).
template <int CH>
__global__ void __launch_bounds__(kBlock) k_prolong_jacobi(int n, const int* __restrict__ arp,
                                                           const int* __restrict__ aci, const float* __restrict__ av,
                                                           const int* __restrict__ prp, const int* __restrict__ pci,
                                                           const float* __restrict__ pv, const float* __restrict__ X,
                                                           const float* __restrict__ Ec, const float* __restrict__ F,
                                                           const float* __restrict__ dinv, float omega,
                                                           float* __restrict__ out, int ldk, int tpr) {
  constexpr int V = 4;
  const int rpb = kBlock / tpr;
  const int row = blockIdx.x * rpb + threadIdx.x / tpr;
  const int lane = threadIdx.x % tpr;
  if (row >= n) return;
  const size_t base = (size_t)row * ldk;
  float y[CH][V], z[CH][V], acc[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    Vec16<float>::load(F + base + (c * tpr + lane) * V, y[c]);
#pragma unroll
    for (int v = 0; v < V; ++v) acc[c][v] = z[c][v] = 0.f;
  }
  const float w = omega * dinv[row];
  const int p1 = __ldg(arp + row + 1);
  for (int p = __ldg(arp + row); p < p1; ++p) {
    const int j = __ldg(aci + p);
    const float a = __ldg(av + p);
    float xn[CH][V], ap[CH][V];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      ldg16<float>(X + (size_t)j * ldk + (c * tpr + lane) * V, xn[c]);
#pragma unroll
      for (int v = 0; v < V; ++v) ap[c][v] = 0.f;
    }
    const int q1 = __ldg(prp + j + 1);
    for (int q = __ldg(prp + j); q < q1; ++q) {
      const int m = __ldg(pci + q);
      const float pw = __ldg(pv + q);
      float e[CH][V];
#pragma unroll
      for (int c = 0; c < CH; ++c) ldg16<float>(Ec + (size_t)m * ldk + (c * tpr + lane) * V, e[c]);
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int v = 0; v < V; ++v) ap[c][v] = fmaf(pw, e[c][v], ap[c][v]);
    }
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const float x = xn[c][v] + ap[c][v];
        if (j == row) z[c][v] = x;
        acc[c][v] = fmaf(a, x, acc[c][v]);
      }
  }
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    float r[V];
#pragma unroll
    for (int v = 0; v < V; ++v) r[v] = fmaf(w, y[c][v] - acc[c][v], z[c][v]);
    Vec16<float>::store(out + base + (c * tpr + lane) * V, r);
  }
}

void prolong_jacobi(const Launch& L, const DCsr& A, const DCsr& P, const float* X, const float* Ec, const float* F,
                    const float* dinv, float omega, float* out, int ldk) {
  if (A.n_rows == 0) return;
  Geo g = geometry<float>(ldk, L.geo);
  const int rpb = kBlock / g.tpr;
  const int grid = (A.n_rows + rpb - 1) / rpb;
  {
    const double rows = A.n_rows, nnz = (double)A.nnz, pnnz = (double)P.nnz;
    // the matrices, X gathered once, Ec (P's columns) once, F read, out written, D^{-1}
    const double bytes = (nnz + pnnz) * 8.0 + 2 * (rows + 1) * 4.0 + 3.0 * rows * ldk * 4.0 +
                         P.n_cols * (double)ldk * 4.0 + rows * 4.0;
    L.rows(A.n_rows);
    L.begin(KC_JACOBI, bytes, 2.0 * (nnz + pnnz) * ldk + 4.0 * rows * ldk);
  }
  PASM_DISPATCH_CH(g.ch, k_prolong_jacobi<CH><<<grid, kBlock, 0, L.s>>>(A.n_rows, A.rp, A.ci, A.v32, P.rp, P.ci,
                                                                          P.v32, X, Ec, F, dinv, omega, out, ldk,
                                                                          g.tpr));
  L.bump();
}

// ----------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_jacobi_zero(int64_t total, int ldk, const T* __restrict__ dinv, T omega, const T* __restrict__ F,
                              T* __restrict__ out) {
  constexpr int V = Vec16<T>::N;
  const int64_t nv = total / V;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i * V;
    const int64_t row = e / ldk;
    const T w = omega * dinv[row];
    T f[V], r[V];
    Vec16<T>::load(F + e, f);
#pragma unroll
    for (int v = 0; v < V; ++v) r[v] = w * f[v];
    Vec16<T>::store(out + e, r);
  }
}

template <typename T>
void jacobi_zero(const Launch& L, int n, const T* dinv, T omega, const T* F, T* out, int ldk) {
  if (n == 0) return;
  const int64_t total = (int64_t)n * ldk;
  const int64_t nv = total / Vec16<T>::N;
  int grid = (int)std::min<int64_t>((nv + kBlock - 1) / kBlock, 152 * 16);
  L.begin(KC_JACOBI0, (2.0 * total + n) * sizeof(T), 2.0 * total);
  k_jacobi_zero<T><<<grid, kBlock, 0, L.s>>>(total, ldk, dinv, omega, F, out);
  L.bump();
}
template void jacobi_zero<double>(const Launch&, int, const double*, double, const double*, double*, int);
template void jacobi_zero<float>(const Launch&, int, const float*, float, const float*, float*, int);

// ----------------------------------------------------------------------------------------------
// Fused multigrid kernels (used for the float32 V-cycle, where arithmetic is
// cheap and HBM passes are the cost).
//
// Two Jacobi sweeps from a zero guess in one pass:
//   e1 = w D^-1 f,  e2 = e1 + w D^-1 (f - A e1) = w D^-1 (2 f - A (w D^-1 f)).
// Float32 sweeps from zero and fused residual-restrictions are held to 64
// registers (four 256-thread blocks per SM): at h = 1/1024, k = 64 the finest
// two-sweep kernel went 187 -> 177 us and the level-2 residual-restriction
// 67 -> 50 us; the other row kernels were as fast or slower that way.  Float64
// kernels keep the compiler's choice.
template <typename T> struct MinBlocks { static constexpr int gather = 1; };
template <> struct MinBlocks<float> { static constexpr int gather = 4; };

template <typename T, int CH>
__global__ void __launch_bounds__(kBlock, MinBlocks<T>::gather) k_jacobi2_zero(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                          const T* __restrict__ av, const T* __restrict__ dinv,
                                                          T omega, const T* __restrict__ F, T* __restrict__ out,
                                                          int ldk, int tpr, int prescaled, int rpt) {
  constexpr int V = Vec16<T>::N;
  const int rpb = kBlock / tpr;
  const int lane = threadIdx.x % tpr;
  for (int rr = 0; rr < RowBlocks<T>::of(rpt); ++rr) {
  const int row = (blockIdx.x * RowBlocks<T>::of(rpt) + rr) * rpb + threadIdx.x / tpr;
  if (row >= n) return;
  T acc[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[c][v] = T(0);
  const T w = omega * dinv[row];
  const size_t base = (size_t)row * ldk;
  T f[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c) ldg16<T>(F + base + (c * tpr + lane) * V, f[c]);
  // prescaled: av already holds omega a_ij / a_jj
  gather_rows<T, CH>(ci, av, prescaled ? nullptr : dinv, omega, F, rp[row], rp[row + 1], lane, tpr, ldk, acc);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const size_t off = base + (c * tpr + lane) * V;
    T r[V];
#pragma unroll
    for (int v = 0; v < V; ++v) r[v] = w * (T(2) * f[c][v] - acc[c][v]);
    Vec16<T>::store(out + off, r);
  }
  }
}

// Residual and restriction in one pass: fc = R (f - A e), the residual of each
// fine row recomputed for every coarse row that restricts it.
template <typename T, int CH>
__global__ void __launch_bounds__(kBlock, MinBlocks<T>::gather) k_resid_restrict(int nc, const int* __restrict__ rrp,
                                                            const int* __restrict__ rci, const T* __restrict__ rv,
                                                            const int* __restrict__ arp, const int* __restrict__ aci,
                                                            const T* __restrict__ av, const T* __restrict__ E,
                                                            const T* __restrict__ F, T* __restrict__ out, int ldk,
                                                            int tpr, int rpt) {
  constexpr int V = Vec16<T>::N;
  const int rpb = kBlock / tpr;
  const int lane = threadIdx.x % tpr;
  for (int rr = 0; rr < RowBlocks<T>::of(rpt); ++rr) {
  const int row = (blockIdx.x * RowBlocks<T>::of(rpt) + rr) * rpb + threadIdx.x / tpr;
  if (row >= nc) return;
  T acc[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[c][v] = T(0);
  const int q0 = rrp[row], q1 = rrp[row + 1];
  for (int q = q0; q < q1; ++q) {
    const int i = __ldg(rci + q);
    const T wq = __ldg(rv + q);
    T r[CH][V], ae[CH][V];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      ldg16<T>(F + (size_t)i * ldk + (c * tpr + lane) * V, r[c]);
#pragma unroll
      for (int v = 0; v < V; ++v) ae[c][v] = T(0);
    }
    gather_rows<T, CH>(aci, av, nullptr, T(0), E, __ldg(arp + i), __ldg(arp + i + 1), lane, tpr, ldk, ae);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[c][v] = fma(wq, r[c][v] - ae[c][v], acc[c][v]);
  }
  const size_t base = (size_t)row * ldk;
#pragma unroll
  for (int c = 0; c < CH; ++c) Vec16<T>::store(out + base + (c * tpr + lane) * V, acc[c]);
  }
}

template <typename T>
void jacobi2_zero(const Launch& L, const DCsr& A, const T* dinv, T omega, const T* F, T* out, int ldk) {
  if (A.n_rows == 0) return;
  Geo g = geometry<T>(ldk, L.geo);
  const int rpb = kBlock / g.tpr;
  const int rpt = rows_per_block<T>(L);
  const int grid = (A.n_rows + rpb * rpt - 1) / (rpb * rpt);
  {
    const double sz = sizeof(T), rows = A.n_rows, nnz = (double)A.nnz;
    L.rows(A.n_rows);
    L.begin(KC_JACOBI, nnz * (4.0 + sz) + (rows + 1) * 4.0 + rows * sz + 2.0 * rows * ldk * sz,
            3.0 * nnz * ldk + 2.0 * rows * ldk);
  }
  const T* ws = scaled_vals<T>(A);
  PASM_DISPATCH_CH(g.ch, k_jacobi2_zero<T, CH><<<grid, kBlock, 0, L.s>>>(A.n_rows, A.rp, A.ci, ws ? ws : vals<T>(A),
                                                                          dinv, omega, F, out, ldk, g.tpr,
                                                                          ws ? 1 : 0, rpt));
  L.bump();
}

template <typename T>
void resid_restrict(const Launch& L, const DCsr& R, const DCsr& A, const T* E, const T* F, T* out, int ldk) {
  if (R.n_rows == 0) return;
  Geo g = geometry<T>(ldk, L.geo);
  const int rpb = kBlock / g.tpr;
  const int rpt = rows_per_block<T>(L);
  const int grid = (R.n_rows + rpb * rpt - 1) / (rpb * rpt);
  {
    const double sz = sizeof(T), nf = A.n_rows, nc = R.n_rows;
    L.rows(A.n_rows);
    L.begin(KC_RESID, (double)(A.nnz + R.nnz) * (4.0 + sz) + (nf + nc + 2) * 4.0 + 2.0 * nf * ldk * sz +
                          nc * ldk * sz,
            2.0 * (double)(A.nnz + R.nnz) * ldk + nf * ldk);
  }
  PASM_DISPATCH_CH(g.ch, k_resid_restrict<T, CH><<<grid, kBlock, 0, L.s>>>(R.n_rows, R.rp, R.ci, vals<T>(R), A.rp,
                                                                            A.ci, vals<T>(A), E, F, out, ldk, g.tpr, rpt));
  L.bump();
}

// Restriction first: out (coarse) = R F - (R A) E, with R A formed once at setup.  The same
// coarse residual as R (F - A E) in exact arithmetic; each coarse row gathers its fine rows of F and
// the fine rows of E that R A couples to it (about 7 + 19 rows in 2D) instead of recomputing the
// residual of every fine row it restricts (7 x 6 row loads).  Float32 cycles only.
template <int CH>
__global__ void __launch_bounds__(kBlock, (RowMinBlocks<float, CH>::v)) k_restrict_first(
    int nc, const int* __restrict__ rrp, const int* __restrict__ rci, const float* __restrict__ rv,
    const int* __restrict__ qrp, const int* __restrict__ qci, const float* __restrict__ qv,
    const float* __restrict__ E, const float* __restrict__ F, float* __restrict__ out, int ldk, int tpr, int rpt) {
  constexpr int V = 4;
  const int rpb = kBlock / tpr;
  const int lane = threadIdx.x % tpr;
  for (int rr = 0; rr < rpt; ++rr) {
    const int row = (blockIdx.x * rpt + rr) * rpb + threadIdx.x / tpr;
    if (row >= nc) return;
    float rf[CH][V], qe[CH][V];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v) rf[c][v] = qe[c][v] = 0.f;
    gather_rows<float, CH>(rci, rv, nullptr, 0.f, F, rrp[row], rrp[row + 1], lane, tpr, ldk, rf);
    gather_rows<float, CH>(qci, qv, nullptr, 0.f, E, qrp[row], qrp[row + 1], lane, tpr, ldk, qe);
    const size_t base = (size_t)row * ldk;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      float o[V];
#pragma unroll
      for (int v = 0; v < V; ++v) o[v] = rf[c][v] - qe[c][v];
      Vec16<float>::store(out + base + (c * tpr + lane) * V, o);
    }
  }
}

void restrict_first(const Launch& L, const DCsr& R, const DCsr& RA, const float* E, const float* F, float* out,
                    int ldk) {
  if (R.n_rows == 0) return;
  Geo g = geometry<float>(ldk, L.geo);
  const int rpb = kBlock / g.tpr;
  const int rpt = rows_per_block<float>(L);
  const int grid = (R.n_rows + rpb * rpt - 1) / (rpb * rpt);
  {
    const double nf = RA.n_cols, nc = R.n_rows;
    L.rows(RA.n_cols);
    L.begin(KC_RESID, (double)(R.nnz + RA.nnz) * 8.0 + 2.0 * (nc + 1) * 4.0 + 2.0 * nf * ldk * 4.0 + nc * ldk * 4.0,
            2.0 * (double)(R.nnz + RA.nnz) * ldk + nc * ldk);
  }
  PASM_DISPATCH_CH(g.ch, k_restrict_first<CH><<<grid, kBlock, 0, L.s>>>(R.n_rows, R.rp, R.ci, R.v32, RA.rp, RA.ci,
                                                                         RA.v32, E, F, out, ldk, g.tpr, rpt));
  L.bump();
}

template void jacobi2_zero<float>(const Launch&, const DCsr&, const float*, float, const float*, float*, int);
template void jacobi2_zero<double>(const Launch&, const DCsr&, const double*, double, const double*, double*, int);
template void resid_restrict<float>(const Launch&, const DCsr&, const DCsr&, const float*, const float*, float*, int);
template void resid_restrict<double>(const Launch&, const DCsr&, const DCsr&, const double*, const double*, double*,
                                     int);

// ----------------------------------------------------------------------------------------------
// Outer float64 kernels of the defect correction.
template <typename TV> __device__ __forceinline__ void store_vec2(TV* p, double a, double b);
template <> __device__ __forceinline__ void store_vec2<double>(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
template <> __device__ __forceinline__ void store_vec2<float>(float* p, double a, double b) {
  *reinterpret_cast<float2*>(p) = make_float2((float)a, (float)b);
}
template <typename TV> __device__ __forceinline__ void load_vec2(const TV* p, double* v);
template <> __device__ __forceinline__ void load_vec2<double>(const double* p, double* v) {
  double2 t = *reinterpret_cast<const double2*>(p); v[0] = t.x; v[1] = t.y;
}
template <> __device__ __forceinline__ void load_vec2<float>(const float* p, double* v) {
  float2 t = *reinterpret_cast<const float2*>(p); v[0] = t.x; v[1] = t.y;
}

// One row, float64 gather of S X over CH chunks of 2 columns.
template <int CH>
__device__ __forceinline__ void gather_row64(const int* __restrict__ rp, const int* __restrict__ ci,
                                             const double* __restrict__ av, const double* __restrict__ X, int row,
                                             int lane, int tpr, int ldk, double (&acc)[CH][2]) {
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c][0] = acc[c][1] = 0.0;
  gather_rows<double, CH>(ci, av, nullptr, 0.0, X, rp[row], rp[row + 1], lane, tpr, ldk, acc);
}

template <typename TV, int CH>
__global__ void __launch_bounds__(kBlock) k_outer_rhs_res(int n, const int* __restrict__ arp, const int* __restrict__ aci,
                                                           const double* __restrict__ aval, const int* __restrict__ mrp,
                                                           const int* __restrict__ mci, const double* __restrict__ mval,
                                                           const double* __restrict__ lam, const double* __restrict__ U,
                                                           double* __restrict__ Fd, TV* __restrict__ R, int ldk, int tpr) {
  const int rpb = kBlock / tpr;
  const int row = blockIdx.x * rpb + threadIdx.x / tpr;
  const int lane = threadIdx.x % tpr;
  if (row >= n) return;
  double mu[CH][2], au[CH][2];
  gather_row64<CH>(mrp, mci, mval, U, row, lane, tpr, ldk, mu);
  gather_row64<CH>(arp, aci, aval, U, row, lane, tpr, ldk, au);
  const size_t base = (size_t)row * ldk;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * tpr + lane) * 2;
    const double f0 = lam[col] * mu[c][0], f1 = lam[col + 1] * mu[c][1];
    *reinterpret_cast<double2*>(Fd + base + col) = make_double2(f0, f1);
    store_vec2<TV>(R + base + col, f0 - au[c][0], f1 - au[c][1]);
  }
}

template <typename TV, int CH>
__global__ void __launch_bounds__(kBlock) k_outer_res(int n, const int* __restrict__ arp, const int* __restrict__ aci,
                                                       const double* __restrict__ aval, const double* __restrict__ Fd,
                                                       const double* __restrict__ X, TV* __restrict__ R, int ldk, int tpr) {
  const int rpb = kBlock / tpr;
  const int row = blockIdx.x * rpb + threadIdx.x / tpr;
  const int lane = threadIdx.x % tpr;
  if (row >= n) return;
  double ax[CH][2];
  gather_row64<CH>(arp, aci, aval, X, row, lane, tpr, ldk, ax);
  const size_t base = (size_t)row * ldk;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * tpr + lane) * 2;
    double2 f = *reinterpret_cast<const double2*>(Fd + base + col);
    store_vec2<TV>(R + base + col, f.x - ax[c][0], f.y - ax[c][1]);
  }
}

template <typename TV>
__global__ void k_outer_axpy(int64_t total, const double* B, const TV* __restrict__ E, double* X) {
  const int64_t np = total / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    double e[2];
    load_vec2<TV>(E + 2 * i, e);
    double2 b = *reinterpret_cast<const double2*>(B + 2 * i);
    *reinterpret_cast<double2*>(X + 2 * i) = make_double2(b.x + e[0], b.y + e[1]);
  }
}

static Geo geometry64(int ldk, int pref = 0) { return geometry<double>(ldk, pref); }

template <typename TV>
void outer_rhs_residual(const Launch& L, const DCsr& A, const DCsr& M, const double* lam, const double* U,
                        double* Fd, TV* R, int ldk) {
  Geo g = geometry64(ldk, L.geo);
  const int rpb = kBlock / g.tpr;
  const int grid = (A.n_rows + rpb - 1) / rpb;
  {
    const double n = A.n_rows, nnz = (double)(A.nnz + M.nnz);
    L.rows(A.n_rows);
    L.begin(KC_OUTER_RHS, nnz * 12.0 + 2 * (n + 1) * 4.0 + n * ldk * (16.0 + sizeof(TV)),
            2.0 * nnz * ldk + 2.0 * n * ldk);
  }
  PASM_DISPATCH_CH(g.ch, k_outer_rhs_res<TV, CH><<<grid, kBlock, 0, L.s>>>(A.n_rows, A.rp, A.ci, A.v64, M.rp, M.ci,
                                                                            M.v64, lam, U, Fd, R, ldk, g.tpr));
  L.bump();
}
template <typename TV>
void outer_residual(const Launch& L, const DCsr& A, const double* Fd, const double* X, TV* R, int ldk) {
  Geo g = geometry64(ldk, L.geo);
  const int rpb = kBlock / g.tpr;
  const int grid = (A.n_rows + rpb - 1) / rpb;
  {
    const double n = A.n_rows, nnz = (double)A.nnz;
    L.rows(A.n_rows);
    L.begin(KC_OUTER_RES, nnz * 12.0 + (n + 1) * 4.0 + n * ldk * (16.0 + sizeof(TV)), 2.0 * nnz * ldk + n * ldk);
  }
  PASM_DISPATCH_CH(g.ch, k_outer_res<TV, CH><<<grid, kBlock, 0, L.s>>>(A.n_rows, A.rp, A.ci, A.v64, Fd, X, R, ldk,
                                                                        g.tpr));
  L.bump();
}
template <typename TV>
void outer_axpy(const Launch& L, int n, const double* B, const TV* E, double* X, int ldk) {
  const int64_t total = (int64_t)n * ldk;
  int grid = (int)std::min<int64_t>((total / 2 + kBlock - 1) / kBlock, 152 * 16);
  L.begin(KC_AXPY, (double)total * (16.0 + sizeof(TV)), (double)total);
  k_outer_axpy<TV><<<grid, kBlock, 0, L.s>>>(total, B, E, X);
  L.bump();
}
template void outer_rhs_residual<double>(const Launch&, const DCsr&, const DCsr&, const double*, const double*,
                                         double*, double*, int);
template void outer_rhs_residual<float>(const Launch&, const DCsr&, const DCsr&, const double*, const double*,
                                        double*, float*, int);
template void outer_residual<double>(const Launch&, const DCsr&, const double*, const double*, double*, int);
template void outer_residual<float>(const Launch&, const DCsr&, const double*, const double*, float*, int);
template void outer_axpy<double>(const Launch&, int, const double*, const double*, double*, int);
template void outer_axpy<float>(const Launch&, int, const double*, const float*, double*, int);

// ----------------------------------------------------------------------------------------------
// Bordering (the matrix form of Section 3.1): YA = A u~, YM = M u~ and the
// column dot products beta = u~^T A u~, zeta = u~^T M u~ as per-block partials.
template <int CH>
__global__ void __launch_bounds__(kBlock) k_border(int n, const int* __restrict__ arp, const int* __restrict__ aci,
                                                    const double* __restrict__ aval, const int* __restrict__ mrp,
                                                    const int* __restrict__ mci, const double* __restrict__ mval,
                                                    const double* __restrict__ X, double* __restrict__ YA,
                                                    double* __restrict__ YM, double* __restrict__ partials, int ldk,
                                                    int tpr) {
  extern __shared__ double red[];  // [rpb][2][ldk]
  const int rpb = kBlock / tpr;
  const int grp = threadIdx.x / tpr;
  const int lane = threadIdx.x % tpr;
  double sA[CH][2], sM[CH][2];
#pragma unroll
  for (int c = 0; c < CH; ++c) sA[c][0] = sA[c][1] = sM[c][0] = sM[c][1] = 0.0;
  for (int row = blockIdx.x * rpb + grp; row < n; row += gridDim.x * rpb) {
    double ya[CH][2], ym[CH][2];
    gather_row64<CH>(arp, aci, aval, X, row, lane, tpr, ldk, ya);
    gather_row64<CH>(mrp, mci, mval, X, row, lane, tpr, ldk, ym);
    const size_t base = (size_t)row * ldk;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int col = (c * tpr + lane) * 2;
      double2 x = *reinterpret_cast<const double2*>(X + base + col);
      *reinterpret_cast<double2*>(YA + base + col) = make_double2(ya[c][0], ya[c][1]);
      *reinterpret_cast<double2*>(YM + base + col) = make_double2(ym[c][0], ym[c][1]);
      sA[c][0] = fma(x.x, ya[c][0], sA[c][0]);
      sA[c][1] = fma(x.y, ya[c][1], sA[c][1]);
      sM[c][0] = fma(x.x, ym[c][0], sM[c][0]);
      sM[c][1] = fma(x.y, ym[c][1], sM[c][1]);
    }
  }
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * tpr + lane) * 2;
    red[(grp * 2 + 0) * ldk + col] = sA[c][0];
    red[(grp * 2 + 0) * ldk + col + 1] = sA[c][1];
    red[(grp * 2 + 1) * ldk + col] = sM[c][0];
    red[(grp * 2 + 1) * ldk + col + 1] = sM[c][1];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * ldk; t += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < rpb; ++r) s += red[r * 2 * ldk + t];
    partials[(size_t)blockIdx.x * 2 * ldk + t] = s;
  }
}

int border_products(const Launch& L, const DCsr& A, const DCsr& M, const double* X, double* YA, double* YM,
                    double* partials, int ldk, int max_blocks) {
  Geo g = geometry64(ldk, L.geo);
  // the per-block reduction buffer (rows per block x 2 x ldk doubles) stays within the
  // default 48 KB of dynamic shared memory; a tile shape that needs more is not used
  if ((size_t)(kBlock / g.tpr) * 2 * ldk * sizeof(double) > 48 * 1024) g = geometry64(ldk, 0);
  const int rpb = kBlock / g.tpr;
  int grid = std::min((A.n_rows + rpb - 1) / rpb, max_blocks);
  if (grid < 1) grid = 1;
  const size_t smem = (size_t)rpb * 2 * ldk * sizeof(double);
  {
    const double n = A.n_rows, nnz = (double)(A.nnz + M.nnz);
    L.rows(A.n_rows);
    L.begin(KC_BORDER, nnz * 12.0 + 2 * (n + 1) * 4.0 + 3.0 * n * ldk * 8.0, 2.0 * nnz * ldk + 4.0 * n * ldk);
  }
  PASM_DISPATCH_CH(g.ch, k_border<CH><<<grid, kBlock, smem, L.s>>>(A.n_rows, A.rp, A.ci, A.v64, M.rp, M.ci, M.v64, X,
                                                                    YA, YM, partials, ldk, g.tpr));
  L.bump();
  return grid;
}

// One block per output: its 128 threads sum strided partials, then a fixed-order
// tree reduction (deterministic).
__global__ void __launch_bounds__(128) k_colsum(const double* __restrict__ partials, int nblk, int width,
                                                double* __restrict__ out) {
  __shared__ double red[4];
  const int t = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 128) s += partials[(size_t)b * width + t];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) out[t] = (red[0] + red[1]) + (red[2] + red[3]);
}

// Eigen-residual report (the paper's stopping quantity, Section 5): per-block
// column partials of sum_i r_ij^2 (r = lambda M u - A u, from the outer
// residual kernel) and sum_i u_ij (lambda M u)_ij, accumulated in float64;
// layout [block][2][ldk] as for column_sums.  FF: Fd and U hold (hi, lo) float
// pairs (mixed precision), else float64.  Thread t of a block owns the column
// pair t % (ldk / 2) on every (kBlock / (ldk / 2))-th row.
template <typename TR, bool FF>
__global__ void __launch_bounds__(kBlock) k_residual_partials(int n, int ldk, const TR* __restrict__ R,
                                                              const double* __restrict__ Fd,
                                                              const double* __restrict__ U,
                                                              double* __restrict__ partials) {
  __shared__ double red[kBlock * 4];
  const int cpairs = ldk / 2, rpb = kBlock / cpairs;
  const int cp = threadIdx.x % cpairs, ro = threadIdx.x / cpairs;
  double rr0 = 0.0, rr1 = 0.0, um0 = 0.0, um1 = 0.0;
  if (ro < rpb) {
    for (int row = blockIdx.x * rpb + ro; row < n; row += gridDim.x * rpb) {
      const size_t off = (size_t)row * ldk + 2 * cp;
      const double r0 = (double)R[off], r1 = (double)R[off + 1];
      double m0, m1, u0, u1;
      if (FF) {
        const float4 f = *reinterpret_cast<const float4*>(Fd + off);
        const float4 u = *reinterpret_cast<const float4*>(U + off);
        m0 = (double)f.x + (double)f.y; m1 = (double)f.z + (double)f.w;
        u0 = (double)u.x + (double)u.y; u1 = (double)u.z + (double)u.w;
      } else {
        m0 = Fd[off]; m1 = Fd[off + 1];
        u0 = U[off]; u1 = U[off + 1];
      }
      rr0 = fma(r0, r0, rr0); rr1 = fma(r1, r1, rr1);
      um0 = fma(u0, m0, um0); um1 = fma(u1, m1, um1);
    }
  }
  double* mine = red + 4 * threadIdx.x;
  mine[0] = rr0; mine[1] = rr1; mine[2] = um0; mine[3] = um1;
  __syncthreads();
  if (ro == 0) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < rpb; ++q)
      for (int e = 0; e < 4; ++e) s[e] += red[4 * (q * cpairs + cp) + e];
    double* out = partials + (size_t)blockIdx.x * 2 * ldk;
    out[2 * cp] = s[0]; out[2 * cp + 1] = s[1];
    out[ldk + 2 * cp] = s[2]; out[ldk + 2 * cp + 1] = s[3];
  }
}

template <typename TR>
int residual_partials(const Launch& L, int n, int ldk, const TR* R, bool ff, const double* Fd, const double* U,
                      double* partials, int max_blocks) {
  const int rpb = kBlock / (ldk / 2);
  const int grid = std::max(1, std::min((n + rpb - 1) / rpb, max_blocks));
  L.begin(KC_COLSUM, (double)n * ldk * (sizeof(TR) + 16.0), 4.0 * n * ldk);
  if (ff) k_residual_partials<TR, true><<<grid, kBlock, 0, L.s>>>(n, ldk, R, Fd, U, partials);
  else k_residual_partials<TR, false><<<grid, kBlock, 0, L.s>>>(n, ldk, R, Fd, U, partials);
  L.bump();
  return grid;
}
template int residual_partials<float>(const Launch&, int, int, const float*, bool, const double*, const double*,
                                      double*, int);
template int residual_partials<double>(const Launch&, int, int, const double*, bool, const double*, const double*,
                                       double*, int);

void column_sums(const Launch& L, const double* partials, int nblk, int nq, int ldk, double* out) {
  const int width = nq * ldk;
  L.begin(KC_COLSUM, (double)nblk * width * 8.0 + width * 8.0, (double)nblk * width);
  k_colsum<<<width, 128, 0, L.s>>>(partials, nblk, width, out);
  L.bump();
}

// ----------------------------------------------------------------------------------------------
// Small dense products on the coarse space (N_H x N_H times N_H x ldk).
template <typename T>
__global__ void k_dense_mm(int m, int p, const T* __restrict__ D, int ldd, int trans, const T* __restrict__ B,
                           T* __restrict__ C, int ldk) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (c >= ldk || i >= m) return;
  T s = T(0);
  if (trans) {
    for (int j = 0; j < p; ++j) s = fma(D[(size_t)j * ldd + i], B[(size_t)j * ldk + c], s);
  } else {
    const T* d = D + (size_t)i * ldd;
    for (int j = 0; j < p; ++j) s = fma(d[j], B[(size_t)j * ldk + c], s);
  }
  C[(size_t)i * ldk + c] = s;
}

template <typename T>
void dense_mm(const Launch& L, int m, int p, const T* D, int ldd, bool trans, const T* B, T* C, int ldk) {
  dim3 grid((ldk + 63) / 64, m);
  L.begin(KC_DENSE, ((double)m * p + (double)p * ldk + (double)m * ldk) * sizeof(T), 2.0 * m * p * ldk);
  k_dense_mm<T><<<grid, 64, 0, L.s>>>(m, p, D, ldd, trans ? 1 : 0, B, C, ldk);
  L.bump();
}
template void dense_mm<double>(const Launch&, int, int, const double*, int, bool, const double*, double*, int);
template void dense_mm<float>(const Launch&, int, int, const float*, int, bool, const float*, float*, int);

__global__ void k_coarse_init(int NH, int k, const double* __restrict__ Q, const double* __restrict__ lamH,
                              double* __restrict__ W0, double* __restrict__ lam, int ldk) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (c >= ldk) return;
  W0[(size_t)j * ldk + c] = c < k ? Q[(size_t)j * NH + c] / sqrt(lamH[c]) : 0.0;
  if (j == 0) lam[c] = c < k ? lamH[c] : 1.0;
}

void coarse_init(const Launch& L, int NH, int k, const double* Q, const double* lamH, double* W0, double* lam,
                 int ldk) {
  dim3 grid((ldk + 63) / 64, NH);
  L.begin(KC_INIT, (double)NH * ldk * 16.0, 0.0);
  k_coarse_init<<<grid, 64, 0, L.s>>>(NH, k, Q, lamH, W0, lam, ldk);
  L.bump();
}

// ----------------------------------------------------------------------------------------------
// Update u^(l+1) = alpha u~ + P_c u_H (Algorithm 1, output of step 2), the last
// prolongation fused with the combination.
template <int CH>
__global__ void __launch_bounds__(kBlock) k_update(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                    const double* __restrict__ pv, const double* __restrict__ W,
                                                    const double* __restrict__ X, const double* __restrict__ alpha,
                                                    const int* __restrict__ upd, double* __restrict__ U, int ldk,
                                                    int tpr, int identity) {
  const int rpb = kBlock / tpr;
  const int row = blockIdx.x * rpb + threadIdx.x / tpr;
  const int lane = threadIdx.x % tpr;
  if (row >= n) return;
  double pw[CH][2];
  if (identity) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      double2 w = *reinterpret_cast<const double2*>(W + (size_t)row * ldk + (c * tpr + lane) * 2);
      pw[c][0] = w.x; pw[c][1] = w.y;
    }
  } else {
    gather_row64<CH>(rp, ci, pv, W, row, lane, tpr, ldk, pw);
  }
  const size_t base = (size_t)row * ldk;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * tpr + lane) * 2;
    double2 x = *reinterpret_cast<const double2*>(X + base + col);
    double2 u = *reinterpret_cast<const double2*>(U + base + col);
    if (upd[col]) u.x = fma(alpha[col], x.x, pw[c][0]);
    if (upd[col + 1]) u.y = fma(alpha[col + 1], x.y, pw[c][1]);
    *reinterpret_cast<double2*>(U + base + col) = u;
  }
}

void update_pairs(const Launch& L, const DCsr& P, const double* W, const double* X, const double* alpha,
                  const int* upd, double* U, int ldk) {
  Geo g = geometry64(ldk, L.geo);
  const int rpb = kBlock / g.tpr;
  const int grid = (P.n_rows + rpb - 1) / rpb;
  {
    const double n = P.n_rows, nnz = (double)P.nnz;
    L.begin(KC_UPDATE, nnz * 12.0 + (n + 1) * 4.0 + (double)P.n_cols * ldk * 8.0 + 3.0 * n * ldk * 8.0,
            2.0 * nnz * ldk + 2.0 * n * ldk);
  }
  PASM_DISPATCH_CH(g.ch, k_update<CH><<<grid, kBlock, 0, L.s>>>(P.n_rows, P.rp, P.ci, P.v64, W, X, alpha, upd, U,
                                                                 ldk, g.tpr, 0));
  L.bump();
}
void update_pairs_identity(const Launch& L, int n, const double* W, const double* X, const double* alpha,
                           const int* upd, double* U, int ldk) {
  Geo g = geometry64(ldk, L.geo);
  const int rpb = kBlock / g.tpr;
  const int grid = (n + rpb - 1) / rpb;
  L.begin(KC_UPDATE, 4.0 * n * ldk * 8.0, 2.0 * n * ldk);
  PASM_DISPATCH_CH(g.ch, k_update<CH><<<grid, kBlock, 0, L.s>>>(n, nullptr, nullptr, nullptr, W, X, alpha, upd, U,
                                                                 ldk, g.tpr, 1));
  L.bump();
}

__global__ void k_count_active(const int* __restrict__ active, int k, int* out) {
  int c = 0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) c += active[i] != 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (threadIdx.x == 0) *out = c;
}
void count_active(const Launch& L, const int* active, int k, int* out) {
  L.begin(KC_COUNT, k * 4.0, 0.0);
  k_count_active<<<1, 32, 0, L.s>>>(active, k, out);
  L.bump();
}

__global__ void k_cast_d2f(const double* __restrict__ in, float* __restrict__ out, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
void cast_d2f(const Launch& L, const double* in, float* out, int64_t count) {
  if (count == 0) return;
  int grid = (int)std::min<int64_t>((count + kBlock - 1) / kBlock, 152 * 16);
  L.begin(KC_CAST, count * 12.0, 0.0);
  k_cast_d2f<<<grid, kBlock, 0, L.s>>>(in, out, count);
  L.bump();
}

}  // namespace pasm

namespace pasm {

// ----------------------------------------------------------------------------------------------
// The last Jacobi sweep of the top-level V-cycle fused with the outer update of
// the mixed path: e' = z + omega dinv (y - A z) in float32 as k_rowop<float, JACOBI>,
// then X = B + e' in double-float ((hi, lo) float pairs, B in pairs or float64),
// so e' is never stored.
template <int CH, bool BFF>
__global__ void __launch_bounds__(kBlock)
    k_jacobi_axpy_ff(int n, const int* __restrict__ rp, const int* __restrict__ ci, const float* __restrict__ av,
                     const float* __restrict__ E, const float* __restrict__ F, const float* __restrict__ dinv,
                     float omega, const double* B, double* X, int ldk, int tpr, int rpt) {
  constexpr int V = 4;
  const int rpb = kBlock / tpr;
  const int lane = threadIdx.x % tpr;
  for (int rr = 0; rr < rpt; ++rr) {
  const int row = (blockIdx.x * rpt + rr) * rpb + threadIdx.x / tpr;
  if (row >= n) return;
  float acc[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[c][v] = 0.f;
  const size_t base = (size_t)row * ldk;
  float y[CH][V], z[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    Vec16<float>::load(F + base + (c * tpr + lane) * V, y[c]);
    Vec16<float>::load(E + base + (c * tpr + lane) * V, z[c]);
  }
  const float w = omega * dinv[row];
  gather_rows<float, CH>(ci, av, nullptr, 0.f, E, rp[row], rp[row + 1], lane, tpr, ldk, acc);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const size_t off = base + (c * tpr + lane) * V;
    float h[V], l[V];
    if (BFF) {
      const float4 b0 = *reinterpret_cast<const float4*>(B + off);
      const float4 b1 = *reinterpret_cast<const float4*>(B + off + 2);
      h[0] = b0.x; l[0] = b0.y; h[1] = b0.z; l[1] = b0.w; h[2] = b1.x; l[2] = b1.y; h[3] = b1.z; l[3] = b1.w;
    } else {
      const double2 b0 = *reinterpret_cast<const double2*>(B + off);
      const double2 b1 = *reinterpret_cast<const double2*>(B + off + 2);
      ff_split(b0.x, h[0], l[0]); ff_split(b0.y, h[1], l[1]); ff_split(b1.x, h[2], l[2]); ff_split(b1.y, h[3], l[3]);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float e = fmaf(w, y[c][v] - acc[c][v], z[c][v]);
      ff_mac(h[v], l[v], e, 0.f, 1.f, 0.f);
      ff_norm(h[v], l[v]);
    }
    *reinterpret_cast<float4*>(X + off) = make_float4(h[0], l[0], h[1], l[1]);
    *reinterpret_cast<float4*>(X + off + 2) = make_float4(h[2], l[2], h[3], l[3]);
  }
  }
}

void jacobi_axpy_ff(const Launch& L, const DCsr& A, const float* E, const float* F, const float* dinv, float omega,
                    const double* B, bool b_ff, double* X, int ldk) {
  if (A.n_rows == 0) return;
  const Geo g = geometry<float>(ldk, L.geo);
  const int rpb = kBlock / g.tpr;
  const int rpt = rows_per_block<float>(L);  // the plain sweep's choice on this level
  const int grid = (A.n_rows + rpb * rpt - 1) / (rpb * rpt);
  {
    const double rows = A.n_rows, cols = A.n_cols, nnz = (double)A.nnz;
    L.rows(A.n_rows);
    L.begin(KC_SWEEP_UPDATE, nnz * 8.0 + (rows + 1) * 4.0 + cols * ldk * 4.0 + rows * ldk * (4.0 + 16.0) + rows * 4.0,
            2.0 * nnz * ldk + 4.0 * rows * ldk);
  }
  if (b_ff) {
    PASM_DISPATCH_CH(g.ch, k_jacobi_axpy_ff<CH, true><<<grid, kBlock, 0, L.s>>>(A.n_rows, A.rp, A.ci, A.v32, E, F, dinv,
                                                                                 omega, B, X, ldk, g.tpr, rpt));
  } else {
    PASM_DISPATCH_CH(g.ch, k_jacobi_axpy_ff<CH, false><<<grid, kBlock, 0, L.s>>>(A.n_rows, A.rp, A.ci, A.v32, E, F,
                                                                                  dinv, omega, B, X, ldk, g.tpr, rpt));
  }
  L.bump();
}

// ----------------------------------------------------------------------------------------------
// Conjugate-gradient smoother (the multigrid smoother of the paper's experiments, Section 5.1):
// nu CG steps for A x = f, each column an independent CG, all columns batched.  Vectors in the
// cycle's precision T; the column dot products are summed per thread in T, per block in float64
// and across blocks in float64 by one block per column (fixed order: deterministic).
namespace {

// Per-block column sums s[c][v] (per thread) -> partial[blockIdx.x][col] in float64.
template <typename T, int CH>
__device__ __forceinline__ void block_column_partials(const T (&s)[CH][Vec16<T>::N], double* red, int grp,
                                                      int lane, int tpr, int rpb, int ldk, double* partial) {
  constexpr int V = Vec16<T>::N;
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) red[grp * ldk + (c * tpr + lane) * V + v] = (double)s[c][v];
  __syncthreads();
  for (int t = threadIdx.x; t < ldk; t += blockDim.x) {
    double a = 0.0;
    for (int r = 0; r < rpb; ++r) a += red[r * ldk + t];
    partial[(size_t)blockIdx.x * ldk + t] = a;
  }
}

// r = f - A x (x == nullptr: r = f), p = r, partial sums of r.r
template <typename T, int CH>
__global__ void __launch_bounds__(kBlock) k_cg_start(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                      const T* __restrict__ av, const T* __restrict__ X,
                                                      const T* __restrict__ F, T* __restrict__ R, T* __restrict__ P,
                                                      double* __restrict__ partial, int ldk, int tpr) {
  extern __shared__ double red[];
  constexpr int V = Vec16<T>::N;
  const int rpb = kBlock / tpr, grp = threadIdx.x / tpr, lane = threadIdx.x % tpr;
  T s[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) s[c][v] = T(0);
  for (int row = blockIdx.x * rpb + grp; row < n; row += gridDim.x * rpb) {
    T acc[CH][V];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[c][v] = T(0);
    if (X) gather_rows<T, CH>(ci, av, nullptr, T(0), X, rp[row], rp[row + 1], lane, tpr, ldk, acc);
    const size_t base = (size_t)row * ldk;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const size_t off = base + (c * tpr + lane) * V;
      T f[V], r[V];
      ldg16<T>(F + off, f);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        r[v] = f[v] - acc[c][v];
        s[c][v] = fma(r[v], r[v], s[c][v]);
      }
      Vec16<T>::store(R + off, r);
      Vec16<T>::store(P + off, r);
    }
  }
  block_column_partials<T, CH>(s, red, grp, lane, tpr, rpb, ldk, partial);
}

// q = A p, partial sums of p.q
template <typename T, int CH>
__global__ void __launch_bounds__(kBlock) k_cg_dir(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                    const T* __restrict__ av, const T* __restrict__ P,
                                                    T* __restrict__ Q, double* __restrict__ partial, int ldk,
                                                    int tpr) {
  extern __shared__ double red[];
  constexpr int V = Vec16<T>::N;
  const int rpb = kBlock / tpr, grp = threadIdx.x / tpr, lane = threadIdx.x % tpr;
  T s[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) s[c][v] = T(0);
  for (int row = blockIdx.x * rpb + grp; row < n; row += gridDim.x * rpb) {
    T acc[CH][V];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[c][v] = T(0);
    gather_rows<T, CH>(ci, av, nullptr, T(0), P, rp[row], rp[row + 1], lane, tpr, ldk, acc);
    const size_t base = (size_t)row * ldk;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const size_t off = base + (c * tpr + lane) * V;
      T p[V];
      ldg16<T>(P + off, p);
#pragma unroll
      for (int v = 0; v < V; ++v) s[c][v] = fma(p[v], acc[c][v], s[c][v]);
      Vec16<T>::store(Q + off, acc[c]);
    }
  }
  block_column_partials<T, CH>(s, red, grp, lane, tpr, rpb, ldk, partial);
}

// x = (x_zero ? 0 : x) + alpha p, r -= alpha q, partial sums of r.r
template <typename T, int CH>
__global__ void __launch_bounds__(kBlock) k_cg_update(int n, T* __restrict__ X, T* __restrict__ R,
                                                       const T* __restrict__ P, const T* __restrict__ Q,
                                                       const double* __restrict__ alpha, double* __restrict__ partial,
                                                       int ldk, int tpr, int x_zero) {
  extern __shared__ double red[];
  constexpr int V = Vec16<T>::N;
  const int rpb = kBlock / tpr, grp = threadIdx.x / tpr, lane = threadIdx.x % tpr;
  T s[CH][V], a[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) {
      s[c][v] = T(0);
      a[c][v] = (T)alpha[(c * tpr + lane) * V + v];
    }
  for (int row = blockIdx.x * rpb + grp; row < n; row += gridDim.x * rpb) {
    const size_t base = (size_t)row * ldk;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const size_t off = base + (c * tpr + lane) * V;
      T x[V], r[V], p[V], q[V];
      if (x_zero) {
#pragma unroll
        for (int v = 0; v < V; ++v) x[v] = T(0);
      } else {
        Vec16<T>::load(X + off, x);
      }
      Vec16<T>::load(R + off, r);
      ldg16<T>(P + off, p);
      ldg16<T>(Q + off, q);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        x[v] = fma(a[c][v], p[v], x[v]);
        r[v] = fma(-a[c][v], q[v], r[v]);
        s[c][v] = fma(r[v], r[v], s[c][v]);
      }
      Vec16<T>::store(X + off, x);
      Vec16<T>::store(R + off, r);
    }
  }
  block_column_partials<T, CH>(s, red, grp, lane, tpr, rpb, ldk, partial);
}

// p = r + beta p
template <typename T>
__global__ void k_cg_pupdate(int64_t total, int ldk, const T* __restrict__ R, T* __restrict__ P,
                             const double* __restrict__ beta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    P[i] = fma((T)beta[i % ldk], P[i], R[i]);
}

// One block per column: s = sum of the partials; mode 0: rr = s; mode 1: alpha = rr / s
// (0 if s <= 0); mode 2: beta = s / rr (0 if rr <= 0), rr = s.
__global__ void __launch_bounds__(128) k_cg_scalar(const double* __restrict__ partial, int nblk, int ldk, int mode,
                                                   double* __restrict__ rr, double* __restrict__ coef) {
  __shared__ double w[4];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 128) s += partial[(size_t)b * ldk + c];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    s = (w[0] + w[1]) + (w[2] + w[3]);
    if (mode == 0) {
      rr[c] = s;
    } else if (mode == 1) {
      coef[c] = s > 0.0 ? rr[c] / s : 0.0;
    } else {
      coef[c] = rr[c] > 0.0 ? s / rr[c] : 0.0;
      rr[c] = s;
    }
  }
}

}  // namespace

template <typename T>
void cg_smooth(const Launch& L, const DCsr& A, const T* F, T* X, bool x_zero, T* R, T* P, T* Q, const CgWork& w,
               int ldk, int nu) {
  if (A.n_rows == 0 || nu < 1) return;
  const Geo g = geometry<T>(ldk, L.geo);
  const int rpb = kBlock / g.tpr;
  const int grid = std::max(1, std::min((A.n_rows + rpb - 1) / rpb, w.max_blocks));
  const size_t smem = (size_t)rpb * ldk * sizeof(double);
  const double sz = sizeof(T), rows = A.n_rows, nnz = (double)A.nnz, vec = rows * ldk * sz;
  const double mat = nnz * (4.0 + sz) + (rows + 1) * 4.0;
  const T* av = vals<T>(A);
  auto scalars = [&](int mode, double* coef) {
    L.begin(KC_CG, (double)grid * ldk * 8.0, (double)grid * ldk);
    k_cg_scalar<<<ldk, 128, 0, L.s>>>(w.partial, grid, ldk, mode, w.rr, coef);
    L.bump();
  };
  L.rows(A.n_rows);
  L.begin(KC_CG, (x_zero ? 0.0 : mat + vec) + 3.0 * vec, x_zero ? 2.0 * rows * ldk : 2.0 * nnz * ldk + 3.0 * rows * ldk);
  PASM_DISPATCH_CH(g.ch, k_cg_start<T, CH><<<grid, kBlock, smem, L.s>>>(A.n_rows, A.rp, A.ci, av, x_zero ? nullptr : X,
                                                                         F, R, P, w.partial, ldk, g.tpr));
  L.bump();
  scalars(0, nullptr);
  for (int it = 0; it < nu; ++it) {
    L.rows(A.n_rows);
    L.begin(KC_CG, mat + 2.0 * vec, 2.0 * nnz * ldk + 2.0 * rows * ldk);
    PASM_DISPATCH_CH(g.ch, k_cg_dir<T, CH><<<grid, kBlock, smem, L.s>>>(A.n_rows, A.rp, A.ci, av, P, Q, w.partial,
                                                                         ldk, g.tpr));
    L.bump();
    scalars(1, w.alpha);
    const bool xz = x_zero && it == 0;
    L.rows(A.n_rows);
    L.begin(KC_CG, (xz ? 5.0 : 6.0) * vec, 6.0 * rows * ldk);
    PASM_DISPATCH_CH(g.ch, k_cg_update<T, CH><<<grid, kBlock, smem, L.s>>>(A.n_rows, X, R, P, Q, w.alpha, w.partial,
                                                                            ldk, g.tpr, xz ? 1 : 0));
    L.bump();
    if (it + 1 < nu) {
      scalars(2, w.beta);
      const int64_t total = (int64_t)A.n_rows * ldk;
      L.begin(KC_CG, 3.0 * vec, 2.0 * rows * ldk);
      k_cg_pupdate<T><<<(int)std::min<int64_t>((total + kBlock - 1) / kBlock, 152 * 16), kBlock, 0, L.s>>>(
          total, ldk, R, P, w.beta);
      L.bump();
    }
  }
}
template void cg_smooth<float>(const Launch&, const DCsr&, const float*, float*, bool, float*, float*, float*,
                               const CgWork&, int, int);
template void cg_smooth<double>(const Launch&, const DCsr&, const double*, double*, bool, double*, double*, double*,
                                const CgWork&, int, int);

}  // namespace pasm
