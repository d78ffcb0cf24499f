// Batched augmented eigensolve and selection (Algorithm 1 step 2) on sm_103a.
//
// For one pair the bordered pencil of Section 3.1,
//     [[A_H, b], [b^T, beta]] x = theta [[M_H, c], [c^T, zeta]] x,
// is reduced once per setup by the coarse eigendecomposition A_H Q = M_H Q Lambda
// (Q^T M_H Q = I).  In the b-orthonormal basis {P_c q_j} + {w^} with
// w = u~ - P_c Q c',  c' = Q^T c,  b' = Q^T b,  zt = zeta - |c'|^2 = |w|_b^2,
// the pencil becomes the symmetric arrowhead matrix [[Lambda, z], [z^T, rho]]:
//     z   = (b' - Lambda c') / sqrt(zt),
//     rho = (beta - 2 c'.b' + c'^T Lambda c') / zt.
// Its eigenvalues are the roots of the secular equation
//     f(theta) = theta - rho + sum_j z_j^2 / (lambda_j - theta) = 0,
// one in each gap between consecutive poles (Cauchy interlacing), plus one
// below and one above.  Eigenvector of root theta: [y; 1] with
// y_j = -z_j / (lambda_j - theta).  Its component along u~ is
// b(v, u~) = (y.c' + sqrt(zt)) / |[y; 1]|  (b-normalised); the a-normalised
// score divides by sqrt(theta).  Since u~ lies in V_{H,h}, the squared
// b-normalised scores of all roots sum to zeta (Parseval), which certifies the
// winner from a window of roots around the current eigenvalue.
//
// Root finder: safeguarded rational interpolation in the spirit of Bunch,
// Nielsen and Sorensen (1978) -- the left and right partial sums are modelled
// by one pole each (the linear term joins the right part), matching value and
// derivative at the iterate, and the model's root in the interval is taken;
// steps leaving the bracket fall back to bisection.  The iterate is kept as an
// offset tau from the nearer pole so that lambda_j - theta is formed without
// cancellation.  Indices with |z_j| below 8 eps times the problem scale are
// deflated: theta = lambda_j with eigenvector e_j.  Two poles that coincide to
// rounding (an exact degeneracy of the coarse pencil, as the symmetries of the
// 3D Kuhn mesh produce) are merged by a rotation in their plane: one pole keeps
// the weight z_a^2 + z_b^2, the other becomes a deflated root with eigenvector
// (z_b e_a - z_a e_b) / r; eigenvectors of the remaining roots keep the
// formula y_j = -z_j / (lambda_j - theta) in the original coordinates.
//
// Launch: one thread-block cluster of cs CTAs per pair (cs = 1..4, as many as
// keep k * cs within the SM count).  Every CTA of the cluster builds the same
// pole data; the roots of a phase are spread over the cluster's warps, and each
// solved root is written into every CTA's shared memory (distributed shared
// memory), so that all CTAs take the same selection and certificate decisions;
// the cluster barrier orders the exchange.  GB300's float64 pipe (2 FMA per
// clock and SM) bounds the root solves, so more SMs per pair is more
// throughput.  Rank 0 alone writes the results.
#include "common.cuh"
#include "kernels.cuh"

#include <cooperative_groups.h>

#include <cfloat>
#include <climits>

namespace pasm {

static constexpr int kSecThreads = 256;
static constexpr int kSecWarps = kSecThreads / 32;
static constexpr int kMaxIter = 80;

enum { ST_ACTIVE = 0, ST_CONVERGED = 1, ST_DEGENERATE = 2, ST_NAN = 3 };

struct SecShared {
  double* d;      // NH
  double* z;      // NH
  double* cq;     // NH
  double* w;      // NH: pole weight z_j^2 (merged weight for a merged pair)
  int* J;         // NH: poles of the secular equation, ascending
  int* K;         // NH: indices with a nonzero eigenvector component (J and merged-away ones)
  int* pole;      // NH: pole whose lambda enters y_i = -z_i / (lambda_pole - theta)
  int* rot;       // NH: for an index merged away into an equal pole, that pole; else -1
  double* theta;  // NH+1 roots
  double* orig;   // NH+1 origin (pole) of each root
  double* tau;    // NH+1 offset from origin
  double* sb;     // NH+1 signed b-normalised score
  int* solved;    // NH+1
};

__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = (threadIdx.x < kSecWarps) ? red[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// 1/x for the pole sums, by Newton-Raphson iteration y <- y + y (1 - x y)
// (quadratic convergence) from a float32 reciprocal of x's leading 24 bits:
// the seed's relative error (< 2^-22) squares to < 2^-44 after one step and to
// float64 rounding after the second, so the result is within a few ulp of 1/x.
// The seed and its widening are formed from the bit fields (integer pipe), so
// only the four FMAs use the float64 pipe, GB300's scarce one.  Exponents
// outside 2^(+-120) (where the float32 seed would leave the normal range),
// zero, Inf and NaN take the float64 division.
__device__ __forceinline__ double rcp_nr(double x) {
  const int hi = __double2hiint(x);
  const int e = (hi >> 20) & 0x7FF;
  if (e < 1023 - 120 || e > 1023 + 120) return 1.0 / x;
  const unsigned fb = ((unsigned)hi & 0x80000000u) | ((unsigned)(e - 896) << 23) | (((unsigned)hi & 0xFFFFFu) << 3) |
                      ((unsigned)__double2loint(x) >> 29);
  const unsigned rb = __float_as_uint(__frcp_rn(__uint_as_float(fb)));
  const unsigned re = (rb >> 23) & 0xFFu;
  double y = __hiloint2double((int)((rb & 0x80000000u) | ((re + 896u) << 20) | ((rb & 0x7FFFFFu) >> 3)),
                              (int)(rb << 29));
  double r = fma(-x, y, 1.0);
  y = fma(y, r, y);
  r = fma(-x, y, 1.0);
  return fma(y, r, y);
}

// Sums over the non-deflated poles at theta = origin + tau, split into the
// poles left of root m (indices t < m) and right of it.  Warp-cooperative.
__device__ __forceinline__ void secular_sums(const SecShared& S, int nJ, int m, double origin, double tau, int lane,
                                             double& psi, double& dpsi, double& phi, double& dphi) {
  psi = dpsi = phi = dphi = 0.0;
  for (int t = lane; t < nJ; t += 32) {
    const int j = S.J[t];
    const double r = rcp_nr((S.d[j] - origin) - tau);
    const double term = S.w[j] * r;
    if (t < m) { psi += term; dpsi = fma(term, r, dpsi); }
    else { phi += term; dphi = fma(term, r, dphi); }
  }
  psi = warp_sum(psi); dpsi = warp_sum(dpsi); phi = warp_sum(phi); dphi = warp_sum(dphi);
}

// One step of the rational model of f around the iterate (see the file
// comment).  da = a - theta < 0 and db = b - theta > 0 are the distances to the
// interval's poles (absent ones ignored).  Returns false if the model has no
// root in the interval (the caller bisects).
template <typename T>
__device__ __forceinline__ bool rational_step(bool has_left, bool has_right, T da, T db, T th, T rho, T psi,
                                              T dpsi, T phi, T dphi, T& s) {
  if (has_left && has_right) {
    const T Q1 = dpsi * da * da, P1 = psi - Q1 / da;
    const T ft = th - rho + phi;
    const T Q2 = (dphi + T(1)) * db * db, P2 = ft - Q2 / db;
    const T P = P1 + P2;
    const T A2 = P, B2 = -(P * (da + db) + Q1 + Q2), C2 = P * da * db + Q1 * db + Q2 * da;
    const T disc = fmax(B2 * B2 - T(4) * A2 * C2, T(0));
    const T q = T(-0.5) * (B2 + copysign(sqrt(disc), B2));
    bool ok = false;
    if (A2 != T(0)) { const T s1 = q / A2; if (s1 > da && s1 < db) { s = s1; ok = true; } }
    if (q != T(0)) { const T s2 = C2 / q; if (s2 > da && s2 < db) { s = s2; ok = true; } }
    return ok;
  }
  if (has_right) {  // first interval: only poles to the right
    const T Q2 = dphi * db * db, P2 = phi - Q2 / db;
    const T f0 = th - rho + P2;
    const T B2 = -(db - f0), C2 = -(f0 * db + Q2);
    const T disc = fmax(B2 * B2 - T(4) * C2, T(0));
    const T q = T(-0.5) * (B2 + copysign(sqrt(disc), B2));
    const T sm = (q != T(0)) ? fmin(q, C2 / q) : q;
    if (sm < db) { s = sm; return true; }
    return false;
  }
  // last interval: only poles to the left
  const T Q1 = dpsi * da * da, P1 = psi - Q1 / da;
  const T f0 = th - rho + P1;
  const T B2 = -(da - f0), C2 = -(f0 * da + Q1);
  const T disc = fmax(B2 * B2 - T(4) * C2, T(0));
  const T q = T(-0.5) * (B2 + copysign(sqrt(disc), B2));
  const T sm = (q != T(0)) ? fmax(q, C2 / q) : q;
  if (sm > da) { s = sm; return true; }
  return false;
}

// float32 pre-solve: the pole offsets d_j - origin and the weights z_j^2 of this
// lane's share of the poles live in registers (at most kPer per lane).
static constexpr int kPer = 32;  // supports NH <= 1024

__device__ __forceinline__ void sums32(const float (&dd)[kPer], const float (&zz)[kPer], int nJ, int m, int lane,
                                       float tau, float& psi, float& dpsi, float& phi, float& dphi) {
  psi = dpsi = phi = dphi = 0.f;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    if (32 * q >= nJ) break;  // warp-uniform: skip the unused register slots
    const int t = lane + 32 * q;
    if (t < nJ) {
      float del = dd[q] - tau;
      if (del == 0.f) del = 1e-30f;
      const float r = __fdividef(1.f, del);
      const float term = zz[q] * r;
      const float dterm = term * r;
      if (t < m) { psi += term; dpsi += dterm; }
      else { phi += term; dphi += dterm; }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    psi += __shfl_xor_sync(0xffffffffu, psi, o);
    dpsi += __shfl_xor_sync(0xffffffffu, dpsi, o);
    phi += __shfl_xor_sync(0xffffffffu, phi, o);
    dphi += __shfl_xor_sync(0xffffffffu, dphi, o);
  }
}

// Root m of the secular equation (0 <= m <= nJ), computed by one warp: a
// float32 rational iteration locates it, then float64 iterations from there
// polish it (usually one or two) inside the float64 bracket.
__device__ void solve_root(const SecShared& S, int nJ, int m, double rho, double lower, double upper, int lane,
                           int* caps) {
  const bool has_left = m > 0, has_right = m < nJ;
  if (!has_left && !has_right) {  // every pole deflated: the bordered row alone, theta = rho
    if (lane == 0) { S.theta[m] = rho; S.orig[m] = rho; S.tau[m] = 0.0; }
    __syncwarp();
    return;
  }
  const double a = has_left ? S.d[S.J[m - 1]] : lower;
  const double b = has_right ? S.d[S.J[m]] : upper;
  double origin, lo, hi;
  float dd[kPer], zz[kPer];
  auto load_offsets = [&](double org) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int t = lane + 32 * q;
      if (t < nJ) {
        const int j = S.J[t];
        dd[q] = (float)(S.d[j] - org);
        zz[q] = (float)S.w[j];
      } else {
        dd[q] = 1.f; zz[q] = 0.f;
      }
    }
  };
  if (!has_left) { origin = b; lo = lower - b; hi = 0.0; load_offsets(origin); }
  else if (!has_right) { origin = a; lo = 0.0; hi = upper - a; load_offsets(origin); }
  else {
    // which half holds the root: the sign of f at the midpoint, in float64 (in
    // float32 the sum cancels badly when rho and the weights are large)
    const double mid = 0.5 * (a + b);
    double psi, dpsi, phi, dphi;
    secular_sums(S, nJ, m, 0.0, mid, lane, psi, dpsi, phi, dphi);
    if (mid - rho + psi + phi >= 0.0) { origin = a; lo = 0.0; hi = mid - a; }
    else { origin = b; lo = mid - b; hi = 0.0; }
    load_offsets(origin);
  }
  // float32 phase
  double tau;
  {
    float flo = (float)lo, fhi = (float)hi;
    float t32 = 0.5f * (flo + fhi);
    const float forg = (float)origin, frho = (float)rho;
    const float fa = (float)(a - origin), fb = (float)(b - origin);
    for (int it = 0; it < 40; ++it) {
      float psi, dpsi, phi, dphi;
      sums32(dd, zz, nJ, m, lane, t32, psi, dpsi, phi, dphi);
      const float th = forg + t32;
      const float f = th - frho + psi + phi;
      if (fabsf(f) <= 8.f * FLT_EPSILON * (fabsf(th) + fabsf(frho) + fabsf(psi) + fabsf(phi))) break;
      if (f > 0.f) fhi = t32; else flo = t32;
      if (fhi - flo <= 4.f * FLT_EPSILON * fmaxf(fabsf(flo), fabsf(fhi))) break;
      float st = 0.f;
      const bool ok = rational_step<float>(has_left, has_right, fa - t32, fb - t32, th, frho, psi, dpsi, phi, dphi, st);
      float tn = t32 + st;
      if (!ok || !(tn > flo && tn < fhi) || !isfinite(tn)) tn = 0.5f * (flo + fhi);
      const bool tiny = fabsf(tn - t32) <= 2.f * FLT_EPSILON * fabsf(tn);
      t32 = tn;
      if (tiny) break;
    }
    tau = (double)t32;
    if (!(tau > lo && tau < hi)) tau = 0.5 * (lo + hi);
  }
  // float64 phase
  int it = 0;
  for (; it < kMaxIter; ++it) {
    double psi, dpsi, phi, dphi;
    secular_sums(S, nJ, m, origin, tau, lane, psi, dpsi, phi, dphi);
    const double th = origin + tau;
    const double f = th - rho + psi + phi;
    const double eb = 16.0 * DBL_EPSILON * (fabs(th) + fabs(rho) + fabs(psi) + fabs(phi));
    if (fabs(f) <= eb) break;
    if (f > 0.0) hi = tau; else lo = tau;
    // accuracy is judged on the offset tau from the pole, not on theta: the
    // eigenvector needs lambda_pole - theta = -tau to full relative accuracy
    if (hi - lo <= 4.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi))) break;
    double st = 0.0;
    const bool ok = rational_step<double>(has_left, has_right, (a - origin) - tau, (b - origin) - tau, th, rho, psi,
                                          dpsi, phi, dphi, st);
    double tn = tau + st;
    if (!ok || !(tn > lo && tn < hi) || !isfinite(tn)) tn = 0.5 * (lo + hi);
    const bool tiny = fabs(tn - tau) <= 2.0 * DBL_EPSILON * fabs(tn);
    tau = tn;
    if (tiny) break;
  }
  if (it == kMaxIter && lane == 0) atomicAdd(caps, 1);
  if (lane == 0) {
    S.theta[m] = origin + tau;
    S.orig[m] = origin;
    S.tau[m] = tau;
  }
  __syncwarp();
}

// Signed b-normalised score and |y|^2 of root m (warp-cooperative).
__device__ __forceinline__ void root_vector_sums(const SecShared& S, int nK, int m, int lane, double& ny2,
                                                 double& yc) {
  const double origin = S.orig[m], tau = S.tau[m];
  ny2 = 0.0; yc = 0.0;
  for (int t = lane; t < nK; t += 32) {
    const int j = S.K[t];
    const double y = -S.z[j] * rcp_nr((S.d[S.pole[j]] - origin) - tau);
    ny2 = fma(y, y, ny2);
    yc = fma(y, S.cq[j], yc);
  }
  ny2 = warp_sum(ny2); yc = warp_sum(yc);
}

// A selection candidate: score, Ritz value, preference order, kind (0 root,
// 1 deflated pole, 2 merged-away pole) and index.  No candidate yet: sc = -1
// (scores are >= 0; NaN scores are never taken).
struct Cand {
  double sc, th;
  int ord, kind, idx;
  __device__ void clear() { sc = -1.0; th = 0.0; ord = INT_MAX; kind = 0; idx = -1; }
  __device__ bool beats(const Cand& o) const {
    return sc > o.sc || (sc == o.sc && (th < o.th || (th == o.th && ord < o.ord)));
  }
  __device__ void offer(double s2, double t2, int o2, int k2, int i2) {
    Cand c;
    c.sc = s2; c.th = t2; c.ord = o2; c.kind = k2; c.idx = i2;
    if (c.beats(*this)) *this = c;
  }
};

__device__ __forceinline__ Cand shfl_cand(const Cand& c, int o) {
  Cand r;
  r.sc = __shfl_xor_sync(0xffffffffu, c.sc, o);
  r.th = __shfl_xor_sync(0xffffffffu, c.th, o);
  r.ord = __shfl_xor_sync(0xffffffffu, c.ord, o);
  r.kind = __shfl_xor_sync(0xffffffffu, c.kind, o);
  r.idx = __shfl_xor_sync(0xffffffffu, c.idx, o);
  return r;
}

// The best candidate of the block (every thread gets it).
__device__ __forceinline__ Cand block_best(Cand c, Cand* buf) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const Cand t = shfl_cand(c, o);
    if (t.beats(c)) c = t;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) buf[w] = c;
  __syncthreads();
  Cand r = buf[0];
  for (int q = 1; q < kSecWarps; ++q)
    if (buf[q].beats(r)) r = buf[q];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int block_min(int v, int* buf) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) buf[w] = v;
  __syncthreads();
  int r = buf[0];
  for (int q = 1; q < kSecWarps; ++q) r = min(r, buf[q]);
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kSecThreads) k_secular(SecularArgs a) {
  extern __shared__ double smem[];
  __shared__ double red[32];
  __shared__ int s_nJ, s_nK, s_m0, s_best, s_best_defl, s_cert, s_list[64], s_nlist;
  __shared__ double s_lower, s_upper;
  __shared__ Cand s_cand[kSecWarps];
  __shared__ int s_imin[kSecWarps];
  namespace cg = cooperative_groups;
  const cg::cluster_group cluster = cg::this_cluster();
  const int cs = a.cs;
  const int rank = cs > 1 ? (int)cluster.block_rank() : 0;
  const int i = blockIdx.x / cs;
  const bool lead = rank == 0;  // the CTA that writes the pair's results
  const int NH = a.NH, ldk = a.ldk;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gwarp = rank * kSecWarps + warp, nwarps = cs * kSecWarps;  // warps of the cluster
  if (!a.active[i]) {
    if (tid == 0 && lead) a.upd[i] = 0;
    return;
  }
  SecShared S;
  S.d = smem;
  S.z = S.d + NH;
  S.cq = S.z + NH;
  S.w = S.cq + NH;
  S.theta = S.w + NH;
  S.orig = S.theta + NH + 1;
  S.tau = S.orig + NH + 1;
  S.sb = S.tau + NH + 1;
  S.J = reinterpret_cast<int*>(S.sb + NH + 1);
  S.K = S.J + NH;
  S.pole = S.K + NH;
  S.rot = S.pole + NH;
  S.solved = S.rot + NH;

  double scc = 0.0, scb = 0.0, sdcc = 0.0;
  for (int j = tid; j < NH; j += kSecThreads) {
    const double dj = a.lamH[j], cj = a.cq[(size_t)j * ldk + i], bj = a.bq[(size_t)j * ldk + i];
    S.d[j] = dj; S.cq[j] = cj; S.z[j] = bj;  // z holds b' until rescaled
    scc = fma(cj, cj, scc); scb = fma(cj, bj, scb); sdcc = fma(dj * cj, cj, sdcc);
  }
  scc = block_sum(scc, red); scb = block_sum(scb, red); sdcc = block_sum(sdcc, red);
  const double beta = a.beta[i], zeta = a.zeta[i];
  const double zt = zeta - scc;
  if (!(zt > 1e-14 * zeta)) {  // u~ numerically inside V_H: keep the pair for this step
    if (tid == 0 && lead) { a.upd[i] = 0; a.status[i] = ST_DEGENERATE; a.steps[i] += 1; }
    return;
  }
  const double sq = sqrt(zt);
  const double rho = (beta - 2.0 * scb + sdcc) / zt;
  double zz = 0.0;
  for (int j = tid; j < NH; j += kSecThreads) {
    const double zj = (S.z[j] - S.d[j] * S.cq[j]) / sq;
    S.z[j] = zj;
    zz = fma(zj, zj, zz);
  }
  zz = block_sum(zz, red);
  const double scale = fmax(fmax(fabs(S.d[NH - 1]), fabs(rho)), sqrt(zz));
  const double tolz = 8.0 * DBL_EPSILON * scale;
  const double lam_prev = a.lam[i];
  if (tid == 0) {
    // poles: indices with |z_j| > tolz.  Two poles closer than told (an exact
    // coarse degeneracy) are merged by a rotation in their plane: the second
    // carries the weight z_a^2 + z_b^2, and the first becomes a deflated root at
    // the same lambda with eigenvector (z_b e_a - z_a e_b) / r.
    const double told = 64.0 * DBL_EPSILON * fabs(S.d[NH - 1]);
    int nJ = 0, nK = 0, m0 = 0;
    bool last_merged = false;
    double zj2 = 0.0, dmin = 0.0, dmax = 0.0;
    for (int j = 0; j < NH; ++j) {
      S.rot[j] = -1;
      S.pole[j] = j;
      if (!(fabs(S.z[j]) > tolz)) continue;
      const double wj = S.z[j] * S.z[j];
      if (nJ > 0 && !last_merged && S.d[j] - S.d[S.J[nJ - 1]] <= told) {
        const int pj = S.J[nJ - 1];
        S.rot[pj] = j;
        S.pole[pj] = j;
        S.w[j] = S.w[pj] + wj;
        S.J[nJ - 1] = j;
        last_merged = true;
      } else {
        S.w[j] = wj;
        S.J[nJ++] = j;
        last_merged = false;
      }
      S.K[nK++] = j;
      zj2 += wj;
    }
    for (int t = 0; t < nJ; ++t) {
      const double dj = S.d[S.J[t]];
      if (t == 0) dmin = dj;
      dmax = dj;
      if (dj < lam_prev) m0 = t + 1;
    }
    const double zn = sqrt(zj2);
    s_nJ = nJ;
    s_nK = nK;
    s_m0 = m0;
    s_lower = (nJ ? fmin(dmin, rho) : rho) - zn;
    s_upper = (nJ ? fmax(dmax, rho) : rho) + zn;
    // phase-1 list: root 0 and a window around the root holding lambda^(l)
    int nl = 0;
    s_list[nl++] = 0;
    const int w = a.window;
    for (int m = max(1, m0 - w); m <= min(nJ, m0 + w); ++m) s_list[nl++] = m;
    if (nl == 1 && nJ == 0) nl = 1;
    s_nlist = nl;
    if (lead) a.steps[i] += 1;
  }
  for (int m = tid; m <= NH; m += kSecThreads) S.solved[m] = 0;
  // every CTA of the cluster is running and initialised before any writes into its shared memory
  if (cs > 1) cluster.sync();
  else __syncthreads();
  const int nJ = s_nJ, nK = s_nK;
  const double lower = s_lower, upper = s_upper;

  for (int phase = 0; phase < 3; ++phase) {
    // phase 0: root 0 and the window around the root holding lambda^(l);
    // phase 1: every root up to m0 + 8; phase 2: every root
    const int mmax = phase == 0 ? -1 : (phase == 1 ? min(nJ, s_m0 + 8) : nJ);
    // a solved root's theta, origin, offset and score go to every CTA of the cluster
    auto solve_and_publish = [&](int m) {
      solve_root(S, nJ, m, rho, lower, upper, lane, a.diag + 2);
      double ny2, yc;
      root_vector_sums(S, nK, m, lane, ny2, yc);
      if (lane == 0) {
        const double sbm = (yc + sq) / sqrt(ny2 + 1.0);
        S.sb[m] = sbm;
        for (int r = 0; r < cs; ++r) {
          if (r == rank) continue;
          *cluster.map_shared_rank(S.theta + m, r) = S.theta[m];
          *cluster.map_shared_rank(S.orig + m, r) = S.orig[m];
          *cluster.map_shared_rank(S.tau + m, r) = S.tau[m];
          *cluster.map_shared_rank(S.sb + m, r) = sbm;
        }
      }
    };
    if (phase == 0) {
      for (int q = gwarp; q < s_nlist; q += nwarps) solve_and_publish(s_list[q]);
    } else {
      // cluster warp w takes the w-th, (w + nwarps)-th, ... unsolved root at or below mmax
      int cnt = 0;
      for (int m = 0; m <= mmax; ++m) {
        if (S.solved[m]) continue;
        if ((cnt++ % nwarps) != gwarp) continue;
        solve_and_publish(m);
      }
    }
    if (cs > 1) cluster.sync();
    else __syncthreads();
    if (phase == 0) {
      for (int q = tid; q < s_nlist; q += kSecThreads) S.solved[s_list[q]] = 1;
    } else {
      for (int m = tid; m <= mmax; m += kSecThreads) S.solved[m] = 1;
    }
    __syncthreads();
    {
      // best candidate among solved roots and deflated poles: each thread scans
      // its share, then a block reduction.  Order of preference: larger score,
      // then smaller theta, then roots before deflated poles, lower index first.
      Cand best;
      best.clear();
      double mass = 0.0;
      int nsolved = 0, m_unsolved = INT_MAX;
      for (int m = tid; m <= nJ; m += kSecThreads) {
        if (!S.solved[m]) { m_unsolved = min(m_unsolved, m); continue; }
        ++nsolved;
        const double sbm = S.sb[m];
        mass += sbm * sbm;
        const double sc = a.score_norm == 0 ? fabs(sbm) / sqrt(S.theta[m]) : fabs(sbm);
        best.offer(sc, S.theta[m], m, 0, m);
      }
      for (int j = tid; j < NH; j += kSecThreads) {
        double sbj, thj;
        int kind;
        if (!(fabs(S.z[j]) > tolz)) {            // plain deflation: eigenvector e_j
          sbj = S.cq[j]; thj = S.d[j]; kind = 1;
        } else if (S.rot[j] >= 0) {             // merged away: (z_b e_j - z_j e_b) / r
          const int b = S.rot[j];
          const double r = sqrt(S.w[b]);
          sbj = (S.z[b] * S.cq[j] - S.z[j] * S.cq[b]) / r; thj = S.d[b]; kind = 2;
        } else {
          continue;
        }
        mass += sbj * sbj;
        const double sc = a.score_norm == 0 ? fabs(sbj) / sqrt(thj) : fabs(sbj);
        best.offer(sc, thj, NH + 1 + j, kind, j);
      }
      best = block_best(best, s_cand);
      mass = block_sum(mass, red);
      const double nsd = block_sum((double)nsolved, red);
      m_unsolved = block_min(m_unsolved, s_imin);
      if (tid == 0) {
        int cert = 1;
        if (m_unsolved != INT_MAX) {
          const double rest = fmax(zeta - mass, 0.0) * (1.0 + 1e-8) + 1e-300;
          double bound;
          if (a.score_norm == 0) {
            // every unsolved root lies above the pole left of the smallest unsolved index
            const double th_lo = m_unsolved > 0 ? S.d[S.J[m_unsolved - 1]] : lower;
            bound = th_lo > 0.0 ? rest / th_lo : INFINITY;
          } else {
            bound = rest;
          }
          cert = best.sc * best.sc > bound;
        }
        if (phase == 0 && lead) atomicAdd(a.diag + 0, (int)nsd);
        s_cert = cert;
        s_best = best.idx;
        s_best_defl = best.kind;
      }
    }
    // every CTA has read its copies before the next phase writes new roots into them
    if (cs > 1) cluster.sync();
    else __syncthreads();
    if (s_cert) break;
    if (tid == 0 && lead) atomicAdd(a.diag + 1, 1);
  }
  if (!lead) return;  // no further access to this CTA's shared memory by the cluster

  // winner -> alpha and coarse coefficients g (Q basis), a-normalised, sign b(u, u~) > 0
  const int bi = s_best;
  if (bi < 0) {  // every score NaN: freeze the pair
    if (tid == 0) { a.upd[i] = 0; a.active[i] = 0; a.status[i] = ST_NAN; }
    return;
  }
  double th, alpha;
  if (s_best_defl == 1) {
    const double sgn = S.cq[bi] >= 0.0 ? 1.0 : -1.0;
    th = S.d[bi];
    alpha = 0.0;
    const double inv = sgn / sqrt(th);
    for (int j = tid; j < NH; j += kSecThreads) a.g[(size_t)j * ldk + i] = (j == bi) ? inv : 0.0;
  } else if (s_best_defl == 2) {
    const int b = S.rot[bi];
    const double r = sqrt(S.w[b]);
    const double va = S.z[b] / r, vb = -S.z[bi] / r;
    const double sbv = va * S.cq[bi] + vb * S.cq[b];
    const double sgn = sbv >= 0.0 ? 1.0 : -1.0;
    th = S.d[b];
    alpha = 0.0;
    const double inv = sgn / sqrt(th);
    for (int j = tid; j < NH; j += kSecThreads)
      a.g[(size_t)j * ldk + i] = (j == bi) ? inv * va : ((j == b) ? inv * vb : 0.0);
  } else {
    th = S.theta[bi];
    double ny2 = 0.0;
    {
      const double origin = S.orig[bi], tau = S.tau[bi];
      double acc = 0.0;
      for (int t = tid; t < nK; t += kSecThreads) {
        const int j = S.K[t];
        const double y = -S.z[j] / ((S.d[S.pole[j]] - origin) - tau);
        acc = fma(y, y, acc);
      }
      ny2 = block_sum(acc, red);
    }
    const double sgn = S.sb[bi] >= 0.0 ? 1.0 : -1.0;
    const double na = sqrt(th) * sqrt(ny2 + 1.0);
    alpha = sgn / (na * sq);
    const double origin = S.orig[bi], tau = S.tau[bi];
    for (int j = tid; j < NH; j += kSecThreads) a.g[(size_t)j * ldk + i] = -alpha * S.cq[j];
    __syncthreads();
    for (int t = tid; t < nK; t += kSecThreads) {
      const int j = S.K[t];
      const double y = -S.z[j] / ((S.d[S.pole[j]] - origin) - tau);
      a.g[(size_t)j * ldk + i] = fma(sgn / na, y, -alpha * S.cq[j]);
    }
  }
  if (tid == 0) {
    if (!isfinite(th) || !isfinite(alpha)) {
      a.upd[i] = 0; a.active[i] = 0; a.status[i] = ST_NAN;
    } else {
      a.lam[i] = th;
      a.alpha[i] = alpha;
      a.upd[i] = 1;
      const double rel = fabs(th - lam_prev) / fabs(th);
      bool res_ok = true;
      if (a.rsum) res_ok = sqrt(a.rsum[i]) <= a.res_tol * sqrt(fabs(lam_prev * a.rsum[a.ldk + i]));
      if (rel < a.tol && res_ok) { a.active[i] = 0; a.status[i] = ST_CONVERGED; }
      else a.status[i] = ST_ACTIVE;
    }
  }
}

static size_t secular_smem(int NH) {
  return sizeof(double) * (4 * (size_t)NH + 4 * ((size_t)NH + 1)) + sizeof(int) * (4 * (size_t)NH + (size_t)NH + 1);
}

cudaError_t secular_prepare(int NH) {
  return allow_dynamic_smem((const void*)k_secular, secular_smem(NH));
}

// CTAs per pair: as many (up to 4) as keep all of them co-resident on the SMs.
static int secular_cluster(int k) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  int cs = 1;
  while (cs < 4 && (size_t)k * (size_t)(cs * 2) <= (size_t)sms) cs *= 2;
  return cs;
}

void secular_select(const Launch& L, const SecularArgs& a0) {
  SecularArgs a = a0;
  a.cs = secular_cluster(a.k);
  L.begin(KC_SECULAR, (double)a.NH * a.ldk * 8.0 * 3.0, 0.0);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.k * a.cs));
  cfg.blockDim = dim3(kSecThreads);
  cfg.dynamicSmemBytes = secular_smem(a.NH);
  cfg.stream = L.s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_secular, a);
  L.bump();
}

}  // namespace pasm
