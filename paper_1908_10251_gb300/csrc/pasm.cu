// C ABI of the GB300 parallel augmented subspace method: context, setup,
// correction step (Algorithm 1 for all pairs at once), solve loop
// (Algorithm 2 on the finest level) and the split entry points.
#include "../../include/pasm.h"
#include "kernels.cuh"
#include "smoother.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <new>
#include <string>
#include <vector>

namespace pasm {
int coarse_generalized_eig(int n, const double* A, const double* M, double* lam, double* Q);

struct Tracer {
  struct Rec { int cls; double bytes, flops; int e0, e1; int rows; };
  std::vector<cudaEvent_t> ev;
  std::vector<Rec> recs;
  size_t used = 0;
  int next_rows = 0;  // rows of the next launch (set by the launcher via tracer_rows)
  int get() {
    if (used == ev.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev.push_back(e);
    }
    return (int)used++;
  }
  ~Tracer() { for (auto e : ev) cudaEventDestroy(e); }
};
void tracer_begin(Tracer* t, cudaStream_t s, int cls, double bytes, double flops) {
  const int e0 = t->get();
  cudaEventRecord(t->ev[(size_t)e0], s);
  t->recs.push_back({cls, bytes, flops, e0, -1, t->next_rows});
  t->next_rows = 0;
}
void tracer_rows(Tracer* t, int rows) { t->next_rows = rows; }
void tracer_end(Tracer* t, cudaStream_t s) {
  if (t->recs.empty() || t->recs.back().e1 >= 0) return;
  const int e1 = t->get();
  cudaEventRecord(t->ev[(size_t)e1], s);
  t->recs.back().e1 = e1;
}
}  // namespace pasm
using namespace pasm;

namespace {

struct LevelDev {
  int n = 0;
  DCsr A, M;       // level stiffness and mass
  DCsr P, R;       // (l >= 1) P: level l-1 -> l, R = P^T
  DCsr RA;         // (l >= 1, mixed precision) R A: the restriction-first residual of the float32 cycles
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  void* vF = nullptr;  // V-cycle right-hand side (precision of the cycle)
  void* vE = nullptr;  // V-cycle iterate
  void* vT = nullptr;  // V-cycle temporary
  double* BA = nullptr;  // float64 chain buffers (restriction of A u~, prolongation of u_H)
  double* BM = nullptr;  // float64 chain buffer (restriction of M u~)
  void* vP = nullptr;    // CG smoothing: search directions and their images (cycle precision)
  void* vQ = nullptr;
};

}  // namespace

struct pasm_ctx {
  int nlev = 0;
  std::vector<LevelDev> lv;
  pasm_opts opts{};
  cudaStream_t s = nullptr;
  cudaStream_t user = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int NH = 0;
  std::vector<double> h_lamH, h_Q;
  double* lamH = nullptr;
  double* Q = nullptr;
  double* AinvH64 = nullptr;
  float* AinvH32 = nullptr;
  std::vector<void*> allocs;     // setup-lifetime device allocations
  std::vector<void*> kallocs;    // k-dependent device allocations
  // pair state (k-dependent)
  int k = 0, ldk = 0;
  double tol = 0.0;
  double *U = nullptr, *Fd = nullptr, *X = nullptr, *YA = nullptr, *YM = nullptr;
  double* Uff = nullptr;  // mixed precision: U split into (hi, lo) float pairs for the gathers
  double *lam = nullptr, *lam2 = nullptr, *alpha = nullptr, *bz = nullptr, *bq = nullptr, *cq = nullptr,
         *g = nullptr, *uH = nullptr, *partials = nullptr;
  double* rsum = nullptr;  // 2 x ldk: residual sums of the state a step starts from (opts.res_tol > 0)
  int *active = nullptr, *upd = nullptr, *steps = nullptr, *status = nullptr, *nact = nullptr, *diag = nullptr;
  int *active2 = nullptr, *steps2 = nullptr, *status2 = nullptr;
  int* h_nact = nullptr;  // pinned
  int max_border_blocks = 152 * 8;
  cudaGraphExec_t graph = nullptr;
  Tracer* tracer = nullptr;  // set only inside pasm_trace_step
  // learned post-smoother
  struct {
    bool ready = false;
    std::vector<int> nx, ny;                 // grid view per level (0 = none)
    float *W = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    int t = 0;
    NNBuf buf;                               // activations, capacity buf.cap pixel-pairs
    int64_t vcap = 0;                        // capacity of the n x ldk temporaries
    int64_t bcap = 0;                        // capacity of the backward activations
    float *R = nullptr, *D = nullptr, *X = nullptr, *Rt = nullptr, *Es = nullptr, *gD = nullptr;
    double *partial = nullptr, *norms = nullptr, *loss = nullptr;
    int* accepted = nullptr;
    int* err = nullptr;                      // timed-out tensor-core waits
    NNOuterWeights w13{};                    // host copy of layers 1 and 3 (kernel parameters)
    uint16_t* w2 = nullptr;                  // layer 2 as bf16 in the tensor-core operand layout
    uint16_t *w2f = nullptr, *w2t = nullptr; // training: forward and flipped layouts, rebuilt per step
    std::vector<void*> allocs;
  } nn;
  int capture_level = -1;        // residual capture for training data (pasm_nn_capture_residuals)
  float* capture_buf = nullptr;
  // test hook of the projection's bounded completion wait (pasm_debug_waits)
  int dbg_wait_limit = 0, dbg_skip_mma = 0;
  // float64-accurate coarse projections on the tensor cores: Q^T (b, c) and Q g
  bool proj_tc = false;
  SplitMat projQT, projQ;
  int* proj_err = nullptr;                 // timed-out tensor-core waits of the projection kernel
  unsigned long long* proj_hl = nullptr;   // integer sums of the projection (k-dependent scratch)
  unsigned int* proj_tickets = nullptr;
  CgWork cg;                               // CG smoothing: partial sums and per-column scalars
  // autotuned row-group geometry per level and kernel kind (0 = default), for block width tuned_ldk
  std::vector<std::array<int, PASM_TILE_N>> geo;
  std::vector<std::array<int, PASM_TILE_N>> rpt;   // row blocks per block (0 = by size)
  int tuned_ldk = 0;
  int launches = 0;
  int last_launches = 0;
  bool initialized = false;
  // mixed precision: the steps keep the state in Uff (pairs) only, so U (float64)
  // is out of date after a step until sync_state rebuilds it
  bool u_stale = false;
};

extern "C" {
static int nn_ensure(pasm_ctx* c, int64_t pixpairs, int64_t vecs, bool backward);
}

namespace {

#define CK(call)                                              \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) {                                  \
      std::fprintf(stderr, "pasm: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(_e), __FILE__, __LINE__); \
      return PASM_ECUDA;                                      \
    }                                                         \
  } while (0)

template <typename T>
int dalloc(std::vector<void*>& list, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) { cudaGetLastError(); return PASM_ENOMEM; }
  list.push_back(*p);
  return PASM_OK;
}
#define AL(list, p, count) do { int _r = dalloc(list, p, count); if (_r) return _r; } while (0)

int check_csr(const pasm_csr& m, int rows, int cols) {
  if (m.n_rows != rows || m.n_cols != cols || m.nnz < 0 || !m.row_ptr) return PASM_EINVAL;
  if (m.nnz > 0 && (!m.col || !m.val)) return PASM_EINVAL;
  if (m.nnz > 2147483647LL) return PASM_EINVAL;
  if (m.row_ptr[0] != 0 || m.row_ptr[rows] != m.nnz) return PASM_EINVAL;
  for (int i = 0; i < rows; ++i)
    if (m.row_ptr[i + 1] < m.row_ptr[i]) return PASM_EINVAL;
  for (int64_t p = 0; p < m.nnz; ++p)
    if (m.col[p] < 0 || m.col[p] >= cols) return PASM_EINVAL;
  return PASM_OK;
}

int upload_csr(pasm_ctx* c, const pasm_csr& h, DCsr& d, bool shadow32, bool split_ff) {
  d.n_rows = h.n_rows; d.n_cols = h.n_cols; d.nnz = h.nnz;
  AL(c->allocs, &d.rp, (size_t)h.n_rows + 1);
  AL(c->allocs, &d.ci, (size_t)h.nnz);
  AL(c->allocs, &d.v64, (size_t)h.nnz);
  CK(cudaMemcpy(d.rp, h.row_ptr, sizeof(int) * ((size_t)h.n_rows + 1), cudaMemcpyHostToDevice));
  if (h.nnz) {
    CK(cudaMemcpy(d.ci, h.col, sizeof(int) * (size_t)h.nnz, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.v64, h.val, sizeof(double) * (size_t)h.nnz, cudaMemcpyHostToDevice));
  }
  if (shadow32) {
    AL(c->allocs, &d.v32, (size_t)h.nnz);
    std::vector<float> f(h.val, h.val + h.nnz);
    if (h.nnz) CK(cudaMemcpy(d.v32, f.data(), sizeof(float) * (size_t)h.nnz, cudaMemcpyHostToDevice));
  }
  if (split_ff) {
    // hi = nearest float, lo = nearest float of the remainder (about 48 bits).  A matrix whose
    // low parts are all below 2^-48 of their high parts (float32 values, or values assembled with a
    // few ulps of float64 rounding, as the constant-coefficient stiffness) is marked exact32 and its
    // low parts are dropped: they lie below the double-float products' own rounding (2^-46).
    AL(c->allocs, &d.vff, (size_t)h.nnz);
    std::vector<float2> f((size_t)h.nnz);
    d.exact32 = true;
    for (int64_t q = 0; q < h.nnz; ++q) {
      const float hi = (float)h.val[q];
      f[(size_t)q] = make_float2(hi, (float)(h.val[q] - (double)hi));
      if (!(std::fabs((double)f[(size_t)q].y) <= std::ldexp(std::fabs((double)hi), -48))) d.exact32 = false;
    }
    if (d.exact32)
      for (auto& v : f) v.y = 0.f;
    if (h.nnz) CK(cudaMemcpy(d.vff, f.data(), sizeof(float2) * (size_t)h.nnz, cudaMemcpyHostToDevice));
  }
  return PASM_OK;
}

// Host sparse product C = S B (CSR, columns ascending per row; row-by-row accumulation into a dense
// marker row, Gustavson's method).  Values in float64, products summed in S's column order.
void multiply_csr(const std::vector<int32_t>& srp, const std::vector<int32_t>& sci, const std::vector<double>& sv,
                  int s_rows, const pasm_csr& b, std::vector<int32_t>& rp, std::vector<int32_t>& ci,
                  std::vector<double>& v) {
  rp.assign((size_t)s_rows + 1, 0);
  ci.clear();
  v.clear();
  std::vector<int32_t> mark((size_t)b.n_cols, -1);
  std::vector<double> acc((size_t)b.n_cols, 0.0);
  std::vector<int32_t> cols;
  for (int i = 0; i < s_rows; ++i) {
    cols.clear();
    for (int q = srp[(size_t)i]; q < srp[(size_t)i + 1]; ++q) {
      const int j = sci[(size_t)q];
      for (int64_t t = b.row_ptr[j]; t < b.row_ptr[j + 1]; ++t) {
        const int col = b.col[t];
        if (mark[(size_t)col] != i) {
          mark[(size_t)col] = i;
          acc[(size_t)col] = 0.0;
          cols.push_back(col);
        }
        acc[(size_t)col] += sv[(size_t)q] * b.val[t];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int col : cols) {
      ci.push_back(col);
      v.push_back(acc[(size_t)col]);
    }
    rp[(size_t)i + 1] = (int32_t)ci.size();
  }
}

// Host CSR transpose (R = P^T), columns ascending.
void transpose_csr(const pasm_csr& p, std::vector<int32_t>& rp, std::vector<int32_t>& ci, std::vector<double>& v) {
  rp.assign((size_t)p.n_cols + 1, 0);
  for (int64_t q = 0; q < p.nnz; ++q) rp[(size_t)p.col[q] + 1]++;
  for (int j = 0; j < p.n_cols; ++j) rp[(size_t)j + 1] += rp[j];
  ci.resize((size_t)p.nnz);
  v.resize((size_t)p.nnz);
  std::vector<int32_t> pos(rp.begin(), rp.end() - 1);
  for (int i = 0; i < p.n_rows; ++i)
    for (int q = p.row_ptr[i]; q < p.row_ptr[i + 1]; ++q) {
      const int j = p.col[q];
      ci[(size_t)pos[j]] = i;
      v[(size_t)pos[j]] = p.val[q];
      pos[j]++;
    }
}

int ldk_for(int k) {
  int l = 4;
  while (l < k) l <<= 1;
  return l;
}

struct Scope {  // order the context stream after the caller's stream and back
  pasm_ctx* c;
  explicit Scope(pasm_ctx* ctx) : c(ctx) {
    cudaEventRecord(c->ev_in, c->user);
    cudaStreamWaitEvent(c->s, c->ev_in, 0);
  }
  ~Scope() {
    cudaEventRecord(c->ev_out, c->s);
    cudaStreamWaitEvent(c->user, c->ev_out, 0);
  }
};

Launch launcher(pasm_ctx* c) {
  Launch L;
  L.s = c->s;
  L.counter = &c->launches;
  L.tr = c->tracer;
  return L;
}

// launcher with the autotuned geometry of kernel kind `kind` on level l
Launch launcher(pasm_ctx* c, int l, int kind) {
  Launch L = launcher(c);
  if (l >= 0 && l < (int)c->geo.size()) {
    L.geo = c->geo[(size_t)l][(size_t)kind];
    L.rpt = c->rpt[(size_t)l][(size_t)kind];
  }
  return L;
}

// ------------------------------------------------------------------------------------------------
// Multigrid V-cycle for A_l E = F_l from a zero guess; returns the buffer holding E.
template <typename T> const T* ainv(pasm_ctx* c);
template <> const double* ainv<double>(pasm_ctx* c) { return c->AinvH64; }
template <> const float* ainv<float>(pasm_ctx* c) { return c->AinvH32; }
template <typename T> const T* dinv(const LevelDev& v);
template <> const double* dinv<double>(const LevelDev& v) { return v.dinv64; }
template <> const float* dinv<float>(const LevelDev& v) { return v.dinv32; }

// float32 cycles use the fused kernels (HBM passes dominate); float64 cycles keep
// the plain ones (FP64 arithmetic dominates on GB300 and fusion recomputes).
template <typename T> struct Fused { static constexpr bool on = false; };
template <> struct Fused<float> { static constexpr bool on = true; };

// Hooks before float32 post-smoothing on level l (cur = iterate after the
// coarse correction, tmp = free buffer): the residual capture for training
// data, and the learned smoothing step with its per-pair Jacobi fallback.
// Returns the number of post-smoothing sweeps done (0 or 1; 1 = result in tmp).
int post_hooks(pasm_ctx* c, int l, float* cur, float* tmp, float* F) {
  const Launch L = launcher(c);
  LevelDev& v = c->lv[l];
  const int ldk = c->ldk;
  if (c->capture_level == l && c->capture_buf) {
    rowop<float>(L, OP_RESID, v.A, cur, F, nullptr, nullptr, 0.f, c->capture_buf, ldk);
    c->capture_level = -1;
  }
  if (c->opts.smoother != PASM_LEARNED || !c->nn.ready || c->nn.nx[l] == 0 || c->opts.nu_post < 1) return 0;
  auto& nn = c->nn;
  NNGrid g{nn.nx[l], nn.ny[l], ldk, c->k};
  const float om = (float)c->opts.omega;
  rowop<float>(L, OP_RESID, v.A, cur, F, nullptr, nullptr, om, nn.R, ldk);        // r = f - A e
  if (nn_tc_supported(ldk)) nn_forward_tc(L, g, nn.w13, nn.w2, nn.R, nn.D, nn.err);        // d = N(r), tensor cores
  else nn_forward(L, g, nn.buf, nn.W, nn.R, nn.D);
  rowop<float>(L, OP_RESID, v.A, nn.D, nn.R, nullptr, nullptr, om, nn.Rt, ldk);   // f - A (e + d) = r - A d
  nn_column_norms(L, v.n, ldk, nn.R, nn.Rt, nn.partial, nn.norms);
  nn_select(L, v.n, ldk, cur, nn.D, nn.R, v.dinv32, om, nn.norms, tmp, nn.accepted);
  return 1;
}

// Top-level output of a mixed-precision V-cycle: the last post-smoothing sweep
// writes X = B + e directly (double-float pairs) instead of e.
struct TopOut {
  const double* B;
  bool b_ff;
  double* X;
};

template <typename T>
T* vcycle(pasm_ctx* c, int l, const TopOut* top = nullptr) {
  const Launch L = launcher(c);
  LevelDev& v = c->lv[l];
  T* F = (T*)v.vF;
  T* E = (T*)v.vE;
  T* Tm = (T*)v.vT;
  const int ldk = c->ldk;
  if (l == 0) {
    dense_mm<T>(L, c->NH, c->NH, ainv<T>(c), c->NH, false, F, E, ldk);
    return E;
  }
  const T om = (T)c->opts.omega;
  const bool fuse = Fused<T>::on;
  T* cur = E;
  T* tmp = Tm;
  int s = 0;
  const bool cg = c->opts.smoother == PASM_CG;
  // a fused kernel whose tile entry is -1 was timed slower than its unfused pair on this level
  if (cg && c->opts.nu_pre >= 1) {
    cg_smooth<T>(L, v.A, F, cur, true, tmp, (T*)v.vP, (T*)v.vQ, c->cg, ldk, c->opts.nu_pre);
    s = c->opts.nu_pre;
  } else if (cg) {
    cudaMemsetAsync(cur, 0, sizeof(T) * (size_t)v.n * ldk, c->s);
  } else if (fuse && c->opts.nu_pre >= 2 && c->geo[(size_t)l][PASM_TILE_JACOBI2_ZERO] >= 0) {
    jacobi2_zero<T>(launcher(c, l, PASM_TILE_JACOBI2_ZERO), v.A, dinv<T>(v), om, F, cur, ldk);
    s = 2;
  } else if (c->opts.nu_pre >= 1) {
    jacobi_zero<T>(L, v.n, dinv<T>(v), om, F, cur, ldk);
    s = 1;
  } else {
    cudaMemsetAsync(cur, 0, sizeof(T) * (size_t)v.n * ldk, c->s);
  }
  for (; s < c->opts.nu_pre; ++s) {
    rowop<T>(launcher(c, l, PASM_TILE_JACOBI), OP_JACOBI, v.A, cur, F, cur, dinv<T>(v), om, tmp, ldk);
    std::swap(cur, tmp);
  }
  bool restricted = false;
  if constexpr (std::is_same<T, float>::value) {
    if (fuse && v.RA.rp && c->geo[(size_t)l][PASM_TILE_RESTRICT_FIRST] > 0) {
      restrict_first(launcher(c, l, PASM_TILE_RESTRICT_FIRST), v.R, v.RA, cur, F, (float*)c->lv[l - 1].vF, ldk);
      restricted = true;
    }
  }
  if (!restricted && fuse && c->geo[(size_t)l][PASM_TILE_RESID_RESTRICT] >= 0) {
    resid_restrict<T>(launcher(c, l, PASM_TILE_RESID_RESTRICT), v.R, v.A, cur, F, (T*)c->lv[l - 1].vF, ldk);
  } else if (!restricted) {
    rowop<T>(launcher(c, l, PASM_TILE_RESID), OP_RESID, v.A, cur, F, nullptr, nullptr, om, tmp, ldk);
    rowop<T>(launcher(c, l, PASM_TILE_RESTRICT), OP_SPMM, v.R, tmp, nullptr, nullptr, nullptr, om,
             (T*)c->lv[l - 1].vF, ldk);
  }
  T* ec = vcycle<T>(c, l - 1);
  // float32 Jacobi post-smoothing: the prolongation and the first sweep in one kernel, unless the
  // autotuner timed the pair faster, the first sweep is the top level's fused last sweep, or the
  // level runs the learned step or captures training data before its first sweep
  const bool fuse_ps = Fused<T>::on && !cg && c->geo[(size_t)l][PASM_TILE_PROLONG_SWEEP] >= 0 &&
                       (c->opts.nu_post >= 2 || (c->opts.nu_post == 1 && !top)) && c->capture_level != l &&
                       !(c->opts.smoother == PASM_LEARNED && c->nn.ready && c->nn.nx[(size_t)l] != 0);
  if (fuse_ps) {
    prolong_jacobi(launcher(c, l, PASM_TILE_PROLONG_SWEEP), v.A, v.P, (const float*)cur, (const float*)ec,
                   (const float*)F, v.dinv32, (float)om, (float*)tmp, ldk);
    std::swap(cur, tmp);
  } else {
    rowop<T>(launcher(c, l, PASM_TILE_PROLONG), OP_SPMM_ADD, v.P, ec, cur, nullptr, nullptr, om, cur, ldk);
  }
  if (cg) {
    cg_smooth<T>(L, v.A, F, cur, false, tmp, (T*)v.vP, (T*)v.vQ, c->cg, ldk, c->opts.nu_post);
    return cur;
  }
  s = fuse_ps ? 1 : 0;
  if (Fused<T>::on && !fuse_ps) s = post_hooks(c, l, (float*)cur, (float*)tmp, (float*)F);
  if (s == 1 && !fuse_ps) std::swap(cur, tmp);
  for (; s < c->opts.nu_post; ++s) {
    if (Fused<T>::on && top && s == c->opts.nu_post - 1) {
      // last sweep fused with the outer update; the cycle's result is in top->X
      jacobi_axpy_ff(launcher(c, l, PASM_TILE_JACOBI), v.A, (const float*)cur, (const float*)F, v.dinv32, (float)om,
                     top->B, top->b_ff, top->X, ldk);
      return nullptr;
    }
    rowop<T>(launcher(c, l, PASM_TILE_JACOBI), OP_JACOBI, v.A, cur, F, cur, dinv<T>(v), om, tmp, ldk);
    std::swap(cur, tmp);
  }
  return cur;
}

// Algorithm 1 step 1 on level lt: X = result of the V-cycles for A x = lam M U from x = U,
// each cycle a defect correction x += V(f - A x) with f = lam M U (float64 residual).
template <typename T>
void bvp_impl(pasm_ctx* c, int lt, const double* lam, const double* U, double* X, bool u_split) {
  const Launch L = launcher(c);
  LevelDev& v = c->lv[lt];
  T* Ftop = (T*)v.vF;
  if (Fused<T>::on) {
    // double-float outer residuals; X (the result u~) is left in (hi, lo) pairs
    if (!u_split) to_ff(L, (int64_t)v.n * c->ldk, U, c->Uff);
    outer_rhs_residual_ff(launcher(c, lt, PASM_TILE_OUTER_RHS), v.A, v.M, lam, c->Uff, c->Fd, (float*)Ftop, c->ldk);
    if (c->opts.res_tol > 0.0 && lt == c->nlev - 1) {  // the starting state's residual, for the freeze test
      const int nb = residual_partials<float>(L, v.n, c->ldk, (const float*)Ftop, true, c->Fd, c->Uff, c->partials,
                                              c->max_border_blocks);
      column_sums(L, c->partials, nb, 2, c->ldk, c->rsum);
    }
    // x = u + e reads u from its pair copy (in a step the state lives there alone)
    const TopOut first{c->Uff, true, X};
    T* e = vcycle<T>(c, lt, lt >= 1 ? &first : nullptr);
    if (e) axpy_ff(L, v.n, c->Uff, true, (const float*)e, X, c->ldk);
    for (int cyc = 1; cyc < c->opts.cycles_per_step; ++cyc) {
      outer_residual_ff(launcher(c, lt, PASM_TILE_OUTER_RES), v.A, c->Fd, X, (float*)Ftop, c->ldk);
      const TopOut next{X, true, X};
      e = vcycle<T>(c, lt, lt >= 1 ? &next : nullptr);
      if (e) axpy_ff(L, v.n, X, true, (const float*)e, X, c->ldk);
    }
    return;
  }
  outer_rhs_residual<T>(launcher(c, lt, PASM_TILE_OUTER_RHS), v.A, v.M, lam, U, c->Fd, Ftop, c->ldk);
  if (c->opts.res_tol > 0.0 && lt == c->nlev - 1) {
    const int nb = residual_partials<T>(L, v.n, c->ldk, Ftop, false, c->Fd, U, c->partials, c->max_border_blocks);
    column_sums(L, c->partials, nb, 2, c->ldk, c->rsum);
  }
  T* e = vcycle<T>(c, lt);
  outer_axpy<T>(L, v.n, U, e, X, c->ldk);
  for (int cyc = 1; cyc < c->opts.cycles_per_step; ++cyc) {
    outer_residual<T>(launcher(c, lt, PASM_TILE_OUTER_RES), v.A, c->Fd, X, Ftop, c->ldk);
    e = vcycle<T>(c, lt);
    outer_axpy<T>(L, v.n, X, e, X, c->ldk);
  }
}

// u_split: c->Uff already holds U in pairs (the state U of a step: the update of
// the previous step, or pasm_init, wrote it); otherwise it is formed here.
void bvp(pasm_ctx* c, int lt, const double* lam, const double* U, double* X, bool u_split = false) {
  if (c->opts.precision == PASM_MIXED) bvp_impl<float>(c, lt, lam, U, X, u_split);
  else bvp_impl<double>(c, lt, lam, U, X, u_split);
}

struct PairState {
  double* lam;
  int* active;
  int* steps;
  int* status;
  double* Uout;
  double tol;
};

// Projection onto the coarse eigenbasis, b' = Q^T b and c' = Q^T c for all
// columns (tensor cores, float64-accurate, or float64 CUDA cores).
void project_bc(pasm_ctx* c, const Launch& L, const double* b, const double* cc, double* bq, double* cq) {
  if (c->proj_tc) {
    proj_tc(L, c->projQT, b, cc, bq, cq, c->ldk, 2 * c->ldk, c->proj_hl, c->proj_tickets, c->proj_err,
            c->dbg_wait_limit, c->dbg_skip_mma);
  } else {
    dense_mm<double>(L, c->NH, c->NH, c->Q, c->NH, true, b, bq, c->ldk);
    dense_mm<double>(L, c->NH, c->NH, c->Q, c->NH, true, cc, cq, c->ldk);
  }
}

// Algorithm 1 step 2 on level lt for the columns of X: bordering, projection,
// secular solve and selection, and the update Uout = alpha X + P_c u_H.
void augmented(pasm_ctx* c, int lt, const double* X, const PairState& ps) {
  const Launch L = launcher(c);
  LevelDev& v = c->lv[lt];
  const int ldk = c->ldk;
  const bool ff = c->opts.precision == PASM_MIXED;
  const Launch Lb = launcher(c, lt, PASM_TILE_BORDER);
  const int nb = ff ? border_products_ff(Lb, v.A, v.M, X, c->YA, c->YM, c->partials, ldk, c->max_border_blocks)
                    : border_products(Lb, v.A, v.M, X, c->YA, c->YM, c->partials, ldk, c->max_border_blocks);
  column_sums(L, c->partials, nb, 2, ldk, c->bz);
  const double* sa = c->YA;
  const double* sm = c->YM;
  for (int l = lt; l >= 1; --l) {
    if (ff) {
      // pairs down to level 1, float64 on the coarse level for the projection
      const Launch Lr = launcher(c, l, PASM_TILE_CHAIN_R);
      spmm2_ff(Lr, c->lv[l].R, sa, sm, true, c->lv[l - 1].BA, c->lv[l - 1].BM, l - 1 >= 1, ldk);
    } else {
      const Launch Lr = launcher(c, l, PASM_TILE_CHAIN_R);
      rowop<double>(Lr, OP_SPMM, c->lv[l].R, sa, nullptr, nullptr, nullptr, 0.0, c->lv[l - 1].BA, ldk);
      rowop<double>(Lr, OP_SPMM, c->lv[l].R, sm, nullptr, nullptr, nullptr, 0.0, c->lv[l - 1].BM, ldk);
    }
    sa = c->lv[l - 1].BA;
    sm = c->lv[l - 1].BM;
  }
  project_bc(c, L, sa, sm, c->bq, c->cq);
  SecularArgs a;
  a.NH = c->NH; a.k = c->k; a.ldk = ldk;
  a.lamH = c->lamH; a.bq = c->bq; a.cq = c->cq;
  a.beta = c->bz; a.zeta = c->bz + ldk;
  a.lam = ps.lam; a.alpha = c->alpha; a.g = c->g;
  a.active = ps.active; a.upd = c->upd; a.steps = ps.steps; a.status = ps.status;
  a.tol = ps.tol; a.score_norm = c->opts.score_norm; a.window = 3; a.diag = c->diag;
  if (c->opts.res_tol > 0.0 && lt == c->nlev - 1) {
    a.rsum = c->rsum;
    a.res_tol = c->opts.res_tol;
  }
  secular_select(L, a);
  if (c->proj_tc)
    proj_tc(L, c->projQ, c->g, nullptr, c->uH, nullptr, ldk, ldk, c->proj_hl, c->proj_tickets, c->proj_err,
            c->dbg_wait_limit, c->dbg_skip_mma);
  else
    dense_mm<double>(L, c->NH, c->NH, c->Q, c->NH, false, c->g, c->uH, ldk);
  const double* w = c->uH;
  bool w_ff = false;
  for (int l = 1; l < lt; ++l) {
    const Launch Lp = launcher(c, l, PASM_TILE_CHAIN_P);
    if (ff) spmm_ff(Lp, c->lv[l].P, w, w_ff, c->lv[l].BA, true, ldk);
    else rowop<double>(Lp, OP_SPMM, c->lv[l].P, w, nullptr, nullptr, nullptr, 0.0, c->lv[l].BA, ldk);
    w = c->lv[l].BA;
    w_ff = ff;
  }
  const Launch Lu = launcher(c, lt, PASM_TILE_UPDATE);
  // the finest-level state update of a mixed-precision step writes the pair copy of U only (the
  // next step's gathers read it); the float64 U is refreshed from it when read (sync_state)
  const bool state_pairs = ff && ps.Uout == c->U && lt == c->nlev - 1;
  if (ff) update_pairs_ff(Lu, lt >= 1 ? &v.P : nullptr, v.n, w, w_ff, X, c->alpha, c->upd,
                          state_pairs ? nullptr : ps.Uout, state_pairs ? c->Uff : nullptr, ldk);
  else if (lt >= 1) update_pairs(Lu, v.P, w, X, c->alpha, c->upd, ps.Uout, ldk);
  else update_pairs_identity(Lu, v.n, w, X, c->alpha, c->upd, ps.Uout, ldk);
}

// One correction step for all active pairs on the finest level.
void step_body(pasm_ctx* c) {
  const int lt = c->nlev - 1;
  bvp(c, lt, c->lam, c->U, c->X, true);
  PairState ps{c->lam, c->active, c->steps, c->status, c->U, c->tol};
  augmented(c, lt, c->X, ps);
  count_active(launcher(c), c->active, c->k, c->nact);
  cudaMemcpyAsync(c->h_nact, c->nact, sizeof(int), cudaMemcpyDeviceToHost, c->s);
}

void free_k(pasm_ctx* c) {
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  for (void* p : c->kallocs) cudaFree(p);
  c->kallocs.clear();
  for (auto& v : c->lv) { v.vF = v.vE = v.vT = nullptr; v.BA = v.BM = nullptr; v.vP = v.vQ = nullptr; }
  c->initialized = false;
  c->k = 0;
}

// The k-dependent buffers.  A re-initialisation with the same k keeps them and
// the captured step graph (whose kernels take k and these pointers); only the
// state below is cleared again.
int alloc_k(pasm_ctx* c, int k) {
  const bool reuse = !c->kallocs.empty() && c->k == k;
  const size_t ldk = (size_t)ldk_for(k);
  const size_t n = (size_t)c->lv.back().n;
  const size_t nh = (size_t)c->NH * ldk;
  const bool mixed = c->opts.precision == PASM_MIXED;
  if (reuse) {
    c->initialized = false;
  } else {
  free_k(c);
  c->k = k;
  c->ldk = (int)ldk;
  auto& K = c->kallocs;
  AL(K, &c->U, n * ldk); AL(K, &c->Fd, n * ldk); AL(K, &c->X, n * ldk);
  AL(K, &c->YA, n * ldk); AL(K, &c->YM, n * ldk);
  if (c->opts.precision == PASM_MIXED) AL(K, &c->Uff, n * ldk);
  for (int l = 0; l < c->nlev; ++l) {
    LevelDev& v = c->lv[l];
    const size_t m = (size_t)v.n * ldk;
    if (mixed) {
      float *a, *b, *t;
      AL(K, &a, m); AL(K, &b, m); AL(K, &t, m);
      v.vF = a; v.vE = b; v.vT = t;
    } else {
      double *a, *b, *t;
      AL(K, &a, m); AL(K, &b, m); AL(K, &t, m);
      v.vF = a; v.vE = b; v.vT = t;
    }
    if (l < c->nlev - 1) { AL(K, &v.BA, m); AL(K, &v.BM, m); }
    if (c->opts.smoother == PASM_CG && l >= 1) {
      if (mixed) { float *p, *q; AL(K, &p, m); AL(K, &q, m); v.vP = p; v.vQ = q; }
      else { double *p, *q; AL(K, &p, m); AL(K, &q, m); v.vP = p; v.vQ = q; }
    }
  }
  AL(K, &c->lam, ldk); AL(K, &c->lam2, ldk); AL(K, &c->alpha, ldk); AL(K, &c->bz, 2 * ldk);
  AL(K, &c->rsum, 2 * ldk);
  CK(cudaMemset(c->rsum, 0, sizeof(double) * 2 * ldk));  // zero sums pass the guard
  AL(K, &c->bq, nh); AL(K, &c->cq, nh); AL(K, &c->g, nh); AL(K, &c->uH, nh);
  AL(K, &c->partials, (size_t)c->max_border_blocks * 2 * ldk);
  AL(K, &c->active, ldk); AL(K, &c->upd, ldk); AL(K, &c->steps, ldk); AL(K, &c->status, ldk);
  AL(K, &c->active2, ldk); AL(K, &c->steps2, ldk); AL(K, &c->status2, ldk);
  AL(K, &c->nact, 1); AL(K, &c->diag, 8);
  if (c->opts.smoother == PASM_CG) {
    c->cg.max_blocks = 152 * 8;
    AL(K, &c->cg.partial, (size_t)c->cg.max_blocks * ldk);
    AL(K, &c->cg.rr, ldk); AL(K, &c->cg.alpha, ldk); AL(K, &c->cg.beta, ldk);
  }
  if (c->proj_tc) {
    AL(K, &c->proj_hl, proj_scratch_words(c->NH, 2 * (int)ldk));
    AL(K, &c->proj_tickets, proj_tickets(c->NH, 2 * (int)ldk));
  }
  }  // allocation
  if (c->proj_tc) {
    const size_t words = proj_scratch_words(c->NH, 2 * (int)ldk), tickets = proj_tickets(c->NH, 2 * (int)ldk);
    CK(cudaMemsetAsync(c->proj_hl, 0, sizeof(unsigned long long) * words, c->s));
    CK(cudaMemsetAsync(c->proj_tickets, 0, sizeof(unsigned int) * tickets, c->s));
  }
  for (double* z : {c->bq, c->cq, c->g, c->uH}) CK(cudaMemsetAsync(z, 0, sizeof(double) * nh, c->s));
  CK(cudaMemsetAsync(c->U, 0, sizeof(double) * n * ldk, c->s));
  CK(cudaMemsetAsync(c->X, 0, sizeof(double) * n * ldk, c->s));
  CK(cudaMemsetAsync(c->diag, 0, sizeof(int) * 8, c->s));
  return PASM_OK;
}

int set_active(pasm_ctx* c, int* active, int* steps, int* status) {
  std::vector<int> h((size_t)c->ldk, 0);
  for (int i = 0; i < c->k; ++i) h[(size_t)i] = 1;
  CK(cudaMemcpyAsync(active, h.data(), sizeof(int) * c->ldk, cudaMemcpyHostToDevice, c->s));
  CK(cudaMemsetAsync(steps, 0, sizeof(int) * c->ldk, c->s));
  CK(cudaMemsetAsync(status, 0, sizeof(int) * c->ldk, c->s));
  CK(cudaStreamSynchronize(c->s));
  return PASM_OK;
}

// Copy an n x k user block (host or device, leading dim k) into an n x ldk device block.
// Block copies between the caller's [n][k] array and the [n][ldk] device block.
// When k == ldk the rows are contiguous on both sides and one linear copy moves
// the block (a pitched copy of n short rows runs far below the link's rate).
int put_block(pasm_ctx* c, const double* src, double* dst, int n) {
  if (c->k == c->ldk) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n * c->k, cudaMemcpyDefault, c->s));
    return PASM_OK;
  }
  CK(cudaMemsetAsync(dst, 0, sizeof(double) * (size_t)n * c->ldk, c->s));
  CK(cudaMemcpy2DAsync(dst, sizeof(double) * c->ldk, src, sizeof(double) * c->k, sizeof(double) * c->k, n,
                       cudaMemcpyDefault, c->s));
  return PASM_OK;
}
int get_block(pasm_ctx* c, const double* src, double* dst, int n) {
  if (c->k == c->ldk) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n * c->k, cudaMemcpyDefault, c->s));
    return PASM_OK;
  }
  CK(cudaMemcpy2DAsync(dst, sizeof(double) * c->k, src, sizeof(double) * c->ldk, sizeof(double) * c->k, n,
                       cudaMemcpyDefault, c->s));
  return PASM_OK;
}
int put_lambda(pasm_ctx* c, const double* src, double* dst) {
  std::vector<double> ones((size_t)c->ldk, 1.0);
  CK(cudaMemcpyAsync(dst, ones.data(), sizeof(double) * c->ldk, cudaMemcpyHostToDevice, c->s));
  CK(cudaMemcpyAsync(dst, src, sizeof(double) * c->k, cudaMemcpyDefault, c->s));
  CK(cudaStreamSynchronize(c->s));
  return PASM_OK;
}

}  // namespace

// ================================================================================================
extern "C" {

void pasm_default_opts(pasm_opts* o) {
  if (!o) return;
  o->omega = 2.0 / 3.0;
  o->nu_pre = 2;
  o->nu_post = 2;
  o->cycles_per_step = 2;
  o->max_steps = 100;
  o->precision = PASM_FP64;
  o->score_norm = PASM_SCORE_A;
  o->init = PASM_INIT_COARSE;
  o->use_graph = 1;
  o->smoother = PASM_JACOBI;
  o->projection = PASM_PROJ_TENSOR;
  o->autotune = 1;
  o->res_tol = 0.0;
}

const char* pasm_strerror(int st) {
  switch (st) {
    case PASM_OK: return "success";
    case PASM_EINVAL: return "invalid argument (malformed CSR, shape mismatch or bad option)";
    case PASM_EK_TOO_BIG: return "k exceeds the coarse space dimension";
    case PASM_ENOMEM: return "out of memory";
    case PASM_ECUDA: return "CUDA runtime error";
    case PASM_ENOTCONV: return "max_steps reached with pairs still active";
    case PASM_EDEGENERATE: return "bordered mass matrix singular for a pair";
    case PASM_ENAN: return "NaN or Inf in a pair";
    case PASM_ESTATE: return "call out of order";
    case PASM_ENOTPD: return "coarse matrix not symmetric positive definite";
    case PASM_ETIMEOUT: return "a bounded device wait gave up";
    default: return "unknown status";
  }
}

void pasm_destroy(pasm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->s);
  free_k(c);
  for (void* p : c->nn.allocs) cudaFree(p);
  for (void* p : c->allocs) cudaFree(p);
  if (c->h_nact) cudaFreeHost(c->h_nact);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->s) cudaStreamDestroy(c->s);
  delete c;
}

// Host-only validation of the hierarchy (no CUDA call): shapes, CSR structure,
// positive diagonal of every A_l (needed by the Jacobi smoother), coarse size.
static int validate_levels(int n_levels, const pasm_csr* A, const pasm_csr* M, const pasm_csr* P) {
  for (int l = 0; l < n_levels; ++l) {
    const int n = A[l].n_rows;
    if (n < 1) return PASM_EINVAL;
    int r = check_csr(A[l], n, n);
    if (!r) r = check_csr(M[l], n, n);
    if (l >= 1 && !r) r = check_csr(P[l - 1], n, A[l - 1].n_rows);
    if (r) return r;
    for (int i = 0; i < n; ++i) {
      double d = 0.0;
      for (int q = A[l].row_ptr[i]; q < A[l].row_ptr[i + 1]; ++q)
        if (A[l].col[q] == i) d += A[l].val[q];
      if (!(d > 0.0)) return PASM_EINVAL;
    }
  }
  if (A[0].n_rows > 1024) return PASM_EINVAL;
  return PASM_OK;
}

static int setup_impl(pasm_ctx* c, int n_levels, const pasm_csr* A, const pasm_csr* M, const pasm_csr* P) {
  c->nlev = n_levels;
  c->lv.resize((size_t)n_levels);
  c->geo.assign((size_t)n_levels, std::array<int, PASM_TILE_N>{});
  c->rpt.assign((size_t)n_levels, std::array<int, PASM_TILE_N>{});
  const bool mixed = c->opts.precision == PASM_MIXED;
  for (int l = 0; l < n_levels; ++l) c->lv[(size_t)l].n = A[l].n_rows;
  for (int l = 0; l < n_levels; ++l) {
    LevelDev& v = c->lv[(size_t)l];
    int r = upload_csr(c, A[l], v.A, mixed, mixed);
    if (!r) r = upload_csr(c, M[l], v.M, false, mixed);
    if (r) return r;
    if (mixed && l >= 1) {
      // A's and M's split values together on M's pattern, for the kernels that gather the same
      // vector through both (f = lam M u with r = f - A u; A u~ and M u~): one gather serves both.
      // Used when every row of A matches a subsequence of the same row of M (column order kept).
      const pasm_csr& a = A[l];
      const pasm_csr& m = M[l];
      std::vector<float4> am((size_t)m.nnz);
      bool ok = true;
      for (int i = 0; i < v.n && ok; ++i) {
        int q = a.row_ptr[i];
        const int qe = a.row_ptr[i + 1];
        for (int p2 = m.row_ptr[i]; p2 < m.row_ptr[i + 1]; ++p2) {
          const float mh = (float)m.val[p2];
          float ah = 0.f, al = 0.f;
          if (q < qe && a.col[q] == m.col[p2]) {
            ah = (float)a.val[q];
            al = v.A.exact32 ? 0.f : (float)(a.val[q] - (double)ah);   // as in A's own split values
            ++q;
          }
          am[(size_t)p2] = make_float4(ah, al, mh, (float)(m.val[p2] - (double)mh));
        }
        if (q != qe) ok = false;
      }
      if (ok && m.nnz > 0) {
        AL(c->allocs, &v.M.am, (size_t)m.nnz);
        CK(cudaMemcpy(v.M.am, am.data(), sizeof(float4) * (size_t)m.nnz, cudaMemcpyHostToDevice));
      }
    }
    std::vector<double> d((size_t)v.n, 0.0);
    for (int i = 0; i < v.n; ++i)
      for (int q = A[l].row_ptr[i]; q < A[l].row_ptr[i + 1]; ++q)
        if (A[l].col[q] == i) d[(size_t)i] = A[l].val[q];
    std::vector<double> di((size_t)v.n);
    std::vector<float> df((size_t)v.n);
    for (int i = 0; i < v.n; ++i) {
      if (!(d[(size_t)i] > 0.0)) return PASM_EINVAL;
      di[(size_t)i] = 1.0 / d[(size_t)i];
      df[(size_t)i] = (float)di[(size_t)i];
    }
    AL(c->allocs, &v.dinv64, (size_t)v.n);
    CK(cudaMemcpy(v.dinv64, di.data(), sizeof(double) * v.n, cudaMemcpyHostToDevice));
    if (mixed) {
      AL(c->allocs, &v.dinv32, (size_t)v.n);
      CK(cudaMemcpy(v.dinv32, df.data(), sizeof(float) * v.n, cudaMemcpyHostToDevice));
    }
    // omega a_ij / a_jj: the second Jacobi sweep from a zero start gathers f with these values
    // (x1 = omega D^-1 f, so A x1 = (omega A D^-1) f), with no per-entry load of a_jj (the fused
    // two-sweep kernel runs in the float32 cycles of mixed precision)
    if (mixed) {
      const int64_t nnz = A[l].row_ptr[v.n];
      std::vector<double> w((size_t)nnz);
      for (int64_t q = 0; q < nnz; ++q) w[(size_t)q] = c->opts.omega * A[l].val[q] * di[(size_t)A[l].col[q]];
      std::vector<float> wf(w.begin(), w.end());
      AL(c->allocs, &v.A.w32, (size_t)nnz);
      CK(cudaMemcpy(v.A.w32, wf.data(), sizeof(float) * (size_t)nnz, cudaMemcpyHostToDevice));
    }
    if (l >= 1) {
      const pasm_csr& p = P[l - 1];
      r = upload_csr(c, p, v.P, mixed, mixed);
      if (r) return r;
      std::vector<int32_t> rp, ci;
      std::vector<double> rv;
      transpose_csr(p, rp, ci, rv);
      pasm_csr rt{p.n_cols, p.n_rows, p.nnz, rp.data(), ci.data(), rv.data()};
      r = upload_csr(c, rt, v.R, mixed, mixed);
      if (r) return r;
      if (mixed) {
        std::vector<int32_t> qrp, qci;
        std::vector<double> qv;
        multiply_csr(rp, ci, rv, p.n_cols, A[l], qrp, qci, qv);
        pasm_csr ra{p.n_cols, A[l].n_cols, (int64_t)qci.size(), qrp.data(), qci.data(), qv.data()};
        r = upload_csr(c, ra, v.RA, true, false);
        if (r) return r;
      }
    }
  }
  // coarse pencil: dense A_H, M_H -> Lambda_H, Q (Algorithm 2 step 1 on V_H)
  const int NH = c->lv[0].n;
  c->NH = NH;
  std::vector<double> Ad((size_t)NH * NH, 0.0), Md((size_t)NH * NH, 0.0);
  for (int i = 0; i < NH; ++i) {
    for (int q = A[0].row_ptr[i]; q < A[0].row_ptr[i + 1]; ++q) Ad[(size_t)i * NH + A[0].col[q]] += A[0].val[q];
    for (int q = M[0].row_ptr[i]; q < M[0].row_ptr[i + 1]; ++q) Md[(size_t)i * NH + M[0].col[q]] += M[0].val[q];
  }
  c->h_lamH.assign((size_t)NH, 0.0);
  c->h_Q.assign((size_t)NH * NH, 0.0);
  if (coarse_generalized_eig(NH, Ad.data(), Md.data(), c->h_lamH.data(), c->h_Q.data())) return PASM_ENOTPD;
  // A_H^{-1} = Q Lambda^{-1} Q^T for the exact coarsest solve of the V-cycle
  std::vector<double> Ai((size_t)NH * NH, 0.0);
  for (int i = 0; i < NH; ++i)
    for (int j = 0; j < NH; ++j) {
      double s = 0.0;
      for (int p = 0; p < NH; ++p) s += c->h_Q[(size_t)i * NH + p] * c->h_Q[(size_t)j * NH + p] / c->h_lamH[(size_t)p];
      Ai[(size_t)i * NH + j] = s;
    }
  CK(secular_prepare(NH));
  CK(nn_tc_prepare());
  CK(nn_tc_train_prepare());
  AL(c->allocs, &c->lamH, (size_t)NH);
  AL(c->allocs, &c->Q, (size_t)NH * NH);
  AL(c->allocs, &c->AinvH64, (size_t)NH * NH);
  CK(cudaMemcpy(c->lamH, c->h_lamH.data(), sizeof(double) * NH, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->Q, c->h_Q.data(), sizeof(double) * NH * NH, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->AinvH64, Ai.data(), sizeof(double) * NH * NH, cudaMemcpyHostToDevice));
  if (mixed) {
    std::vector<float> af(Ai.begin(), Ai.end());
    AL(c->allocs, &c->AinvH32, (size_t)NH * NH);
    CK(cudaMemcpy(c->AinvH32, af.data(), sizeof(float) * NH * NH, cudaMemcpyHostToDevice));
  }
  AL(c->allocs, &c->proj_err, 1);
  CK(cudaMemset(c->proj_err, 0, sizeof(int)));
  ProjPlan plan;
  if (c->opts.projection == PASM_PROJ_TENSOR && proj_plan(NH, plan)) {
    // digit planes of Q^T (for b' = Q^T b, c' = Q^T c) and of Q (for u_H = Q g)
    std::vector<double> QT((size_t)NH * NH);
    for (int i = 0; i < NH; ++i)
      for (int j = 0; j < NH; ++j) QT[(size_t)i * NH + j] = c->h_Q[(size_t)j * NH + i];
    SplitMat* dst[2] = {&c->projQT, &c->projQ};
    const double* srcm[2] = {QT.data(), c->h_Q.data()};
    for (int q = 0; q < 2; ++q) {
      std::vector<uint16_t> planes;
      std::vector<int> rexp;
      SplitMat& sm = *dst[q];
      sm.m = NH;
      sm.K = NH;
      sm.plan = plan;
      proj_split_host(srcm[q], NH, NH, plan, sm.Kpad, sm.mtiles, planes, rexp);
      uint16_t* dp = nullptr;
      int* de = nullptr;
      AL(c->allocs, &dp, planes.size());
      AL(c->allocs, &de, rexp.size());
      CK(cudaMemcpy(dp, planes.data(), sizeof(uint16_t) * planes.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(de, rexp.data(), sizeof(int) * rexp.size(), cudaMemcpyHostToDevice));
      sm.planes = dp;
      sm.rexp = de;
    }
    CK(proj_tc_prepare());
    c->proj_tc = true;
  }
  return PASM_OK;
}

int pasm_setup(pasm_ctx** out, int n_levels, const pasm_csr* A, const pasm_csr* M, const pasm_csr* P,
               const pasm_opts* opts, void* stream) {
  if (!out) return PASM_EINVAL;
  *out = nullptr;
  if (n_levels < 1 || !A || !M || (n_levels > 1 && !P)) return PASM_EINVAL;
  pasm_opts o;
  pasm_default_opts(&o);
  if (opts) o = *opts;
  if (o.nu_pre < 0 || o.nu_post < 0 || o.cycles_per_step < 1 || o.max_steps < 0 || !(o.omega > 0.0) ||
      (o.precision != PASM_FP64 && o.precision != PASM_MIXED) ||
      (o.score_norm != PASM_SCORE_A && o.score_norm != PASM_SCORE_B) ||
      (o.init != PASM_INIT_COARSE && o.init != PASM_INIT_NESTED) ||
      (o.smoother != PASM_JACOBI && o.smoother != PASM_LEARNED && o.smoother != PASM_CG) ||
      (o.smoother == PASM_LEARNED && o.precision != PASM_MIXED) ||
      (o.projection != PASM_PROJ_TENSOR && o.projection != PASM_PROJ_FP64) || !(o.res_tol >= 0.0))
    return PASM_EINVAL;
  int v = validate_levels(n_levels, A, M, P);
  if (v) return v;
  pasm_ctx* c = new (std::nothrow) pasm_ctx();
  if (!c) return PASM_ENOMEM;
  c->opts = o;
  c->user = (cudaStream_t)stream;
  if (cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost((void**)&c->h_nact, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    pasm_destroy(c);
    return PASM_ECUDA;
  }
  int r = setup_impl(c, n_levels, A, M, P);
  if (r) { pasm_destroy(c); return r; }
  *out = c;
  return PASM_OK;
}

extern "C++" {
// Autotuner of the row-group kernels: for every level with at least
// kTuneRows rows and every kernel kind of the context's precision, time each
// valid number of 16-byte chunks per thread (1, 2, 4, 8) on the level's own
// matrices (one warm-up, then the mean of three launches, CUDA events on the
// context's stream) and keep the fastest.  Runs once per block width ldk; the
// buffers it uses are scratch of the step (the mixed-precision update writes
// into scratch; the float64 update runs with no pair selected, so U is read
// and rewritten unchanged).
static constexpr int kTuneRows = 16384;

template <typename Fn>
static float time_launch(pasm_ctx* c, cudaEvent_t e0, cudaEvent_t e1, int geo, Fn&& fn, int rpt = 0) {
  Launch L;
  L.s = c->s;
  L.geo = geo;
  L.rpt = rpt;
  fn(L);
  cudaEventRecord(e0, c->s);
  for (int q = 0; q < 3; ++q) fn(L);
  cudaEventRecord(e1, c->s);
  if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

static int autotune(pasm_ctx* c) {
  if (!c->opts.autotune || c->tuned_ldk == c->ldk) return PASM_OK;
  for (auto& g : c->geo) g.fill(0);
  for (auto& g : c->rpt) g.fill(0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return PASM_ECUDA;
  }
  const bool mixed = c->opts.precision == PASM_MIXED;
  const int ldk = c->ldk;
  CK(cudaMemsetAsync(c->upd, 0, sizeof(int) * (size_t)ldk, c->s));
  // rows: the kernel kind also takes a number of row blocks per block (1 or 4)
  auto pick = [&](int l, int kind, int chunks, auto&& fn, bool rows = false) -> float {
    int best = 0, best_rpt = 0;
    float best_ms = 1e30f;
    for (int ch : {1, 2, 4, 8}) {
      if (chunks % ch != 0 || chunks / ch > 32) continue;
      // the bordering kernel keeps its per-block reduction within 48 KB of shared memory
      if (kind == PASM_TILE_BORDER && (size_t)(256 / (chunks / ch)) * 2 * ldk * sizeof(double) > 48 * 1024) continue;
      for (int r : {1, 4}) {
        if (r > 1 && !rows) break;
        const float ms = time_launch(c, e0, e1, ch, fn, rows ? r : 0);
        if (ms < best_ms) { best_ms = ms; best = ch; best_rpt = rows ? r : 0; }
      }
    }
    c->geo[(size_t)l][(size_t)kind] = best;
    c->rpt[(size_t)l][(size_t)kind] = best_rpt;
    return best_ms;
  };
  const int c32 = ldk / 4, c64 = ldk / 2;  // 16-byte chunks per row: float32, float64 / pairs
  for (int l = 1; l < c->nlev; ++l) {
    LevelDev& v = c->lv[(size_t)l];
    LevelDev& w = c->lv[(size_t)l - 1];
    if (v.n < kTuneRows) continue;
    if (mixed) {
      float *F = (float*)v.vF, *E = (float*)v.vE, *Tm = (float*)v.vT;
      const float om = (float)c->opts.omega;
      const float t_j2 = pick(l, PASM_TILE_JACOBI2_ZERO, c32,
                              [&](const Launch& L) { jacobi2_zero<float>(L, v.A, v.dinv32, om, F, E, ldk); }, true);
      const float t_j = pick(l, PASM_TILE_JACOBI, c32,
                             [&](const Launch& L) { rowop<float>(L, OP_JACOBI, v.A, E, F, E, v.dinv32, om, Tm, ldk); },
                             true);
      const float t_j0 = time_launch(c, e0, e1, 0, [&](const Launch& L) { jacobi_zero<float>(L, v.n, v.dinv32, om, F, E, ldk); });
      if (t_j0 + t_j < t_j2) c->geo[(size_t)l][PASM_TILE_JACOBI2_ZERO] = -1;   // split: one sweep from zero + one sweep
      const float t_rr = pick(l, PASM_TILE_RESID_RESTRICT, c32,
                              [&](const Launch& L) { resid_restrict<float>(L, v.R, v.A, E, F, (float*)w.vF, ldk); },
                              true);
      const float t_r = pick(l, PASM_TILE_RESID, c32, [&](const Launch& L) {
        rowop<float>(L, OP_RESID, v.A, E, F, nullptr, nullptr, om, Tm, ldk);
      }, true);
      const float t_s = pick(l, PASM_TILE_RESTRICT, c32, [&](const Launch& L) {
        rowop<float>(L, OP_SPMM, v.R, Tm, nullptr, nullptr, nullptr, om, (float*)w.vF, ldk);
      }, true);
      if (t_r + t_s < t_rr) c->geo[(size_t)l][PASM_TILE_RESID_RESTRICT] = -1;    // split: residual, then restriction
      // restriction first (R f - (R A) e) against the faster of the two forms above
      const float t_rf = pick(l, PASM_TILE_RESTRICT_FIRST, c32, [&](const Launch& L) {
        restrict_first(L, v.R, v.RA, E, F, (float*)w.vF, ldk);
      }, true);
      if (!(t_rf < std::min(t_rr, t_r + t_s))) {
        c->geo[(size_t)l][PASM_TILE_RESTRICT_FIRST] = 0;
        c->rpt[(size_t)l][PASM_TILE_RESTRICT_FIRST] = 0;
      }
      const float t_p = pick(l, PASM_TILE_PROLONG, c32, [&](const Launch& L) {
        rowop<float>(L, OP_SPMM_ADD, v.P, (float*)w.vE, E, nullptr, nullptr, om, E, ldk);
      }, true);
      const float t_ps = pick(l, PASM_TILE_PROLONG_SWEEP, c32, [&](const Launch& L) {
        prolong_jacobi(L, v.A, v.P, E, (float*)w.vE, F, v.dinv32, om, Tm, ldk);
      });
      if (t_p + t_j < t_ps) c->geo[(size_t)l][PASM_TILE_PROLONG_SWEEP] = -1;   // split: prolongation, then sweep
      pick(l, PASM_TILE_OUTER_RHS, c64, [&](const Launch& L) {
        outer_rhs_residual_ff(L, v.A, v.M, c->lam, c->Uff, c->Fd, F, ldk);
      }, true);
      pick(l, PASM_TILE_OUTER_RES, c64, [&](const Launch& L) { outer_residual_ff(L, v.A, c->Fd, c->X, F, ldk); },
           true);
      pick(l, PASM_TILE_BORDER, c64, [&](const Launch& L) {
        border_products_ff(L, v.A, v.M, c->X, c->YA, c->YM, c->partials, ldk, c->max_border_blocks);
      });
      pick(l, PASM_TILE_CHAIN_R, c64, [&](const Launch& L) {
        spmm2_ff(L, v.R, c->YA, c->YM, true, w.BA, w.BM, l - 1 >= 1, ldk);
      }, true);
      if (l < c->nlev - 1)
        pick(l, PASM_TILE_CHAIN_P, c64, [&](const Launch& L) { spmm_ff(L, v.P, w.BA, l - 1 >= 1, v.BA, true, ldk); },
             true);
      const double* wsrc = (l - 1 >= 1) ? w.BA : c->uH;
      // the update skips frozen pairs, so it is timed with every pair selected, writing
      // into scratch (YM) instead of U
      CK(cudaMemsetAsync(c->upd, 1, sizeof(int) * (size_t)ldk, c->s));
      pick(l, PASM_TILE_UPDATE, c64, [&](const Launch& L) {
        update_pairs_ff(L, &v.P, v.n, wsrc, l - 1 >= 1, c->X, c->alpha, c->upd, c->YM, nullptr, ldk);
      }, true);
      CK(cudaMemsetAsync(c->upd, 0, sizeof(int) * (size_t)ldk, c->s));
    } else {
      double *F = (double*)v.vF, *E = (double*)v.vE, *Tm = (double*)v.vT;
      const double om = c->opts.omega;
      pick(l, PASM_TILE_JACOBI, c64, [&](const Launch& L) { rowop<double>(L, OP_JACOBI, v.A, E, F, E, v.dinv64, om, Tm, ldk); });
      pick(l, PASM_TILE_RESID, c64,
           [&](const Launch& L) { rowop<double>(L, OP_RESID, v.A, E, F, nullptr, nullptr, om, Tm, ldk); });
      pick(l, PASM_TILE_RESTRICT, c64, [&](const Launch& L) {
        rowop<double>(L, OP_SPMM, v.R, Tm, nullptr, nullptr, nullptr, om, (double*)w.vF, ldk);
      });
      pick(l, PASM_TILE_PROLONG, c64, [&](const Launch& L) {
        rowop<double>(L, OP_SPMM_ADD, v.P, (double*)w.vE, E, nullptr, nullptr, om, E, ldk);
      });
      pick(l, PASM_TILE_OUTER_RHS, c64, [&](const Launch& L) {
        outer_rhs_residual<double>(L, v.A, v.M, c->lam, c->U, c->Fd, F, ldk);
      });
      pick(l, PASM_TILE_OUTER_RES, c64, [&](const Launch& L) { outer_residual<double>(L, v.A, c->Fd, c->X, F, ldk); });
      pick(l, PASM_TILE_BORDER, c64, [&](const Launch& L) {
        border_products(L, v.A, v.M, c->X, c->YA, c->YM, c->partials, ldk, c->max_border_blocks);
      });
      pick(l, PASM_TILE_CHAIN_R, c64, [&](const Launch& L) {
        rowop<double>(L, OP_SPMM, v.R, c->YA, nullptr, nullptr, nullptr, 0.0, w.BA, ldk);
      });
      if (l < c->nlev - 1)
        pick(l, PASM_TILE_CHAIN_P, c64, [&](const Launch& L) {
          rowop<double>(L, OP_SPMM, v.P, w.BA, nullptr, nullptr, nullptr, 0.0, v.BA, ldk);
        });
      const double* wsrc = (l - 1 >= 1) ? w.BA : c->uH;
      pick(l, PASM_TILE_UPDATE, c64,
           [&](const Launch& L) { update_pairs(L, v.P, wsrc, c->X, c->alpha, c->upd, c->U, ldk); });
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  c->tuned_ldk = ldk;
  return PASM_OK;
}
}  // extern "C++"

// Rebuild the float64 state U from its pair copy after mixed-precision steps
// (one elementwise pass, on the context's stream).
static void sync_state(pasm_ctx* c) {
  if (!c->u_stale) return;
  from_ff(launcher(c), (int64_t)c->lv.back().n * c->ldk, c->Uff, c->U);
  c->u_stale = false;
}

int pasm_init(pasm_ctx* c, int k, double tol, const double* lambda0, const double* U0) {
  if (!c || k < 1 || k > 256 || !(tol >= 0.0)) return PASM_EINVAL;
  if ((lambda0 == nullptr) != (U0 == nullptr)) return PASM_EINVAL;
  if (!lambda0 && k > c->NH) return PASM_EK_TOO_BIG;
  Scope sc(c);
  int r = alloc_k(c, k);
  if (!r) r = autotune(c);
  if (r) return r;
  c->tol = tol;
  const int nf = c->lv.back().n;
  const Launch L = launcher(c);
  if (lambda0) {
    r = put_lambda(c, lambda0, c->lam);
    if (!r) r = put_block(c, U0, c->U, nf);
    if (r) return r;
  } else if (c->opts.init == PASM_INIT_NESTED && c->nlev >= 3) {
    // Algorithm 2 with h_1 = H: pairs on V_H, then one correction step on every
    // intermediate level l (step 2(A), varpi = 1), each started from the
    // prolongated pairs of level l - 1; finally prolongation to the finest level.
    const size_t ldk = (size_t)c->ldk;
    coarse_init(L, c->NH, k, c->Q, c->lamH, c->uH, c->lam, c->ldk);
    r = set_active(c, c->active, c->steps, c->status);
    if (r) return r;
    const double* src = c->uH;
    for (int l = 1; l < c->nlev; ++l) {
      rowop<double>(L, OP_SPMM, c->lv[l].P, src, nullptr, nullptr, nullptr, 0.0, c->YM, c->ldk);
      CK(cudaMemcpyAsync(c->U, c->YM, sizeof(double) * (size_t)c->lv[l].n * ldk, cudaMemcpyDeviceToDevice, c->s));
      if (l == c->nlev - 1) break;
      bvp(c, l, c->lam, c->U, c->X);
      PairState ps{c->lam, c->active, c->steps, c->status, c->U, 0.0};
      augmented(c, l, c->X, ps);
      src = c->U;
    }
  } else {
    // u_i = P_c q_i / sqrt(Lambda_i), lambda_i = Lambda_i
    double* w = (c->nlev == 1) ? c->U : c->uH;
    coarse_init(L, c->NH, k, c->Q, c->lamH, w, c->lam, c->ldk);
    for (int l = 1; l < c->nlev; ++l) {
      double* dst = (l == c->nlev - 1) ? c->U : c->lv[l].BA;
      rowop<double>(L, OP_SPMM, c->lv[l].P, w, nullptr, nullptr, nullptr, 0.0, dst, c->ldk);
      w = dst;
    }
  }
  r = set_active(c, c->active, c->steps, c->status);
  if (r) return r;
  if (c->nn.ready) {
    int64_t maxn = 0;
    for (int l = 0; l < c->nlev; ++l)
      if (c->nn.nx[(size_t)l]) maxn = std::max<int64_t>(maxn, c->lv[(size_t)l].n);
    r = nn_ensure(c, maxn * c->ldk, maxn * c->ldk, false);
    if (r) return r;
    CK(cudaMemsetAsync(c->nn.accepted, 0, sizeof(int) * 256, c->s));
  }
  // the pair copy of the state U that the first step's gathers read (later steps: the update)
  if (c->opts.precision == PASM_MIXED) to_ff(L, (int64_t)nf * c->ldk, c->U, c->Uff);
  c->u_stale = false;
  CK(cudaMemsetAsync(c->diag, 0, sizeof(int) * 8, c->s));  // secular counters count the steps only
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->s));
  c->initialized = true;
  return PASM_OK;
}

int pasm_step(pasm_ctx* c, int* n_active) {
  if (!c || !c->initialized) return PASM_ESTATE;
  Scope sc(c);
  if (c->opts.use_graph) {
    if (!c->graph) {
      cudaGraph_t g;
      c->launches = 0;
      CK(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
      step_body(c);
      CK(cudaStreamEndCapture(c->s, &g));
      cudaError_t e = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      CK(e);
      c->last_launches = c->launches;
    }
    CK(cudaGraphLaunch(c->graph, c->s));
  } else {
    c->launches = 0;
    step_body(c);
    c->last_launches = c->launches;
    CK(cudaGetLastError());
  }
  if (c->opts.precision == PASM_MIXED) c->u_stale = true;
  if (n_active) {
    CK(cudaStreamSynchronize(c->s));
    *n_active = *c->h_nact;
  }
  return PASM_OK;
}

// Enqueue one correction step on the context's own stream, with no ordering
// against the caller's stream, no graph of its own and no synchronisation, so
// that the batch driver can capture the steps of many contexts into one graph
// (the step's active count lands in the context's pinned word, read by
// pasm_ctx_active_host once the work is done).
int pasm_ctx_enqueue_step(pasm_ctx* c) {
  if (!c || !c->initialized) return PASM_ESTATE;
  step_body(c);
  if (c->opts.precision == PASM_MIXED) c->u_stale = true;
  return PASM_OK;
}

void* pasm_ctx_stream(pasm_ctx* c) { return c ? (void*)c->s : nullptr; }

int pasm_ctx_active_host(pasm_ctx* c) { return c && c->h_nact ? *c->h_nact : 0; }

// Wait for the context's queued work and return the active-pair count the
// last step left in pinned memory (used by the batch driver).
int pasm_ctx_wait_active(pasm_ctx* c, int* n_active) {
  if (!c || !c->initialized) return PASM_ESTATE;
  CK(cudaStreamSynchronize(c->s));
  *n_active = *c->h_nact;
  return PASM_OK;
}

int pasm_get(pasm_ctx* c, double* lambda, double* U, int* steps, int* status) {
  if (!c || !c->initialized) return PASM_ESTATE;
  Scope sc(c);
  if (lambda) CK(cudaMemcpyAsync(lambda, c->lam, sizeof(double) * c->k, cudaMemcpyDefault, c->s));
  if (U) {
    sync_state(c);
    int r = get_block(c, c->U, U, c->lv.back().n);
    if (r) return r;
  }
  if (steps) CK(cudaMemcpyAsync(steps, c->steps, sizeof(int) * c->k, cudaMemcpyDefault, c->s));
  if (status) CK(cudaMemcpyAsync(status, c->status, sizeof(int) * c->k, cudaMemcpyDefault, c->s));
  int perr = 0;
  CK(cudaMemcpyAsync(&perr, c->proj_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  return perr ? PASM_ETIMEOUT : PASM_OK;
}

// The residual guard of opts.res_tol, after a step in which pairs froze: a pair
// the |dlambda| test froze is made active again while its relative residual
// exceeds the bound; *n_active counts it again.  No-op when res_tol <= 0.
int pasm_ctx_guard_freezes(pasm_ctx* c, int* n_active) {
  if (!c || !c->initialized) return PASM_ESTATE;
  if (!(c->opts.res_tol > 0.0)) return PASM_OK;
  const int k = c->k;
  std::vector<double> res((size_t)k, 0.0);
  std::vector<int> status((size_t)k, 0), active((size_t)k, 0);
  int r = pasm_residuals(c, res.data());
  if (r) return r;
  // copies on the context's stream (non-blocking: the legacy-stream cudaMemcpy would not be
  // ordered with it), completed before the host reads or the next step runs
  CK(cudaMemcpyAsync(status.data(), c->status, sizeof(int) * k, cudaMemcpyDeviceToHost, c->s));
  CK(cudaMemcpyAsync(active.data(), c->active, sizeof(int) * k, cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  int back = 0;
  for (int i = 0; i < k; ++i)
    if (status[(size_t)i] == PASM_PAIR_CONVERGED && !(res[(size_t)i] <= c->opts.res_tol)) {
      status[(size_t)i] = PASM_PAIR_ACTIVE;
      active[(size_t)i] = 1;
      ++back;
    }
  if (back) {
    CK(cudaMemcpyAsync(c->status, status.data(), sizeof(int) * k, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->active, active.data(), sizeof(int) * k, cudaMemcpyHostToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (n_active) *n_active += back;
  }
  return PASM_OK;
}

int pasm_solve(pasm_ctx* c, int k, double tol, const double* lambda0, const double* U0, double* lambda_out,
               double* U_out, int* steps_out, int* status_out) {
  if (!c) return PASM_EINVAL;
  int r = pasm_init(c, k, tol, lambda0, U0);
  if (r) return r;
  int act = k;
  for (int s = 0; s < c->opts.max_steps && act > 0; ++s) {
    const int before = act;
    r = pasm_step(c, &act);
    if (!r && act < before) r = pasm_ctx_guard_freezes(c, &act);
    if (r) return r;
  }
  r = pasm_get(c, lambda_out, U_out, steps_out, status_out);
  if (r) return r;
  return act > 0 ? PASM_ENOTCONV : PASM_OK;
}

int pasm_bvp(pasm_ctx* c, const double* lambda, const double* U, double* Uhat) {
  if (!c || !c->initialized || !lambda || !U || !Uhat) return PASM_ESTATE;
  Scope sc(c);
  sync_state(c);  // the pair copy is rebuilt from U below
  const int nf = c->lv.back().n;
  int r = put_lambda(c, lambda, c->lam2);
  if (!r) r = put_block(c, U, c->YM, nf);
  if (r) return r;
  bvp(c, c->nlev - 1, c->lam2, c->YM, c->X);
  CK(cudaGetLastError());
  const double* xout = c->X;
  if (c->opts.precision == PASM_MIXED) {  // u~ comes back in (hi, lo) pairs
    from_ff(launcher(c), (int64_t)nf * c->ldk, c->X, c->YA);
    xout = c->YA;
    to_ff(launcher(c), (int64_t)nf * c->ldk, c->U, c->Uff);  // the step's pair copy of the state U again
  }
  r = get_block(c, xout, Uhat, nf);
  if (r) return r;
  CK(cudaStreamSynchronize(c->s));
  return PASM_OK;
}

int pasm_augmented(pasm_ctx* c, const double* lambda_prev, const double* Uhat, double* lambda_out, double* U_out,
                   double* beta, double* zeta) {
  if (!c || !c->initialized || !lambda_prev || !Uhat) return PASM_ESTATE;
  Scope sc(c);
  sync_state(c);
  const int nf = c->lv.back().n;
  int r = put_lambda(c, lambda_prev, c->lam2);
  if (!r) r = put_block(c, Uhat, c->X, nf);
  if (!r) r = set_active(c, c->active2, c->steps2, c->status2);
  if (r) return r;
  CK(cudaMemcpyAsync(c->Fd, c->X, sizeof(double) * (size_t)nf * c->ldk, cudaMemcpyDeviceToDevice, c->s));
  if (c->opts.precision == PASM_MIXED) to_ff(launcher(c), (int64_t)nf * c->ldk, c->X, c->X);
  PairState ps{c->lam2, c->active2, c->steps2, c->status2, c->Fd, 0.0};
  augmented(c, c->nlev - 1, c->X, ps);
  CK(cudaGetLastError());
  if (lambda_out) CK(cudaMemcpyAsync(lambda_out, c->lam2, sizeof(double) * c->k, cudaMemcpyDefault, c->s));
  if (U_out) { r = get_block(c, c->Fd, U_out, nf); if (r) return r; }
  if (beta) CK(cudaMemcpyAsync(beta, c->bz, sizeof(double) * c->k, cudaMemcpyDefault, c->s));
  if (zeta) CK(cudaMemcpyAsync(zeta, c->bz + c->ldk, sizeof(double) * c->k, cudaMemcpyDefault, c->s));
  CK(cudaStreamSynchronize(c->s));
  return PASM_OK;
}

int pasm_project(pasm_ctx* c, const double* b, const double* cc, double* bq, double* cq) {
  if (!c || !c->initialized) return PASM_ESTATE;
  if (!b || !cc || !bq || !cq) return PASM_EINVAL;
  Scope sc(c);
  const int NH = c->NH;
  int before = 0, after = 0;
  CK(cudaMemcpyAsync(&before, c->proj_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
  int r = put_block(c, b, c->g, NH);
  if (!r) r = put_block(c, cc, c->uH, NH);
  if (r) return r;
  project_bc(c, launcher(c), c->g, c->uH, c->bq, c->cq);
  CK(cudaGetLastError());
  r = get_block(c, c->bq, bq, NH);
  if (!r) r = get_block(c, c->cq, cq, NH);
  if (r) return r;
  CK(cudaMemcpyAsync(&after, c->proj_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  return after != before ? PASM_ETIMEOUT : PASM_OK;
}

int pasm_debug_waits(pasm_ctx* c, int skip_mma, int wait_limit) {
  if (!c || wait_limit < 0) return PASM_EINVAL;
  c->dbg_skip_mma = skip_mma ? 1 : 0;
  c->dbg_wait_limit = wait_limit;
  // a captured step graph holds the old launch arguments
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return PASM_OK;
}

int pasm_tiles(pasm_ctx* c, int level, int* chunks_per_thread) {
  if (!c || !chunks_per_thread || level < 0 || level >= c->nlev) return PASM_EINVAL;
  for (int q = 0; q < PASM_TILE_N; ++q) chunks_per_thread[q] = c->geo[(size_t)level][(size_t)q];
  return PASM_OK;
}

int pasm_tile_rows(pasm_ctx* c, int level, int* rows_per_block) {
  if (!c || !rows_per_block || level < 0 || level >= c->nlev) return PASM_EINVAL;
  for (int q = 0; q < PASM_TILE_N; ++q) rows_per_block[q] = c->rpt[(size_t)level][(size_t)q];
  return PASM_OK;
}

int pasm_set_tiles(pasm_ctx* c, int level, const int* chunks_per_thread, const int* rows_per_block) {
  if (!c || !chunks_per_thread || level < 0 || level >= c->nlev) return PASM_EINVAL;
  for (int q = 0; q < PASM_TILE_N; ++q) {
    const int ch = chunks_per_thread[q], r = rows_per_block ? rows_per_block[q] : 0;
    const bool fusable = q == PASM_TILE_JACOBI2_ZERO || q == PASM_TILE_RESID_RESTRICT || q == PASM_TILE_PROLONG_SWEEP;
    if (q == PASM_TILE_RESTRICT_FIRST && ch > 0 && !c->lv[(size_t)level].RA.rp) return PASM_EINVAL;
    if (!(ch == 0 || ch == 1 || ch == 2 || ch == 4 || ch == 8 || (ch == -1 && fusable))) return PASM_EINVAL;
    if (!(r == 0 || r == 1 || r == 4)) return PASM_EINVAL;
  }
  for (int q = 0; q < PASM_TILE_N; ++q) {
    c->geo[(size_t)level][(size_t)q] = chunks_per_thread[q];
    c->rpt[(size_t)level][(size_t)q] = rows_per_block ? rows_per_block[q] : 0;
  }
  // a captured step graph holds the old launch shapes
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return PASM_OK;
}

int pasm_projection_kind(pasm_ctx* c, int* kind) {
  if (!c || !kind) return PASM_EINVAL;
  *kind = c->proj_tc ? PASM_PROJ_TENSOR : PASM_PROJ_FP64;
  return PASM_OK;
}

int pasm_residuals(pasm_ctx* c, double* res) {
  if (!c || !res) return PASM_EINVAL;
  if (!c->initialized) return PASM_ESTATE;
  Scope sc(c);
  const int lt = c->nlev - 1, ldk = c->ldk;
  LevelDev& v = c->lv[(size_t)lt];
  const Launch L = launcher(c);
  int nb;
  if (c->opts.precision == PASM_MIXED) {
    outer_rhs_residual_ff(launcher(c, lt, PASM_TILE_OUTER_RHS), v.A, v.M, c->lam, c->Uff, c->Fd, (float*)v.vF, ldk);
    nb = residual_partials<float>(L, v.n, ldk, (const float*)v.vF, true, c->Fd, c->Uff, c->partials,
                                  c->max_border_blocks);
  } else {
    outer_rhs_residual<double>(launcher(c, lt, PASM_TILE_OUTER_RHS), v.A, v.M, c->lam, c->U, c->Fd, (double*)v.vF,
                               ldk);
    nb = residual_partials<double>(L, v.n, ldk, (const double*)v.vF, false, c->Fd, c->U, c->partials,
                                   c->max_border_blocks);
  }
  column_sums(L, c->partials, nb, 2, ldk, c->bz);
  std::vector<double> sums((size_t)2 * ldk), lam((size_t)c->k);
  CK(cudaMemcpyAsync(sums.data(), c->bz, sizeof(double) * 2 * ldk, cudaMemcpyDeviceToHost, c->s));
  CK(cudaMemcpyAsync(lam.data(), c->lam, sizeof(double) * c->k, cudaMemcpyDeviceToHost, c->s));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->s));
  // |A u - lam M u|_2 / (|lam| |u|_M), with sum u (lam M u) = lam u^T M u
  for (int i = 0; i < c->k; ++i) {
    const double rr = sums[(size_t)i], um = sums[(size_t)ldk + i];
    res[i] = std::sqrt(rr) / std::sqrt(std::fabs(lam[(size_t)i] * um));
  }
  return PASM_OK;
}

int pasm_secular_stats(pasm_ctx* c, int* out) {
  if (!c || !out) return PASM_EINVAL;
  if (!c->initialized) return PASM_ESTATE;
  Scope sc(c);
  CK(cudaMemcpyAsync(out, c->diag, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  return PASM_OK;
}

static std::vector<Tracer::Rec> g_last_trace;  // launch list of the last traced step
static std::vector<float> g_last_trace_ms;

int pasm_trace_step(pasm_ctx* c, double* ms, double* bytes, double* flops, int* launches) {
  if (!c || !c->initialized) return PASM_ESTATE;
  Scope sc(c);
  Tracer tr;
  c->tracer = &tr;
  c->launches = 0;
  step_body(c);
  c->tracer = nullptr;
  if (c->opts.precision == PASM_MIXED) c->u_stale = true;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->s));
  for (int q = 0; q < KC_N; ++q) {
    if (ms) ms[q] = 0.0;
    if (bytes) bytes[q] = 0.0;
    if (flops) flops[q] = 0.0;
    if (launches) launches[q] = 0;
  }
  g_last_trace.clear();
  g_last_trace_ms.clear();
  for (const auto& r : tr.recs) {
    if (r.e1 < 0 || r.cls < 0 || r.cls >= KC_N) continue;
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, tr.ev[(size_t)r.e0], tr.ev[(size_t)r.e1]));
    g_last_trace.push_back(r);
    g_last_trace_ms.push_back(t);
    if (ms) ms[r.cls] += t;
    if (bytes) bytes[r.cls] += r.bytes;
    if (flops) flops[r.cls] += r.flops;
    if (launches) launches[r.cls] += 1;
  }
  return PASM_OK;
}

// ------------------------------------------------------------------------------------------------
// Learned post-smoother

// Grow the learned smoother's buffers: forward activations for `pixpairs`
// pixel-pairs, backward ones too when `backward` (training), and the n x ldk
// temporaries for `vecs` entries.  (Inference needs only the forward ones.)
static int nn_ensure(pasm_ctx* c, int64_t pixpairs, int64_t vecs, bool backward) {
  auto& nn = c->nn;
  if (pixpairs > nn.buf.cap) {
    const size_t m = (size_t)pixpairs * 16;
    float** bufs[] = {&nn.buf.z1, &nn.buf.z2p, &nn.buf.z2m, &nn.buf.h};
    for (float** b : bufs) AL(nn.allocs, b, m);
    nn.buf.cap = pixpairs;
  }
  if (backward && pixpairs > nn.bcap) {
    const size_t m = (size_t)pixpairs * 16;
    float** bufs[] = {&nn.buf.gh, &nn.buf.gzp, &nn.buf.gzm, &nn.buf.gap, &nn.buf.gam, &nn.buf.gz1};
    for (float** b : bufs) AL(nn.allocs, b, m);
    nn.bcap = pixpairs;
  }
  if (vecs > nn.vcap) {
    AL(nn.allocs, &nn.R, (size_t)vecs); AL(nn.allocs, &nn.D, (size_t)vecs); AL(nn.allocs, &nn.X, (size_t)vecs);
    AL(nn.allocs, &nn.Rt, (size_t)vecs); AL(nn.allocs, &nn.Es, (size_t)vecs); AL(nn.allocs, &nn.gD, (size_t)vecs);
    AL(nn.allocs, &nn.partial, (size_t)((vecs / 4 + 64) / 64 + 1) * 2 * 256);
    nn.vcap = vecs;
  }
  return PASM_OK;
}

// Copy layers 1 and 3 of the device weights into the host copy the
// tensor-core forward passes as kernel parameters.
static int nn_refresh_host_weights(pasm_ctx* c) {
  std::vector<float> h((size_t)kNNWeights);
  CK(cudaMemcpy(h.data(), c->nn.W, sizeof(float) * kNNWeights, cudaMemcpyDeviceToHost));
  std::memcpy(c->nn.w13.w1, h.data(), sizeof(float) * 144);
  std::memcpy(c->nn.w13.w3, h.data() + 144 + 2304, sizeof(float) * 144);
  if (c->nn.w2) {
    std::vector<uint16_t> w2((size_t)2304);
    nn_tc_layer2_layout(h.data() + 144, w2.data());
    CK(cudaMemcpy(c->nn.w2, w2.data(), sizeof(uint16_t) * 2304, cudaMemcpyHostToDevice));
  }
  return PASM_OK;
}

int pasm_nn_setup(pasm_ctx* c, const int32_t* nx, const float* weights) {
  if (!c || !nx || !weights) return PASM_EINVAL;
  if (c->opts.precision != PASM_MIXED) return PASM_EINVAL;
  auto& nn = c->nn;
  nn.nx.assign((size_t)c->nlev, 0);
  nn.ny.assign((size_t)c->nlev, 0);
  int64_t maxn = 0;
  for (int l = 0; l < c->nlev; ++l) {
    if (nx[l] <= 0) continue;
    const int n = c->lv[(size_t)l].n;
    if (n % nx[l]) return PASM_EINVAL;
    nn.nx[(size_t)l] = nx[l];
    nn.ny[(size_t)l] = n / nx[l];
    maxn = std::max<int64_t>(maxn, n);
  }
  if (!nn.W) {
    AL(nn.allocs, &nn.W, kNNWeights); AL(nn.allocs, &nn.m, kNNWeights); AL(nn.allocs, &nn.v, kNNWeights);
    AL(nn.allocs, &nn.grad, kNNWeights);
    AL(nn.allocs, &nn.buf.wpart, (size_t)NNBuf::kWgradBlocks * 2304);
    AL(nn.allocs, &nn.buf.wflip2, 2304); AL(nn.allocs, &nn.buf.wflip3, 144);
    AL(nn.allocs, &nn.norms, 2 * 256); AL(nn.allocs, &nn.loss, 1); AL(nn.allocs, &nn.accepted, 256);
    AL(nn.allocs, &nn.err, 4);
    AL(nn.allocs, &nn.w2, 2304);
    AL(nn.allocs, &nn.w2f, 2304);
    AL(nn.allocs, &nn.w2t, 2304);
    CK(cudaMemset(nn.err, 0, sizeof(int) * 4));
  }
  CK(cudaMemcpy(nn.W, weights, sizeof(float) * kNNWeights, cudaMemcpyDefault));
  if (int rw = nn_refresh_host_weights(c)) return rw;
  CK(cudaMemset(nn.m, 0, sizeof(float) * kNNWeights));
  CK(cudaMemset(nn.v, 0, sizeof(float) * kNNWeights));
  CK(cudaMemset(nn.accepted, 0, sizeof(int) * 256));
  nn.t = 0;
  // V-cycle use needs the n x ldk temporaries and activations of the largest grid level
  if (c->k > 0 && maxn > 0) {
    int r = nn_ensure(c, maxn * c->ldk, maxn * c->ldk, false);
    if (r) return r;
  }
  nn.ready = true;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return PASM_OK;
}

int pasm_nn_get_weights(pasm_ctx* c, float* weights) {
  if (!c || !weights || !c->nn.W) return PASM_ESTATE;
  CK(cudaMemcpy(weights, c->nn.W, sizeof(float) * kNNWeights, cudaMemcpyDefault));
  return PASM_OK;
}

// copy a user n x k float block into an n x ldk2 device block (zero padding)
static int put_block_f(pasm_ctx* c, const float* src, float* dst, int n, int k, int ldk2) {
  CK(cudaMemsetAsync(dst, 0, sizeof(float) * (size_t)n * ldk2, c->s));
  CK(cudaMemcpy2DAsync(dst, sizeof(float) * ldk2, src, sizeof(float) * k, sizeof(float) * k, n, cudaMemcpyDefault,
                       c->s));
  return PASM_OK;
}

static int nn_level_check(pasm_ctx* c, int level, int k) {
  if (!c || !c->nn.ready || level < 0 || level >= c->nlev || c->nn.nx[(size_t)level] == 0 || k < 1 || k > 256)
    return PASM_EINVAL;
  return PASM_OK;
}

int pasm_nn_apply(pasm_ctx* c, int level, int k, const float* R, float* D) {
  int r = nn_level_check(c, level, k);
  if (r) return r;
  if (!R || !D) return PASM_EINVAL;
  Scope sc(c);
  const int n = c->lv[(size_t)level].n, ldk2 = ldk_for(k);
  r = nn_ensure(c, (int64_t)n * ldk2, (int64_t)n * ldk2, false);
  if (r) return r;
  auto& nn = c->nn;
  r = put_block_f(c, R, nn.R, n, k, ldk2);
  if (r) return r;
  NNGrid g{nn.nx[(size_t)level], nn.ny[(size_t)level], ldk2, k};
  if (c->opts.smoother == PASM_LEARNED && nn_tc_supported(ldk2))
    nn_forward_tc(launcher(c), g, nn.w13, nn.w2, nn.R, nn.D, nn.err);
  else
    nn_forward(launcher(c), g, nn.buf, nn.W, nn.R, nn.D);
  CK(cudaMemcpy2DAsync(D, sizeof(float) * k, nn.D, sizeof(float) * ldk2, sizeof(float) * k, n, cudaMemcpyDefault,
                       c->s));
  CK(cudaStreamSynchronize(c->s));
  return PASM_OK;
}

// loss and gradient for the batch already in nn.R (n x ldk2); gradient in nn.grad
static void nn_loss_grad_dev(pasm_ctx* c, int level, int k, int ldk2) {
  auto& nn = c->nn;
  const Launch L = launcher(c);
  LevelDev& v = c->lv[(size_t)level];
  NNGrid g{nn.nx[(size_t)level], nn.ny[(size_t)level], ldk2, k};
  // a learned-smoother context trains layer 2 on the tensor cores (the form its V-cycles run),
  // others on float32 CUDA cores
  const bool tc = c->opts.smoother == PASM_LEARNED && nn_tc_supported(ldk2);
  if (tc) nn_forward_train_tc(L, g, nn.buf, nn.W, nn.w2f, nn.R, nn.D, nn.err);
  else nn_forward(L, g, nn.buf, nn.W, nn.R, nn.D);
  rowop<float>(L, OP_RESID, v.A, nn.D, nn.R, nullptr, nullptr, 0.f, nn.X, ldk2);   // E = R - A D
  nn_column_norms(L, v.n, ldk2, nn.R, nn.X, nn.partial, nn.norms);
  nn_loss_seed(L, (int64_t)v.n * ldk2, ldk2, k, nn.X, nn.norms, nn.Es, nn.loss);
  rowop<float>(L, OP_SPMM, v.A, nn.Es, nullptr, nullptr, nullptr, 0.f, nn.gD, ldk2);  // dL/dD = A^T Es
  if (tc) nn_backward_tc(L, g, nn.buf, nn.W, nn.w2t, nn.R, nn.gD, nn.grad, nn.err);
  else nn_backward(L, g, nn.buf, nn.W, nn.R, nn.gD, nn.grad);
}

int pasm_nn_loss_grad(pasm_ctx* c, int level, int k, const float* R, double* loss, float* grad) {
  int r = nn_level_check(c, level, k);
  if (r) return r;
  if (!R) return PASM_EINVAL;
  Scope sc(c);
  const int n = c->lv[(size_t)level].n, ldk2 = ldk_for(k);
  r = nn_ensure(c, (int64_t)n * ldk2, (int64_t)n * ldk2, true);
  if (!r) r = put_block_f(c, R, c->nn.R, n, k, ldk2);
  if (r) return r;
  nn_loss_grad_dev(c, level, k, ldk2);
  if (loss) CK(cudaMemcpyAsync(loss, c->nn.loss, sizeof(double), cudaMemcpyDefault, c->s));
  if (grad) CK(cudaMemcpyAsync(grad, c->nn.grad, sizeof(float) * kNNWeights, cudaMemcpyDefault, c->s));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->s));
  return PASM_OK;
}

int pasm_nn_train(pasm_ctx* c, int level, int k, const float* R, int iters, float lr, double* losses) {
  int r = nn_level_check(c, level, k);
  if (r) return r;
  if (!R || iters < 0 || !(lr > 0.f)) return PASM_EINVAL;
  Scope sc(c);
  const int n = c->lv[(size_t)level].n, ldk2 = ldk_for(k);
  r = nn_ensure(c, (int64_t)n * ldk2, (int64_t)n * ldk2, true);
  if (!r) r = put_block_f(c, R, c->nn.R, n, k, ldk2);
  if (r) return r;
  auto& nn = c->nn;
  for (int it = 0; it < iters; ++it) {
    nn_loss_grad_dev(c, level, k, ldk2);
    if (losses) CK(cudaMemcpyAsync(losses + it, nn.loss, sizeof(double), cudaMemcpyDeviceToHost, c->s));
    nn_adam(launcher(c), kNNWeights, nn.W, nn.grad, nn.m, nn.v, lr, ++nn.t);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->s));
  // the tensor-core forward takes layers 1 and 3 as kernel parameters: refresh them and
  // drop a captured step graph that holds the old values
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return nn_refresh_host_weights(c);
}

int pasm_nn_capture_residuals(pasm_ctx* c, int level, float* R_out) {
  if (!c || !c->initialized || level < 1 || level >= c->nlev || !R_out) return PASM_EINVAL;
  if (c->opts.precision != PASM_MIXED) return PASM_EINVAL;
  Scope sc(c);
  const int n = c->lv[(size_t)level].n;
  int r = nn_ensure(c, 0, (int64_t)n * c->ldk, false);
  if (r) return r;
  c->capture_level = level;
  c->capture_buf = c->nn.Rt;
  sync_state(c);                               // the pair copy is rebuilt from U here
  bvp(c, c->nlev - 1, c->lam, c->U, c->YA);   // scratch output; the pair state is not touched
  c->capture_level = -1;
  c->capture_buf = nullptr;
  CK(cudaMemcpy2DAsync(R_out, sizeof(float) * c->k, c->nn.Rt, sizeof(float) * c->ldk, sizeof(float) * c->k, n,
                       cudaMemcpyDefault, c->s));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->s));
  return PASM_OK;
}

int pasm_nn_errors(pasm_ctx* c, int* count) {
  if (!c || !count || !c->nn.err) return PASM_ESTATE;
  CK(cudaMemcpy(count, c->nn.err, sizeof(int), cudaMemcpyDefault));
  return PASM_OK;
}

int pasm_nn_accepted(pasm_ctx* c, int* counts) {
  if (!c || !counts || !c->nn.accepted || c->k < 1) return PASM_ESTATE;
  CK(cudaMemcpy(counts, c->nn.accepted, sizeof(int) * c->k, cudaMemcpyDefault));
  return PASM_OK;
}

int pasm_trace_launches(pasm_ctx* c, int max, int* cls, int* rows, float* ms, double* bytes, double* flops,
                        int* count) {
  if (!c || !count) return PASM_EINVAL;
  const int n = (int)g_last_trace.size();
  *count = n;
  for (int q = 0; q < n && q < max; ++q) {
    if (cls) cls[q] = g_last_trace[(size_t)q].cls;
    if (rows) rows[q] = g_last_trace[(size_t)q].rows;
    if (ms) ms[q] = g_last_trace_ms[(size_t)q];
    if (bytes) bytes[q] = g_last_trace[(size_t)q].bytes;
    if (flops) flops[q] = g_last_trace[(size_t)q].flops;
  }
  return PASM_OK;
}

const char* pasm_kernel_class_name(int cls) {
  static const char* names[KC_N] = {"jacobi", "jacobi0", "resid", "spmm", "prolong", "dense", "outer_rhs",
                                    "outer_res", "axpy", "border", "colsum", "init", "secular", "update",
                                    "count", "cast", "nn", "proj", "cg", "sweep_update"};
  return (cls >= 0 && cls < KC_N) ? names[cls] : "unknown";
}

int pasm_coarse_eigs(pasm_ctx* c, double* lambda_H, double* Q) {
  if (!c) return PASM_EINVAL;
  if (lambda_H) std::memcpy(lambda_H, c->h_lamH.data(), sizeof(double) * c->NH);
  if (Q) std::memcpy(Q, c->h_Q.data(), sizeof(double) * (size_t)c->NH * c->NH);
  return PASM_OK;
}

int pasm_sizes(pasm_ctx* c, int64_t* n_fine, int32_t* n_coarse, int32_t* n_levels, int32_t* k) {
  if (!c) return PASM_EINVAL;
  if (n_fine) *n_fine = c->lv.back().n;
  if (n_coarse) *n_coarse = c->NH;
  if (n_levels) *n_levels = c->nlev;
  if (k) *k = c->k;
  return PASM_OK;
}

int pasm_last_launches(pasm_ctx* c, int* launches) {
  if (!c || !launches) return PASM_EINVAL;
  *launches = c->last_launches;
  return PASM_OK;
}

}  // extern "C"
