// Host-side launchers of the PASM device kernels (implemented in kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace pasm {

// Device CSR matrix with float64 values and an optional float32 shadow.
struct DCsr {
  int n_rows = 0, n_cols = 0;
  int64_t nnz = 0;
  int* rp = nullptr;
  int* ci = nullptr;
  double* v64 = nullptr;
  float* v32 = nullptr;
  float2* vff = nullptr;  // (hi, lo) float split of v64 for the double-float kernels (mixed precision)
  bool exact32 = false;   // every value is a float32 (lo = 0): the double-float products drop that term
  // (M of a level only) on M's pattern, A's split value beside M's: (a hi, a lo, m hi, m lo), a = 0
  // where A has no entry; present when A's pattern lies inside M's, for one gather of both products
  float4* am = nullptr;
  // omega a_ij / a_jj (A only): the values of the second Jacobi sweep from a zero start
  double* w64 = nullptr;
  float* w32 = nullptr;
};

template <typename T> inline const T* vals(const DCsr& m);
template <> inline const double* vals<double>(const DCsr& m) { return m.v64; }
template <> inline const float* vals<float>(const DCsr& m) { return m.v32; }
template <typename T> inline const T* scaled_vals(const DCsr& m);
template <> inline const double* scaled_vals<double>(const DCsr& m) { return m.w64; }
template <> inline const float* scaled_vals<float>(const DCsr& m) { return m.w32; }

// Kernel classes for tracing (keep in sync with PASM_KC_* in pasm.h).
enum KernelClass {
  KC_JACOBI = 0, KC_JACOBI0, KC_RESID, KC_SPMM, KC_PROLONG, KC_DENSE, KC_OUTER_RHS, KC_OUTER_RES, KC_AXPY,
  KC_BORDER, KC_COLSUM, KC_INIT, KC_SECULAR, KC_UPDATE, KC_COUNT, KC_CAST, KC_NN, KC_PROJ, KC_CG, KC_SWEEP_UPDATE, KC_N
};

// Host-side event recorder (defined in pasm.cu); null when not tracing.
struct Tracer;
void tracer_begin(Tracer* t, cudaStream_t s, int cls, double bytes, double flops);
void tracer_rows(Tracer* t, int rows);
void tracer_end(Tracer* t, cudaStream_t s);

// Launch bookkeeping shared by every launcher: the stream, a launch counter
// and an optional tracer that brackets each launch with CUDA events and
// records its algorithmic bytes and flops.
struct Launch {
  cudaStream_t s = nullptr;
  int* counter = nullptr;
  Tracer* tr = nullptr;
  int geo = 0;  // row-group kernels: 16-byte chunks per thread (0 = default; set by the autotuner)
  int rpt = 0;  // float32 row kernels: row blocks each block walks (0 = by size; set by the autotuner)
  void begin(int cls, double bytes, double flops) const { if (tr) tracer_begin(tr, s, cls, bytes, flops); }
  void rows(int n) const { if (tr) tracer_rows(tr, n); }
  void bump() const {
    if (counter) ++*counter;
    if (tr) tracer_end(tr, s);
  }
};

enum RowOp { OP_JACOBI = 0, OP_RESID = 1, OP_SPMM = 2, OP_SPMM_ADD = 3 };

// out = op(S, X, Y, Z) row by row on n x ldk block vectors (row-major):
//   OP_JACOBI : out = Z + omega * dinv .* (Y - S X)      (damped Jacobi sweep)
//   OP_RESID  : out = Y - S X                            (residual)
//   OP_SPMM   : out = S X                                (restriction / product)
//   OP_SPMM_ADD: out = Y + S X                           (prolongate and correct)
template <typename T>
void rowop(const Launch& L, RowOp op, const DCsr& S, const T* X, const T* Y, const T* Z, const T* dinv,
           T omega, T* out, int ldk);
// out = xn + omega D^{-1} (F - A xn), xn = X + P Ec (prolongation fused with the first float32
// post-smoothing sweep; the operations of rowop(OP_SPMM_ADD) then rowop(OP_JACOBI), in their order)
void prolong_jacobi(const Launch& L, const DCsr& A, const DCsr& P, const float* X, const float* Ec, const float* F,
                    const float* dinv, float omega, float* out, int ldk);

// out = omega * dinv .* F  (first Jacobi sweep from a zero guess)
template <typename T>
void jacobi_zero(const Launch& L, int n, const T* dinv, T omega, const T* F, T* out, int ldk);

// Fused V-cycle kernels (see kernels.cu):
//   jacobi2_zero:   out = two Jacobi sweeps on A e = F from e = 0
//   resid_restrict: out (coarse) = R (F - A E)
template <typename T>
void jacobi2_zero(const Launch& L, const DCsr& A, const T* dinv, T omega, const T* F, T* out, int ldk);
template <typename T>
void resid_restrict(const Launch& L, const DCsr& R, const DCsr& A, const T* E, const T* F, T* out, int ldk);
// out (coarse) = R F - RA E with RA = R A formed at setup (float32 cycles; same value as
// resid_restrict in exact arithmetic)
void restrict_first(const Launch& L, const DCsr& R, const DCsr& RA, const float* E, const float* F, float* out,
                    int ldk);

// Fd = lam .* (M U)  and  R = Fd - A U  (float64 arithmetic, R stored as TV)
template <typename TV>
void outer_rhs_residual(const Launch& L, const DCsr& A, const DCsr& M, const double* lam, const double* U,
                        double* Fd, TV* R, int ldk);
// R = Fd - A X  (float64 arithmetic, stored as TV)
template <typename TV>
void outer_residual(const Launch& L, const DCsr& A, const double* Fd, const double* X, TV* R, int ldk);
// X = B + E (float64 result; X may alias B)
template <typename TV>
void outer_axpy(const Launch& L, int n, const double* B, const TV* E, double* X, int ldk);

// YA = A X, YM = M X and per-column partial sums of X.*YA, X.*YM into
// partials[nblk][2][ldk]; returns the number of blocks used.
int border_products(const Launch& L, const DCsr& A, const DCsr& M, const double* X, double* YA, double* YM,
                    double* partials, int ldk, int max_blocks);
// out[q*ldk + c] = sum_b partials[(b*nq + q)*ldk + c]
void column_sums(const Launch& L, const double* partials, int nblk, int nq, int ldk, double* out);
// Per-block column partials [block][2][ldk] of sum r^2 and sum u (lambda M u) (eigen-residual
// report); returns the number of blocks.
template <typename TR>
int residual_partials(const Launch& L, int n, int ldk, const TR* R, bool ff, const double* Fd, const double* U,
                      double* partials, int max_blocks);

// C (m x ldk) = op(D) (m x p) * B (p x ldk); D row-major with leading dim ldd;
// trans: op(D) = D^T (then D is p x m).
template <typename T>
void dense_mm(const Launch& L, int m, int p, const T* D, int ldd, bool trans, const T* B, T* C, int ldk);

// Coarse initial state: W0[j][c] = Q[j][c] / sqrt(lamH[c]) for c < k, 0 otherwise;
// lam[c] = lamH[c] (c < k).
void coarse_init(const Launch& L, int NH, int k, const double* Q, const double* lamH, double* W0, double* lam,
                 int ldk);

struct SecularArgs {
  int NH, k, ldk;
  int cs;                 // CTAs per pair: a thread-block cluster sharing the root solves (set by secular_select)
  const double* lamH;     // NH, ascending
  const double* bq;       // NH x ldk: Q^T b
  const double* cq;       // NH x ldk: Q^T c
  const double* beta;     // ldk
  const double* zeta;     // ldk
  double* lam;            // ldk: in = lambda^(l), out = lambda^(l+1)
  double* alpha;          // ldk out
  double* g;              // NH x ldk out: coarse coefficients in the Q basis
  int* active;            // ldk in/out
  int* upd;               // ldk out: 1 = pair updated this step
  int* steps;             // ldk in/out
  int* status;            // ldk out
  double tol;
  // residual guard (null: none): rsum[i] = sum_j r_ji^2, rsum[ldk + i] = sum_j u_ji (lambda_i M u_i)_j
  // of the state the step started from; a pair freezes only if sqrt(rsum[i] / (lambda_i rsum[ldk + i]))
  // (the relative residual of Section 5) is at most res_tol
  const double* rsum = nullptr;
  double res_tol = 0.0;
  int score_norm;
  int window;             // half-width of the first root window
  int* diag;              // diagnostics: [0] = roots solved, [1] = full solves, [2] = iteration caps hit
};
void secular_select(const Launch& L, const SecularArgs& a);
// Raise the kernel's dynamic shared memory limit for a coarse dimension NH (once per setup).
cudaError_t secular_prepare(int NH);

// U[row][c] = upd[c] ? alpha[c] * X[row][c] + (P W)[row][c] : U[row][c]
void update_pairs(const Launch& L, const DCsr& P, const double* W, const double* X, const double* alpha,
                  const int* upd, double* U, int ldk);
// Same with P = identity (single-level hierarchy): U = alpha X + W.
void update_pairs_identity(const Launch& L, int n, const double* W, const double* X, const double* alpha,
                           const int* upd, double* U, int ldk);

// ----------------------------------------------------------------------------------------------
// Conjugate-gradient smoothing (kernels.cu): nu CG steps for A x = F, every
// column its own CG.  x_zero: start from x = 0 (X is written, not read).
// R, P, Q are n x ldk scratch blocks; the work arrays hold per-block partial
// sums (max_blocks x ldk) and the per-column scalars r.r, alpha, beta.
struct CgWork {
  double* partial = nullptr;
  int max_blocks = 0;
  double *rr = nullptr, *alpha = nullptr, *beta = nullptr;
};
template <typename T>
void cg_smooth(const Launch& L, const DCsr& A, const T* F, T* X, bool x_zero, T* R, T* P, T* Q, const CgWork& w,
               int ldk, int nu);

// ----------------------------------------------------------------------------------------------
// Double-float versions of the float64-accuracy kernels (ff.cu), used in mixed
// precision.  A block vector "in pairs" holds (hi, lo) floats in place of each
// float64 (same size and layout); matrices go through S.vff.
// Fd = lam .* (M U) (pairs), R = Fd - A U (float32); U in pairs.
void outer_rhs_residual_ff(const Launch& L, const DCsr& A, const DCsr& M, const double* lam, const double* U,
                           double* Fd, float* R, int ldk);
// R = Fd - A X (float32); Fd and X in pairs.
void outer_residual_ff(const Launch& L, const DCsr& A, const double* Fd, const double* X, float* R, int ldk);
// YA = A X, YM = M X (X, YA, YM in pairs) and float64 partial sums as border_products.
int border_products_ff(const Launch& L, const DCsr& A, const DCsr& M, const double* X, double* YA, double* YM,
                       double* partials, int ldk, int max_blocks);
// Last float32 Jacobi sweep of the top-level V-cycle fused with X = B + e'
// (e' = E + omega dinv .* (F - A E), never stored; X in pairs, B in pairs if b_ff).
void jacobi_axpy_ff(const Launch& L, const DCsr& A, const float* E, const float* F, const float* dinv, float omega,
                    const double* B, bool b_ff, double* X, int ldk);
// out = S X; x_ff / out_ff: X / out in pairs (else float64).
void spmm_ff(const Launch& L, const DCsr& S, const double* X, bool x_ff, double* out, bool out_ff, int ldk);
// outA = S XA, outM = S XM in one launch (each as spmm_ff computes it)
void spmm2_ff(const Launch& L, const DCsr& S, const double* XA, const double* XM, bool x_ff, double* outA,
              double* outM, bool out_ff, int ldk);
// X = B + E (X in pairs; B in pairs if b_ff, else float64; X may alias B).
void axpy_ff(const Launch& L, int n, const double* B, bool b_ff, const float* E, double* X, int ldk);
// Conversions of total entries: float64 -> pairs (may be in place), pairs -> float64.
void to_ff(const Launch& L, int64_t total, const double* in, double* out);
void from_ff(const Launch& L, int64_t total, const double* in, double* out);
// U = alpha X + P W for updated pairs (X in pairs, W in pairs if w_ff); P ==
// nullptr means P = identity on n rows.  With U given, U is float64 and Usplit
// (optional) receives it as pairs; with U null the result goes to Usplit alone
// (the pair state).  Frozen pairs are not touched.
void update_pairs_ff(const Launch& L, const DCsr* P, int n, const double* W, bool w_ff, const double* X,
                     const double* alpha, const int* upd, double* U, double* Usplit, int ldk);

// ----------------------------------------------------------------------------------------------
// Float64-accurate dense product C = A B on the tensor cores (proj_tc.cu).
// A (m x K) is split once into S = 8 signed 7-bit digit planes per row
// (error-free slicing in the manner of Ozaki, Ogita, Oishi and Rump), B (K x n)
// per call per column; the digit-plane products run as bf16 x bf16 -> f32
// tcgen05 MMAs over chunks of 32 inner indices, whose integer sums are exact in
// float32; they are added exactly in 64-bit integers and rounded once.
struct ProjPlan {
  int beta = 0, S = 0;  // digit width and digits per operand
};
struct SplitMat {
  int m = 0, K = 0, Kpad = 0, mtiles = 0;
  ProjPlan plan;
  const uint16_t* planes = nullptr;  // bf16 [mtiles][S][Kpad/8][16][8][8] (tensor-core operand layout)
  const int* rexp = nullptr;          // m row exponents: |A[i][j]| < 2^rexp[i]
};
// Plan for inner dimension K (false if K is too large for the exact sums).
bool proj_plan(int K, ProjPlan& plan);
// Split the row-major m x K host matrix A per the plan: planes (bf16 bits) and
// row exponents, in the layout SplitMat describes.
void proj_split_host(const double* A, int m, int K, const ProjPlan& plan, int& Kpad, int& mtiles,
                     std::vector<uint16_t>& planes, std::vector<int>& rexp);
// Device scratch of proj_tc for m rows and up to ncols_max columns: 64-bit
// words of the integer sums and per-tile tickets, both zero-initialised once
// (each call leaves them zero).
size_t proj_scratch_words(int m, int ncols_max);
size_t proj_tickets(int m, int ncols_max);
cudaError_t proj_tc_prepare();
// C = A B for ncols output columns: column c < ldk comes from B0/C0 column c,
// column c >= ldk from B1/C1 column c - ldk (B1, C1 unused when ncols <= ldk).
// B0, B1, C0, C1 are K x ldk and m x ldk row-major.  err counts bounded waits
// that gave up (the affected chunk then adds nothing to its tile).
void proj_tc(const Launch& L, const SplitMat& A, const double* B0, const double* B1, double* C0, double* C1,
             int ldk, int ncols, unsigned long long* hl, unsigned int* tickets, int* err, int wait_limit = 0,
             int skip_mma = 0);

// *out = number of nonzero entries of active[0..k)
void count_active(const Launch& L, const int* active, int k, int* out);

// cast between float64 and float32 block vectors
void cast_d2f(const Launch& L, const double* in, float* out, int64_t count);

}  // namespace pasm
