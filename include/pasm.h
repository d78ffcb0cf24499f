/*
 * pasm.h -- C ABI of the GB300 (sm_103a) parallel augmented subspace method.
 *
 * The library computes the k smallest eigenpairs of the generalized finite
 * element eigenproblem A u = lambda M u (Section 2: the discrete problem on the
 * linear element space V_h) with the parallel augmented subspace method of
 * Xu, Xie and Zhang: Algorithm 1 (one correction step) applied to all k pairs
 * at once, inside Algorithm 2 (the parallel scheme).  The k pairs never
 * exchange data (Section 3.2: the correction runs independently per pair and
 * needs no orthogonalisation), so the library batches them: every block vector
 * is an n x k row-major array and every sparse product reuses each matrix entry
 * k times.
 *
 * Conventions shared by all entry points
 *   - Level 0 is the coarse space V_H; level n_levels-1 is the finest V_h.
 *     P[l] is the interpolation from level l to level l+1 (n_{l+1} x n_l), so
 *     the nested spaces of Section 3.1 are given by their prolongations.
 *   - CSR arrays are HOST pointers owned by the caller.  The library copies them
 *     during pasm_setup; the caller may free them afterwards.
 *   - Block vectors U are n x k, row-major (U[i*k + j] = entry i of pair j),
 *     float64.  Vector and eigenvalue arguments may be host or device pointers
 *     (the library detects which; copies run on the context's stream).
 *   - Eigenvectors are a-normalised, a(u, u) = u^T A u = 1 (the normalisation
 *     of the weak eigenproblem in Section 2), with the sign fixed by
 *     b(u_new, u~) > 0 (u~ = the multigrid iterate of the step).
 *   - Every function returns a pasm_status code (0 = success).  On error no
 *     output is written unless stated.  pasm_strerror names the code.
 *   - A context owns all its device memory and its CUDA graph; it is not
 *     thread-safe; distinct contexts are independent.
 */
#ifndef PASM_H
#define PASM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PASM_OK = 0,
  PASM_EINVAL = 1,      /* malformed CSR, shape mismatch, bad option or size   */
  PASM_EK_TOO_BIG = 2,  /* k > dim V_H: the coarse space cannot seed k pairs   */
  PASM_ENOMEM = 3,      /* device or host allocation failed                     */
  PASM_ECUDA = 4,       /* a CUDA runtime call failed                           */
  PASM_ENOTCONV = 5,    /* max_steps reached with pairs still active            */
  PASM_EDEGENERATE = 6, /* bordered mass matrix singular for a pair (u~ in V_H) */
  PASM_ENAN = 7,        /* a NaN/Inf appeared in a pair                         */
  PASM_ESTATE = 8,      /* call out of order (e.g. pasm_step before pasm_init)  */
  PASM_ENOTPD = 9,      /* coarse A_H or M_H not symmetric positive definite    */
  PASM_ETIMEOUT = 10    /* a bounded device wait gave up (tensor-core kernel)   */
} pasm_status;

/* Per-pair status values written by pasm_get / pasm_solve. */
enum {
  PASM_PAIR_ACTIVE = 0,     /* still iterating                                 */
  PASM_PAIR_CONVERGED = 1,  /* |lambda_new - lambda_old| / lambda_new < tol    */
  PASM_PAIR_DEGENERATE = 2, /* kept its previous pair this step (u~ in V_H)     */
  PASM_PAIR_NAN = 3         /* frozen after a NaN/Inf                           */
};

enum { PASM_FP64 = 0, PASM_MIXED = 1 };           /* precision of the V-cycles   */
enum { PASM_SCORE_A = 0, PASM_SCORE_B = 1 };      /* normalisation in the score  */
enum { PASM_INIT_COARSE = 0, PASM_INIT_NESTED = 1 };
enum { PASM_JACOBI = 0, PASM_LEARNED = 1, PASM_CG = 2 };  /* multigrid smoother     */
enum { PASM_PROJ_TENSOR = 0, PASM_PROJ_FP64 = 1 };  /* coarse projection product */

/* Kernel kinds whose tile shape the autotuner chooses (see pasm_tiles). */
enum {
  PASM_TILE_JACOBI = 0,         /* damped Jacobi sweep                               */
  PASM_TILE_JACOBI2_ZERO,       /* two sweeps from a zero guess (float32 cycles)     */
  PASM_TILE_RESID_RESTRICT,     /* residual + restriction (float32 cycles)           */
  PASM_TILE_RESID,              /* residual (float64 cycles)                         */
  PASM_TILE_RESTRICT,           /* restriction (float64 cycles)                      */
  PASM_TILE_PROLONG,            /* prolongate and correct                            */
  PASM_TILE_OUTER_RHS,          /* f = lambda M u and the first outer residual       */
  PASM_TILE_OUTER_RES,          /* later outer residuals                             */
  PASM_TILE_BORDER,             /* A u~, M u~ and their dot products                 */
  PASM_TILE_CHAIN_R,            /* restriction chain of A u~, M u~                   */
  PASM_TILE_CHAIN_P,            /* prolongation chain of u_H                         */
  PASM_TILE_UPDATE,             /* u = alpha u~ + P_c u_H                            */
  PASM_TILE_PROLONG_SWEEP,      /* prolongation fused with the first post-smoothing
                                   sweep (float32 cycles)                            */
  PASM_TILE_RESTRICT_FIRST,     /* coarse residual as R f - (R A) e (float32 cycles) */
  PASM_TILE_N
};

/* A sparse matrix in CSR form: n_rows x n_cols, nnz entries, 32-bit indices,
 * float64 values, column indices ascending within each row. */
typedef struct {
  int32_t n_rows;
  int32_t n_cols;
  int64_t nnz;
  const int32_t* row_ptr; /* n_rows + 1 entries, row_ptr[0] = 0, nondecreasing */
  const int32_t* col;     /* nnz entries in [0, n_cols)                         */
  const double* val;      /* nnz entries                                        */
} pasm_csr;

/* Method parameters.  pasm_default_opts fills the defaults in brackets. */
typedef struct {
  double omega;        /* damped Jacobi weight [2/3]                             */
  int nu_pre;          /* pre-smoothing sweeps per level [2]                     */
  int nu_post;         /* post-smoothing sweeps per level [2]                    */
  int cycles_per_step; /* V-cycles per correction step (Algorithm 1 step 1) [2]  */
  int max_steps;       /* step limit in pasm_solve [100]                         */
  int precision;       /* PASM_FP64: all arithmetic float64; PASM_MIXED: V-cycles
                          in float32 as a defect correction under float64
                          residuals, bordering and small eigensolve [PASM_FP64] */
  int score_norm;      /* PASM_SCORE_A (a-normalised Ritz vectors, as the paper
                          states the normalisation) or PASM_SCORE_B [A]          */
  int init;            /* PASM_INIT_COARSE: prolongated coarse eigenpairs
                          (Algorithm 2 step 1 on V_H, then step 2(B));
                          PASM_INIT_NESTED: additionally one correction step on
                          every intermediate level (Algorithm 2 step 2(A))
                          [PASM_INIT_COARSE]                                     */
  int use_graph;       /* capture the finest-level step in a CUDA graph [1]      */
  int smoother;        /* PASM_JACOBI (damped Jacobi sweeps); PASM_CG: nu_pre /
                          nu_post conjugate-gradient steps, each pair its own
                          unpreconditioned CG restarted at every smoothing (the
                          smoother of the paper's experiments, Section 5.1);
                          PASM_LEARNED: on levels given a grid by pasm_nn_setup
                          the first post-smoothing sweep is the learned step
                          with a per-pair Jacobi fallback (mixed precision
                          only) [PASM_JACOBI]                                   */
  int projection;      /* PASM_PROJ_TENSOR: the dense coarse products Q^T b,
                          Q^T c and Q g run on the tensor cores (tcgen05) in
                          exact digit planes, added exactly and rounded once
                          to float64 (error about 2^-56 N_H max|Q| max|b|);
                          PASM_PROJ_FP64: float64 CUDA-core products
                          [PASM_PROJ_TENSOR]                                    */
  int autotune;        /* 1: at the first pasm_init for a block width, time each
                          row-group tile shape (16-byte chunks per thread: 1, 2,
                          4, 8) of every sparse kernel on every level with at
                          least 16384 rows and keep the fastest; 0: fixed
                          default shapes [1]                                     */
  double res_tol;      /* > 0: a pair that meets the |dlambda| test is kept
                          iterating while its relative residual
                          ||A u - lambda M u|| / (|lambda| ||u||_M) (the stopping
                          quantity of Section 5) exceeds res_tol, so a freeze on
                          a value that is not an eigenvalue is not reported as
                          converged.  Inside every step (pasm_step, the captured
                          graph) for the state the step starts from, summed in
                          float64 from the step's first outer residual; pasm_solve
                          and pasm_batch_solve also check the state after the
                          step with pasm_residuals on the steps where pairs
                          freeze.  0: the |dlambda| test alone [0]               */
} pasm_opts;

typedef struct pasm_ctx pasm_ctx;

/* Fill *opts with the defaults listed above. */
void pasm_default_opts(pasm_opts* opts);

/* Build a context: validate and copy the level hierarchy to the device, form
 * the float32 shadows used by PASM_MIXED, and compute the coarse generalized
 * eigendecomposition A_H Q = M_H Q Lambda_H (Q^T M_H Q = I) once (Algorithm 2
 * step 1 on V_H).
 *   out       receives the context (NULL on error).
 *   n_levels  >= 1 levels; A[l], M[l] square n_l x n_l symmetric (the library
 *             relies on symmetry and does not check it), P[l] n_{l+1} x n_l.
 *   opts      may be NULL (defaults).
 *   stream    a cudaStream_t to run on, or NULL for the default stream.
 * Errors: PASM_EINVAL (shapes/CSR), PASM_ENOTPD (A_H or M_H), PASM_ENOMEM,
 * PASM_ECUDA. */
int pasm_setup(pasm_ctx** out, int n_levels, const pasm_csr* A, const pasm_csr* M,
               const pasm_csr* P, const pasm_opts* opts, void* stream);

/* Set the k pairs to iterate (Algorithm 2).  lambda0 (k) and U0 (n x k) give
 * an explicit starting state (host or device; both NULL = the start selected
 * by opts.init).  tol is the per-pair freeze threshold on the relative
 * eigenvalue change.  Errors: PASM_EK_TOO_BIG (k > dim V_H when starting from
 * the coarse space), PASM_EINVAL (k < 1 or one of lambda0/U0 NULL). */
int pasm_init(pasm_ctx* ctx, int k, double tol, const double* lambda0, const double* U0);

/* One correction step (Algorithm 1) for every active pair on the finest
 * level: k multigrid solves of A u^ = lambda M u started from u, then the
 * bordered eigenproblem on V_H + span{u~} and the selection of the Ritz pair
 * with the largest |b(u_{H,h}, u~)|.  Runs asynchronously on the context's
 * stream; *n_active (may be NULL) receives the number of pairs still active,
 * which synchronises the stream.  Errors: PASM_ESTATE, PASM_ECUDA. */
int pasm_step(pasm_ctx* ctx, int* n_active);

/* Copy the current state out: lambda (k), U (n x k), steps (k, correction
 * steps taken per pair), status (k, PASM_PAIR_*).  Any pointer may be NULL.
 * Synchronises the stream.  Returns PASM_ETIMEOUT (outputs still written) if a
 * tensor-core projection has ever given up a bounded wait in this context. */
int pasm_get(pasm_ctx* ctx, double* lambda, double* U, int* steps, int* status);

/* pasm_init + pasm_step until no pair is active or opts.max_steps, then
 * pasm_get.  Returns PASM_ENOTCONV (outputs still written) if pairs remain
 * active. */
int pasm_solve(pasm_ctx* ctx, int k, double tol, const double* lambda0, const double* U0,
               double* lambda_out, double* U_out, int* steps_out, int* status_out);

/* Algorithm 1 step 1 alone: Uhat = result of opts.cycles_per_step V-cycles for
 * A x = lambda M U started from x = U (all k columns).  lambda (k), U and
 * Uhat (n x k) host or device.  Does not touch the context's pair state except
 * for scratch; needs pasm_init with the same k first.  Errors: PASM_ESTATE. */
int pasm_bvp(pasm_ctx* ctx, const double* lambda, const double* U, double* Uhat);

/* Algorithm 1 step 2 alone: for each column u~ of Uhat, the bordered
 * eigenproblem on V_H + span{u~}, its selected a-normalised Ritz pair
 * (lambda_out, U_out) and the bordering scalars beta = a(u~,u~),
 * zeta = b(u~,u~) (either may be NULL).  lambda_prev (k) is the eigenvalue
 * the Ritz roots are searched around.  Needs pasm_init with the same k. */
int pasm_augmented(pasm_ctx* ctx, const double* lambda_prev, const double* Uhat,
                   double* lambda_out, double* U_out, double* beta, double* zeta);

/* The projection of Algorithm 1 step 2 onto the coarse eigenbasis alone:
 * bq = Q^T b and cq = Q^T c for the k columns of b and c (N_H x k row-major,
 * host or device; b = P_c^T A u~ and c = P_c^T M u~ are the bordering vectors
 * of the bordered matrix form in Section 3.1, and Q is the M_H-orthonormal
 * coarse eigenbasis of pasm_coarse_eigs).  The product follows
 * opts.projection.  Needs pasm_init (for k); uses the coarse scratch of a
 * step.  Errors: PASM_ESTATE, PASM_EINVAL (NULL pointer), PASM_ETIMEOUT (a
 * tensor-core wait gave up; outputs then incomplete). */
int pasm_project(pasm_ctx* ctx, const double* b, const double* c, double* bq, double* cq);

/* The tile shapes in use on `level`: chunks_per_thread[PASM_TILE_N] receives,
 * per kernel kind, the 16-byte chunks of a block-vector row each thread
 * handles (0 = the default shape: one chunk, or as many as keep at most 32
 * threads per row).  For PASM_TILE_JACOBI2_ZERO, PASM_TILE_RESID_RESTRICT and
 * PASM_TILE_PROLONG_SWEEP, -1 means the autotuner timed the fused kernel
 * slower than its unfused pair (one sweep from zero + one sweep; residual +
 * restriction; prolongation + sweep) on this level, which then runs instead.
 * PASM_TILE_RESTRICT_FIRST is above 0 only where the autotuner timed the
 * restriction-first form of the coarse residual, R f - (R A) e with R A formed
 * at setup, faster than both forms of R (f - A e); it then runs instead.
 * Errors: PASM_EINVAL. */
int pasm_tiles(pasm_ctx* ctx, int level, int* chunks_per_thread);

/* Row blocks per thread block in use on `level`: rows_per_block[PASM_TILE_N]
 * receives, per kernel kind, how many consecutive row blocks (of 256 / threads
 * per row rows) one thread block walks -- 1 or 4 as the autotuner timed the
 * row kernels of the mixed-precision step (float32 sweeps, residuals and
 * transfers; double-float outer residuals, transfer chains and update), 0 for
 * kinds it does not choose this for and in float64 mode (these take 1).
 * Errors: PASM_EINVAL. */
int pasm_tile_rows(pasm_ctx* ctx, int level, int* rows_per_block);

/* Set the tile shapes of `level` (a tuning cache: the values pasm_tiles and
 * pasm_tile_rows returned for a context of the same hierarchy, block width and
 * precision).  chunks_per_thread[PASM_TILE_N]: 0, 1, 2, 4 or 8, and -1 only for
 * PASM_TILE_JACOBI2_ZERO, PASM_TILE_RESID_RESTRICT and PASM_TILE_PROLONG_SWEEP
 * (PASM_TILE_RESTRICT_FIRST above 0 selects that form, mixed precision only);
 * rows_per_block[PASM_TILE_N] (NULL: all 0): 0, 1 or 4.  A shape that does not
 * fit the block width runs the default shape.  The autotuner of a later
 * pasm_init replaces them unless opts.autotune is 0 or the block width is the
 * one already tuned.  Drops a captured step graph.  Errors: PASM_EINVAL (NULL
 * chunks, bad level or value). */
int pasm_set_tiles(pasm_ctx* ctx, int level, const int* chunks_per_thread, const int* rows_per_block);

/* *kind = PASM_PROJ_TENSOR if the tensor-core projection is in use, else
 * PASM_PROJ_FP64. */
int pasm_projection_kind(pasm_ctx* ctx, int* kind);

/* Relative eigen-residuals of the current pairs, the stopping quantity of the
 * paper's experiments (Section 5) with u scaled to unit M-norm:
 * res[i] = ||A u_i - lambda_i M u_i||_2 / (|lambda_i| ||u_i||_M), i < k, in
 * the context's precision (double-float in mixed mode).  Uses the step's
 * scratch buffers (not during a step); synchronises the context's stream.
 * Errors: PASM_EINVAL (NULL), PASM_ESTATE (before pasm_init), PASM_ECUDA. */
int pasm_residuals(pasm_ctx* ctx, double* res);

/* Counters of the batched bordered eigensolve (Section 3.1's selection by
 * secular roots) since the last pasm_init: out[0] = roots solved in the first
 * window (root 0 and the roots next to lambda^(l)), out[1] = windows whose
 * Parseval certificate failed (more roots were solved), out[2] = root
 * iterations that reached their cap.  Synchronises the context's stream.
 * Errors: PASM_EINVAL, PASM_ESTATE (before pasm_init), PASM_ECUDA. */
int pasm_secular_stats(pasm_ctx* ctx, int* out);

/* The coarse eigendecomposition computed at setup: Lambda_H (N_H, ascending)
 * and Q (N_H x N_H row-major, column j = eigenvector j, Q^T M_H Q = I); host
 * pointers, either may be NULL. */
int pasm_coarse_eigs(pasm_ctx* ctx, double* lambda_H, double* Q);

/* Sizes: finest n, coarse N_H, number of levels, current k (0 before init). */
int pasm_sizes(pasm_ctx* ctx, int64_t* n_fine, int32_t* n_coarse, int32_t* n_levels, int32_t* k);

/* Number of kernel launches the last pasm_step issued (graph nodes when a
 * graph is used). */
int pasm_last_launches(pasm_ctx* ctx, int* launches);

/* Kernel classes reported by pasm_trace_step. */
enum {
  PASM_KC_JACOBI = 0,   /* damped Jacobi sweep (multigrid smoother)               */
  PASM_KC_JACOBI0,      /* first sweep from a zero guess                          */
  PASM_KC_RESID,        /* multigrid residual f - A e                             */
  PASM_KC_SPMM,         /* restriction P^T r and float64 transfer chains          */
  PASM_KC_PROLONG,      /* prolongate and correct e += P e_c                      */
  PASM_KC_DENSE,        /* coarse dense products (A_H^-1, Q^T, Q)                 */
  PASM_KC_OUTER_RHS,    /* f = lambda M u and the first float64 residual          */
  PASM_KC_OUTER_RES,    /* later float64 residuals of the defect correction       */
  PASM_KC_AXPY,         /* x += e                                                 */
  PASM_KC_BORDER,       /* A u~, M u~, beta, zeta partial sums                    */
  PASM_KC_COLSUM,       /* reduction of the partial sums                          */
  PASM_KC_INIT,         /* coarse initial state                                   */
  PASM_KC_SECULAR,      /* bordered eigenproblem: secular roots and selection     */
  PASM_KC_UPDATE,       /* u = alpha u~ + P_c u_H                                 */
  PASM_KC_COUNT,        /* active-pair count                                      */
  PASM_KC_CAST,         /* precision conversion                                   */
  PASM_KC_NN,           /* learned smoother (convolutions, training, fallback)    */
  PASM_KC_PROJ,         /* coarse projections Q^T b, Q^T c, Q g on tensor cores   */
  PASM_KC_CG,           /* conjugate-gradient smoothing (vectors and scalars)     */
  PASM_KC_SWEEP_UPDATE, /* last Jacobi sweep fused with the outer update x += e    */
  PASM_KC_N
};

/* Run one correction step (same arithmetic as pasm_step, so the pair state
 * advances) eagerly with a CUDA event pair around every kernel launch, and
 * accumulate per kernel class: elapsed milliseconds, algorithmic bytes (the
 * compulsory traffic of each launch: matrices, gathered and streamed vectors
 * once), flops, and launch counts.  Each array has PASM_KC_N entries and may
 * be NULL.  Synchronises the stream. */
int pasm_trace_step(pasm_ctx* ctx, double* ms, double* bytes, double* flops, int* launches);

/* The launch list of the last pasm_trace_step: *count launches; for the first
 * `max` of them the class, rows of the matrix the launch runs on (0 when not
 * a row kernel), event-timed milliseconds, algorithmic bytes and flops.  Any
 * array may be NULL. */
int pasm_trace_launches(pasm_ctx* ctx, int max, int* cls, int* rows, float* ms, double* bytes, double* flops,
                        int* count);

/* A static name of kernel class cls ("jacobi", "border", ...). */
const char* pasm_kernel_class_name(int cls);

/* ---- Learned post-smoother.  Not in the paper: the workload specification
 * asks for a small convolutional network standing in for damped Jacobi inside
 * the V-cycles of Algorithm 1 step 1.  Network: three bias-free 3x3
 * convolutions 1 -> 16 -> 16 -> 1, ReLU after the first two, made odd,
 * N(r) = (Nt(r) - Nt(-r)) / 2; on a level with an nx x ny grid view of its
 * interior nodes (x fastest, zero outside) it maps a residual r to a
 * correction.  Weights: 2592 float32, W1[3][3][1][16] | W2[3][3][16][16] |
 * W3[3][3][16][1], index [dy+1][dx+1][cin][cout] multiplying pixel
 * (y+dy, x+dx).  Training minimises L = mean_pairs |r - A N(r)|^2 / |r|^2 with
 * Adam.  All of it needs precision = PASM_MIXED (float32 cycles). */

/* Install the network: nx[l] = grid width of level l (n_l = nx * ny), 0 = do
 * not use it on that level; weights (host or device) are copied and the Adam
 * state is reset.  Errors: PASM_EINVAL (not mixed precision, n_l not a multiple
 * of nx[l], NULL). */
int pasm_nn_setup(pasm_ctx* ctx, const int32_t* nx, const float* weights);

/* Current weights (2592 float32, host or device). */
int pasm_nn_get_weights(pasm_ctx* ctx, float* weights);

/* D = N(R) for the k columns of R on level `level` (n_l x k float32 row-major,
 * host or device).  Synchronises. */
int pasm_nn_apply(pasm_ctx* ctx, int level, int k, const float* R, float* D);

/* loss L and its gradient dL/dW (2592 float32, host or device) for the
 * residual batch R (n_l x k float32) on level `level`. */
int pasm_nn_loss_grad(pasm_ctx* ctx, int level, int k, const float* R, double* loss, float* grad);

/* `iters` Adam steps (betas 0.9, 0.999, eps 1e-8, learning rate lr) on the
 * fixed batch R; losses[it] (host, may be NULL) receives L before step it. */
int pasm_nn_train(pasm_ctx* ctx, int level, int k, const float* R, int iters, float lr, double* losses);

/* Training data from the method's own iterations: run the multigrid solve of
 * Algorithm 1 step 1 on the current pairs (pasm_init first) and return the
 * residual f - A e on level `level` (>= 1) of the first V-cycle just before
 * its post-smoothing, n_l x k float32 (host or device).  The pair state is
 * not changed. */
int pasm_nn_capture_residuals(pasm_ctx* ctx, int level, float* R_out);

/* Per pair, how many learned steps were accepted (residual did not grow)
 * since pasm_init or pasm_nn_setup; counts has k entries (host or device). */
int pasm_nn_accepted(pasm_ctx* ctx, int* counts);

/* Number of tensor-core tiles of the learned smoother whose completion wait
 * timed out (their output was left unwritten) since pasm_nn_setup. */
int pasm_nn_errors(pasm_ctx* ctx, int* count);

/* Test hook of the tensor-core projection's bounded completion wait (its MMAs
 * commit to an mbarrier that one thread polls at most `wait_limit` times; 0 =
 * the library's limit, about 4 million polls).  With skip_mma != 0 the kernel
 * issues no MMA, so nothing arrives on that mbarrier and the wait runs out with
 * nothing in flight: pasm_project then returns PASM_ETIMEOUT and leaves its
 * outputs unspecified, and the context stays usable.  (0, 0) restores normal
 * operation.  Drops the context's captured step graph.  Errors: PASM_EINVAL. */
int pasm_debug_waits(pasm_ctx* ctx, int skip_mma, int wait_limit);

/* Bordering products of the correction step for callers that cannot allocate
 * device memory.  The paper has no counterpart to this entry point: it exists
 * for hosts that reserve the whole device heap for their own pool, that must
 * not allocate inside a latency-critical loop, or whose device memory belongs
 * to another framework's allocator.  It allocates nothing (no cudaMalloc,
 * cudaFree or allocating library call); all inputs and outputs are caller
 * device memory:
 *   n            rows of the square CSR matrices A and M (device arrays,
 *                int32 row_ptr (n+1) / col (nnz), float64 values)
 *   k            columns of X; a power of two with 4 <= k <= 256, else
 *                PASM_EINVAL
 *   X            n x k row-major float64 block (one column per pair)
 *   YA, YM       n x k outputs: A X and M X
 *   beta, zeta   k outputs: beta_j = X_j^T A X_j, zeta_j = X_j^T M X_j
 *   stream       cudaStream_t (NULL = legacy default stream); the call is
 *                asynchronous on it.
 * Its only scratch -- per-block partial sums -- lives in one fixed array of
 * 156,160 doubles (about 1.25 MB) inside the library, held by every GPU that
 * loads the library until the process exits; nothing in it needs clearing,
 * since each call writes every entry it later reads.  All calls share that
 * array, so calls whose kernels may overlap on the GPU (different streams,
 * or concurrent host threads) race; serialise them.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * caches it for the life of the process; make that first call outside any
 * stream capture.  A cudaDeviceReset invalidates the cached address: do not
 * call this entry point on a device after resetting it.  Errors: PASM_EINVAL
 * (sizes or NULL pointers), PASM_ECUDA. */
int pasm_border_noalloc(int n, const int32_t* A_row_ptr, const int32_t* A_col, const double* A_val,
                        int64_t A_nnz, const int32_t* M_row_ptr, const int32_t* M_col, const double* M_val,
                        int64_t M_nnz, int k, const double* X, double* YA, double* YM, double* beta,
                        double* zeta, void* stream);

/* ---- Batches of independent problems of uneven size (several meshes, several
 * k per mesh).  Distinct problems, like the pairs of Algorithm 2, never
 * exchange data (Section 3.2, the remark after Algorithm 2 on distributing
 * eigenpairs over processes); the batch steps them together: one batch step is
 * one replay of one captured CUDA graph holding the correction step of every
 * unfinished problem on its own branch, so the small problems' kernels run
 * beside the large ones' and the host launches and waits once per batch step. */
typedef struct pasm_batch pasm_batch;

/* One context per problem p: n_levels[p] levels, A[p], M[p] arrays of
 * n_levels[p] matrices, P[p] of n_levels[p] - 1 (see pasm_setup); opts shared
 * (NULL = defaults); stream = the caller's stream the batch orders itself
 * after.  Errors as pasm_setup. */
int pasm_batch_setup(pasm_batch** out, int n_problems, const int* n_levels, const pasm_csr* const* A,
                     const pasm_csr* const* M, const pasm_csr* const* P, const pasm_opts* opts, void* stream);

/* Solve every problem p for its k[p] smallest pairs from its coarse start:
 * batch steps (one graph replay each; the graph is captured again only when a
 * problem finishes) until every pair is frozen or opts.max_steps rounds.
 * Outputs per problem (each array of pointers may be NULL; entries host or
 * device): lambda_out[p] (k[p]), U_out[p] (n_p x k[p]), steps_out[p],
 * status_out[p]; *batch_steps = rounds.  Returns PASM_ENOTCONV if any pair is
 * still active (outputs written); on every return the caller's stream is
 * ordered after all work the batch queued. */
int pasm_batch_solve(pasm_batch* b, const int* k, double tol, double* const* lambda_out, double* const* U_out,
                     int* const* steps_out, int* const* status_out, int* batch_steps);

/* Change the batch's step cap (opts.max_steps at setup); max_steps >= 0, else
 * PASM_EINVAL. */
int pasm_batch_set_max_steps(pasm_batch* b, int max_steps);

/* Number of step graphs pasm_batch_solve has captured over the batch's life
 * (one per change of the set of unfinished problems). */
int pasm_batch_captures(pasm_batch* b, int* captures);

/* Release the batch and every context in it.  NULL is a no-op. */
void pasm_batch_destroy(pasm_batch* b);

/* Release the context and all its device memory.  NULL is a no-op. */
void pasm_destroy(pasm_ctx* ctx);

/* A static string naming a pasm_status code. */
const char* pasm_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* PASM_H */
