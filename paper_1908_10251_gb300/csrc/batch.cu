// Batch of independent eigenproblems of uneven size (several meshes, several
// k): one context per problem, stepped together.  Problems never exchange
// data (the pairs of Algorithm 2 are independent, Section 3.2, and so are
// distinct problems).
//
// One batch step = one replay of one captured CUDA graph that holds the
// correction step of every unfinished problem, each on its own branch (the
// context's stream forked from and joined back to the capture stream), so the
// GPU runs the small problems' launches beside the large ones' and the host
// launches once and waits once per batch step, whatever the number of
// problems.  The graph is captured again only when a problem finishes (its
// branch is dropped).  Each branch ends by copying its active-pair count to
// pinned host memory, read after the step.
#include "../../include/pasm.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

extern "C" int pasm_ctx_guard_freezes(pasm_ctx* c, int* n_active);
extern "C" int pasm_ctx_enqueue_step(pasm_ctx* c);
extern "C" void* pasm_ctx_stream(pasm_ctx* c);
extern "C" int pasm_ctx_active_host(pasm_ctx* c);

struct pasm_batch {
  std::vector<pasm_ctx*> ctx;
  std::vector<cudaStream_t> streams;      // one per problem: the stream its context orders itself after
  std::vector<cudaEvent_t> fork, join;    // per problem: capture fork / join, and the final join
  std::vector<int> k, active;
  cudaStream_t caller = nullptr;
  cudaStream_t run = nullptr;             // capture and replay stream of the batch graph
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<int> in_graph;              // which problems the current graph steps
  int max_steps = 100;
  int captures = 0;
};

namespace {

void drop_graph(pasm_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->in_graph.clear();
}

// Capture one correction step of every problem with active pairs into one graph.  The large
// problems (block-vector work n_fine x k at least a quarter of the largest one's) run one after
// another in one chain, largest first: their kernels are HBM-bound and gain nothing from sharing
// the memory system, while two of them at once evict each other's rows from L2.  The small
// problems run on their own branches beside the chain, so their launch-bound steps hide under it.
int capture_step_graph(pasm_batch* b) {
  drop_graph(b);
  const int np = (int)b->ctx.size();
  std::vector<int> members;
  std::vector<double> work((size_t)np, 0.0);
  double wmax = 0.0;
  for (int p = 0; p < np; ++p) {
    if (b->active[(size_t)p] <= 0) continue;
    int64_t n = 0;
    pasm_sizes(b->ctx[(size_t)p], &n, nullptr, nullptr, nullptr);
    work[(size_t)p] = (double)n * b->k[(size_t)p];
    wmax = std::max(wmax, work[(size_t)p]);
    members.push_back(p);
  }
  std::vector<int> order = members;   // large ones first, by decreasing work
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return work[(size_t)a] > work[(size_t)c]; });
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->run, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return PASM_ECUDA;
  }
  int r = PASM_OK;
  int prev_large = -1;
  for (int p : order) {
    if (r) break;
    const bool large = work[(size_t)p] >= 0.25 * wmax;
    // the context's own stream, where its step's kernels go
    cudaStream_t s = (cudaStream_t)pasm_ctx_stream(b->ctx[(size_t)p]);
    cudaEvent_t after = b->fork[(size_t)p];
    if (cudaEventRecord(after, b->run) != cudaSuccess) { r = PASM_ECUDA; break; }
    if (cudaStreamWaitEvent(s, after, 0) != cudaSuccess) { r = PASM_ECUDA; break; }
    if (large && prev_large >= 0 && cudaStreamWaitEvent(s, b->join[(size_t)prev_large], 0) != cudaSuccess) {
      r = PASM_ECUDA;
      break;
    }
    r = pasm_ctx_enqueue_step(b->ctx[(size_t)p]);
    if (!r && cudaEventRecord(b->join[(size_t)p], s) != cudaSuccess) r = PASM_ECUDA;
    if (large) prev_large = p;
  }
  for (int p : members)
    if (!r && cudaStreamWaitEvent(b->run, b->join[(size_t)p], 0) != cudaSuccess) r = PASM_ECUDA;
  // end the capture in every case, so that no stream is left capturing
  const cudaError_t e = cudaStreamEndCapture(b->run, &g);
  if (!r && e != cudaSuccess) r = PASM_ECUDA;
  if (!r && cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) r = PASM_ECUDA;
  if (g) cudaGraphDestroy(g);
  if (r) {
    cudaGetLastError();
    b->graph = nullptr;
    return r;
  }
  b->in_graph = members;
  ++b->captures;
  return PASM_OK;
}

// Order the caller's stream after everything the batch queued (also on error paths).
void join_caller(pasm_batch* b) {
  const int np = (int)b->ctx.size();
  for (int p = 0; p < np; ++p) {
    cudaEventRecord(b->join[(size_t)p], b->streams[(size_t)p]);
    cudaStreamWaitEvent(b->caller, b->join[(size_t)p], 0);
  }
  cudaEventRecord(b->ev_end, b->run);
  cudaStreamWaitEvent(b->caller, b->ev_end, 0);
}

}  // namespace

extern "C" {

void pasm_batch_destroy(pasm_batch* b) {
  if (!b) return;
  drop_graph(b);
  for (pasm_ctx* c : b->ctx) pasm_destroy(c);
  for (cudaEvent_t e : b->fork) cudaEventDestroy(e);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->ev_start) cudaEventDestroy(b->ev_start);
  if (b->ev_end) cudaEventDestroy(b->ev_end);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  if (b->run) cudaStreamDestroy(b->run);
  delete b;
}

int pasm_batch_setup(pasm_batch** out, int n_problems, const int* n_levels, const pasm_csr* const* A,
                     const pasm_csr* const* M, const pasm_csr* const* P, const pasm_opts* opts, void* stream) {
  if (!out) return PASM_EINVAL;
  *out = nullptr;
  if (n_problems < 1 || !n_levels || !A || !M || !P) return PASM_EINVAL;
  pasm_batch* b = new (std::nothrow) pasm_batch();
  if (!b) return PASM_ENOMEM;
  b->caller = (cudaStream_t)stream;
  pasm_opts o;
  pasm_default_opts(&o);
  if (opts) o = *opts;
  b->max_steps = o.max_steps;
  if (cudaStreamCreateWithFlags(&b->run, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_end, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    pasm_batch_destroy(b);
    return PASM_ECUDA;
  }
  for (int p = 0; p < n_problems; ++p) {
    cudaStream_t s;
    cudaEvent_t ef, ej;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      pasm_batch_destroy(b);
      return PASM_ECUDA;
    }
    b->streams.push_back(s);
    if (cudaEventCreateWithFlags(&ef, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      pasm_batch_destroy(b);
      return PASM_ECUDA;
    }
    b->fork.push_back(ef);
    if (cudaEventCreateWithFlags(&ej, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      pasm_batch_destroy(b);
      return PASM_ECUDA;
    }
    b->join.push_back(ej);
    pasm_ctx* c = nullptr;
    const int r = pasm_setup(&c, n_levels[p], A[p], M[p], P[p], &o, s);
    if (r) {
      pasm_batch_destroy(b);
      return r;
    }
    b->ctx.push_back(c);
  }
  b->k.assign((size_t)n_problems, 0);
  b->active.assign((size_t)n_problems, 0);
  *out = b;
  return PASM_OK;
}

int pasm_batch_solve(pasm_batch* b, const int* k, double tol, double* const* lambda_out, double* const* U_out,
                     int* const* steps_out, int* const* status_out, int* batch_steps) {
  if (!b || !k) return PASM_EINVAL;
  const int np = (int)b->ctx.size();
  // the problems start after the caller's queued work
  if (cudaEventRecord(b->ev_start, b->caller) != cudaSuccess) return PASM_ECUDA;
  cudaStreamWaitEvent(b->run, b->ev_start, 0);
  for (int p = 0; p < np; ++p) cudaStreamWaitEvent(b->streams[(size_t)p], b->ev_start, 0);
  drop_graph(b);
  int r = PASM_OK;
  for (int p = 0; p < np && !r; ++p) {
    r = pasm_init(b->ctx[(size_t)p], k[p], tol, nullptr, nullptr);
    if (!r) {
      b->k[(size_t)p] = k[p];
      b->active[(size_t)p] = k[p];
    }
  }
  // every problem's start is ordered before the first graph replay on the run stream
  for (int p = 0; p < np && !r; ++p) {
    cudaEventRecord(b->join[(size_t)p], b->streams[(size_t)p]);
    cudaStreamWaitEvent(b->run, b->join[(size_t)p], 0);
  }
  int it = 0, left = np;
  for (; !r && it < b->max_steps && left > 0; ++it) {
    // capture again only when the set of unfinished problems has changed
    bool same = b->graph != nullptr;
    if (same) {
      std::vector<int> want;
      for (int p = 0; p < np; ++p)
        if (b->active[(size_t)p] > 0) want.push_back(p);
      same = want == b->in_graph;
    }
    if (!same) r = capture_step_graph(b);
    if (r) break;
    if (cudaGraphLaunch(b->graph, b->run) != cudaSuccess || cudaStreamSynchronize(b->run) != cudaSuccess) {
      cudaGetLastError();
      r = PASM_ECUDA;
      break;
    }
    left = 0;
    for (int p : b->in_graph) {
      int act = pasm_ctx_active_host(b->ctx[(size_t)p]);
      if (act < b->active[(size_t)p]) r = pasm_ctx_guard_freezes(b->ctx[(size_t)p], &act);
      if (r) break;
      b->active[(size_t)p] = act;
    }
    for (int p = 0; p < np; ++p) left += b->active[(size_t)p] > 0;
  }
  if (batch_steps) *batch_steps = it;
  int notconv = 0;
  for (int p = 0; p < np && !r; ++p) {
    r = pasm_get(b->ctx[(size_t)p], lambda_out ? lambda_out[p] : nullptr, U_out ? U_out[p] : nullptr,
                 steps_out ? steps_out[p] : nullptr, status_out ? status_out[p] : nullptr);
    notconv |= b->active[(size_t)p] > 0;
  }
  join_caller(b);
  if (r) return r;
  return notconv ? PASM_ENOTCONV : PASM_OK;
}

int pasm_batch_set_max_steps(pasm_batch* b, int max_steps) {
  if (!b || max_steps < 0) return PASM_EINVAL;
  b->max_steps = max_steps;
  return PASM_OK;
}

int pasm_batch_captures(pasm_batch* b, int* captures) {
  if (!b || !captures) return PASM_EINVAL;
  *captures = b->captures;
  return PASM_OK;
}

}  // extern "C"
