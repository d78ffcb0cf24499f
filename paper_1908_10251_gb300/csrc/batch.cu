// Batch of independent eigenproblems of uneven size (several meshes, several
// k): one context per problem, each with its own stream, stepped together so
// that the correction steps of small problems overlap on the GPU.  Problems
// never exchange data (the pairs of Algorithm 2 are independent, Section 3.2,
// and so are distinct problems).
#include "../../include/pasm.h"

#include <cuda_runtime.h>

#include <new>
#include <vector>

extern "C" int pasm_ctx_wait_active(pasm_ctx* c, int* n_active);
extern "C" int pasm_ctx_guard_freezes(pasm_ctx* c, int* n_active);

struct pasm_batch {
  std::vector<pasm_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<int> k, active;
  cudaStream_t caller = nullptr;
  int max_steps = 100;
};

extern "C" {

void pasm_batch_destroy(pasm_batch* b) {
  if (!b) return;
  for (pasm_ctx* c : b->ctx) pasm_destroy(c);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
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
  for (int p = 0; p < n_problems; ++p) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      pasm_batch_destroy(b);
      return PASM_ECUDA;
    }
    b->streams.push_back(s);
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      pasm_batch_destroy(b);
      return PASM_ECUDA;
    }
    b->events.push_back(e);
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
  cudaEvent_t start;
  if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) return PASM_ECUDA;
  cudaEventRecord(start, b->caller);
  for (int p = 0; p < np; ++p) cudaStreamWaitEvent(b->streams[(size_t)p], start, 0);
  cudaEventDestroy(start);
  for (int p = 0; p < np; ++p) {
    const int r = pasm_init(b->ctx[(size_t)p], k[p], tol, nullptr, nullptr);
    if (r) return r;
    b->k[(size_t)p] = k[p];
    b->active[(size_t)p] = k[p];
  }
  int it = 0, left = np;
  for (; it < b->max_steps && left > 0; ++it) {
    // launch one correction step of every unfinished problem, each on its own stream
    for (int p = 0; p < np; ++p)
      if (b->active[(size_t)p] > 0) {
        const int r = pasm_step(b->ctx[(size_t)p], nullptr);
        if (r) return r;
      }
    left = 0;
    for (int p = 0; p < np; ++p)
      if (b->active[(size_t)p] > 0) {
        int act = 0;
        int r = pasm_ctx_wait_active(b->ctx[(size_t)p], &act);
        if (!r && act < b->active[(size_t)p]) r = pasm_ctx_guard_freezes(b->ctx[(size_t)p], &act);
        if (r) return r;
        b->active[(size_t)p] = act;
        left += act > 0;
      }
  }
  if (batch_steps) *batch_steps = it;
  int notconv = 0;
  for (int p = 0; p < np; ++p) {
    const int r = pasm_get(b->ctx[(size_t)p], lambda_out ? lambda_out[p] : nullptr, U_out ? U_out[p] : nullptr,
                           steps_out ? steps_out[p] : nullptr, status_out ? status_out[p] : nullptr);
    if (r) return r;
    notconv |= b->active[(size_t)p] > 0;
    cudaEventRecord(b->events[(size_t)p], b->streams[(size_t)p]);
    cudaStreamWaitEvent(b->caller, b->events[(size_t)p], 0);
  }
  return notconv ? PASM_ENOTCONV : PASM_OK;
}

}  // extern "C"
