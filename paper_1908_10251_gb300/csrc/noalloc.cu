// Bordering products without any device allocation.
//
// Some callers cannot call cudaMalloc: applications that reserve the whole
// device heap up front for their own pool or arena, code that must not
// allocate inside a latency-critical loop (allocation can synchronise the
// device and fragment memory), and hosts whose device memory is owned by
// another framework's caching allocator.  For them this file offers the
// bordering kernel of the correction step with its only scratch buffer -- the
// per-block partial sums of beta = u~^T A u~ and zeta = u~^T M u~ -- placed in
// a fixed-size device array that is part of the library image, so the call
// allocates nothing.  The caller passes every input and output.
#include "../../include/pasm.h"
#include "kernels.cuh"

#include <cuda_runtime.h>

#include <mutex>

namespace {

// Capacity of the shared scratch in doubles: 1216 blocks x 2 sums x 64 pairs,
// plus room for the 2 x 256 reduced sums.  About 1.25 MB per device.
constexpr int kScratchDoubles = 1216 * 2 * 64 + 2 * 256;
constexpr int kMaxPairs = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_border_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_border_scratch on the current device, looked up once per
// device.  The host-side name of the array is only a stand-in, never a device
// address, so it is never passed to a kernel.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return PASM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_border_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return PASM_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return PASM_OK;
}

}  // namespace

extern "C" int pasm_border_noalloc(int n, const int32_t* A_row_ptr, const int32_t* A_col, const double* A_val,
                                   int64_t A_nnz, const int32_t* M_row_ptr, const int32_t* M_col,
                                   const double* M_val, int64_t M_nnz, int k, const double* X, double* YA,
                                   double* YM, double* beta, double* zeta, void* stream) {
  using namespace pasm;
  if (n < 1 || k < 4 || k > kMaxPairs || (k & (k - 1)) != 0) return PASM_EINVAL;
  if (!A_row_ptr || !A_col || !A_val || !M_row_ptr || !M_col || !M_val || !X || !YA || !YM || !beta || !zeta)
    return PASM_EINVAL;
  if (A_nnz < 0 || M_nnz < 0 || A_nnz > 2147483647LL || M_nnz > 2147483647LL) return PASM_EINVAL;
  double* scratch = nullptr;
  int r = scratch_address(&scratch);
  if (r) return r;
  // per-block partial sums take 2 k doubles per block; the reduced sums follow them
  const int max_blocks = (kScratchDoubles - 2 * kMaxPairs) / (2 * k);
  DCsr A, M;
  A.n_rows = A.n_cols = n; A.nnz = A_nnz;
  A.rp = const_cast<int*>(A_row_ptr); A.ci = const_cast<int*>(A_col); A.v64 = const_cast<double*>(A_val);
  M.n_rows = M.n_cols = n; M.nnz = M_nnz;
  M.rp = const_cast<int*>(M_row_ptr); M.ci = const_cast<int*>(M_col); M.v64 = const_cast<double*>(M_val);
  Launch L;
  L.s = static_cast<cudaStream_t>(stream);
  // every scratch entry read below is written earlier in the same call, so no part of it needs clearing
  const int nblk = border_products(L, A, M, X, YA, YM, scratch, k, max_blocks);
  double* sums = scratch + (size_t)nblk * 2 * k;
  column_sums(L, scratch, nblk, 2, k, sums);
  if (cudaMemcpyAsync(beta, sums, sizeof(double) * k, cudaMemcpyDeviceToDevice, L.s) != cudaSuccess ||
      cudaMemcpyAsync(zeta, sums + k, sizeof(double) * k, cudaMemcpyDeviceToDevice, L.s) != cudaSuccess) {
    cudaGetLastError();
    return PASM_ECUDA;
  }
  if (cudaGetLastError() != cudaSuccess) return PASM_ECUDA;
  return PASM_OK;
}
