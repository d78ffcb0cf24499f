// Shared device helpers of the PASM library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PASM_WARP 32

// 16-byte vector of T: 2 doubles or 4 floats.
template <typename T> struct Vec16;
template <> struct Vec16<double> {
  static constexpr int N = 2;
  using type = double2;
  __device__ __forceinline__ static void load(const double* p, double* v) {
    double2 t = *reinterpret_cast<const double2*>(p); v[0] = t.x; v[1] = t.y;
  }
  __device__ __forceinline__ static void store(double* p, const double* v) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};
template <> struct Vec16<float> {
  static constexpr int N = 4;
  using type = float4;
  __device__ __forceinline__ static void load(const float* p, float* v) {
    float4 t = *reinterpret_cast<const float4*>(p); v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  __device__ __forceinline__ static void store(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

// Read-only streaming load of a 16-byte vector through the non-coherent path.
template <typename T>
__device__ __forceinline__ void ldg16(const T* p, T* v);
template <>
__device__ __forceinline__ void ldg16<double>(const double* p, double* v) {
  double2 t = __ldg(reinterpret_cast<const double2*>(p)); v[0] = t.x; v[1] = t.y;
}
template <>
__device__ __forceinline__ void ldg16<float>(const float* p, float* v) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p)); v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block layout of a block-vector kernel: a "row group" of TPR threads owns one
// row; each thread owns CH chunks of VEC consecutive columns, chunk c of lane t
// covering columns (c * TPR + t) * VEC ... + VEC - 1.  ldk = TPR * VEC * CH.
struct RowMap {
  int tpr;   // threads per row (power of two, <= 32)
  int rpb;   // rows per block
};

// Allow `func` up to `need` bytes of dynamic shared memory on the current
// device.  The limit is set to the device's opt-in maximum less the kernel's
// static shared memory, so it never drops below what an earlier context of a
// larger size needs; fails with cudaErrorInvalidValue if `need` exceeds it.
inline cudaError_t allow_dynamic_smem(const void* func, size_t need) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  const size_t cap = (size_t)optin - fa.sharedSizeBytes;
  if (need > cap) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
}
