// Double-float ("ff") arithmetic for the float64-accuracy kernels of the
// mixed-precision path.  A value is hi + lo in two float32s (about 47
// significant bits), evaluated on the float32 pipes, which GB300 runs at 64x
// its float64 rate.  Products use the exact float32 product error of an FMA,
// sums Knuth's two-sum; every rounding-sensitive operation uses the _rn
// intrinsics so that the compiler cannot contract or reorder it.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// float64 -> hi + lo from the bit fields, with no float64 instruction: hi = x
// truncated to 24 significant bits, lo = the next 23 bits (truncated), both
// with the sign of x; |x - hi - lo| < 2^-46 |x|.  |x| < 2^-126 gives 0, lo is
// dropped below |x| = 2^-80, and NaN, Inf or |x| >= 2^128 give NaN.
__device__ __forceinline__ void ff_split(double x, float& hi, float& lo) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t w1 = (uint32_t)(b >> 32), w0 = (uint32_t)b;
  const uint32_t sign = w1 & 0x80000000u;
  const int e = (int)((w1 >> 20) & 0x7FFu);
  const int ef = e - 896;  // float exponent field of x
  const uint32_t hb = sign | ((uint32_t)ef << 23) | ((w1 & 0xFFFFFu) << 3) | (w0 >> 29);
  hi = ef > 0 ? __uint_as_float(hb) : __uint_as_float(sign);
  if (ef >= 255) hi = __uint_as_float(0x7FC00000u);
  // the next 23 significand bits as an exact float integer, times 2^(e - 1069)
  const float m = __fsub_rn(__uint_as_float(0x4B000000u | ((w0 & 0x1FFFFFFFu) >> 6)), 8388608.0f);
  const int es = e - 942;
  const float s = __uint_as_float((uint32_t)(es > 0 ? (es < 255 ? es : 0) : 0) << 23);
  lo = __uint_as_float(__float_as_uint(__fmul_rn(m, s)) | sign);
}

// float32 -> float64 from the bit fields (float subnormals flush to 0).
__device__ __forceinline__ double ff_f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ef = (u >> 23) & 0xFFu;
  if (ef == 0) return __longlong_as_double((long long)((uint64_t)(u & 0x80000000u) << 32));
  const uint64_t ed = ef == 255 ? 2047ull : (uint64_t)(ef + 896);
  return __longlong_as_double(
      (long long)(((uint64_t)(u & 0x80000000u) << 32) | (ed << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

// hi + lo rounded to float64 (one float64 addition).
__device__ __forceinline__ double ff_to_double(float hi, float lo) { return __dadd_rn(ff_f2d(hi), ff_f2d(lo)); }

// (hi, lo) += (ah + al) * (xh + xl): exact product error by FMA, two-sum of
// the leading parts; the low-order cross terms and errors collect in lo.
__device__ __forceinline__ void ff_mac(float& hi, float& lo, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  float e = __fmaf_rn(ah, xh, -p);
  e = __fmaf_rn(ah, xl, e);
  e = __fmaf_rn(al, xh, e);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(t, e));
}

// ff_mac for a float32 coefficient a (no low part): one FMA fewer.
__device__ __forceinline__ void ff_mac_exact(float& hi, float& lo, float a, float xh, float xl) {
  const float p = __fmul_rn(a, xh);
  float e = __fmaf_rn(a, xh, -p);
  e = __fmaf_rn(a, xl, e);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(t, e));
}

// Renormalise so that |lo| <= ulp(hi) / 2.
__device__ __forceinline__ void ff_norm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
}

// (hi, lo) = (ah + al) * (bh + bl), renormalised.
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& hi, float& lo) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  hi = p;
  lo = e;
  ff_norm(hi, lo);
}
