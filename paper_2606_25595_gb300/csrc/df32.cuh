// "df32": a real number stored as the unevaluated sum hi + lo of two FP32 values with
// |lo| <= ulp(hi)/2 (about 48 significand bits, FP32's 8-bit exponent).  The emulated-FP64 sweep keeps
// every intermediate block in this form: GB300's FP64 pipe runs at ~1/64 of its FP32 rate, so
// elementwise work and GEMM epilogues in FP64 would cost more than the tensor-core products
// themselves.  The exponent range suffices: the paper's storage study (Sec. III-A) finds all NEGF
// data within [1e-39, 1e3], the FP32 range.
//
// Arithmetic: error-free transformations (Knuth's TwoSum, FMA-based TwoProd), renormalised to a
// (hi, lo) pair after each operation.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace qtx {

__host__ __device__ __forceinline__ df mkdf(float h, float l) {
  df r;
  r.hi = h;
  r.lo = l;
  return r;
}

__device__ __forceinline__ df df_add(df a, df b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  float e = (a.hi - (s - v)) + (b.hi - v);
  e += a.lo + b.lo;
  const float h = s + e;
  return mkdf(h, e - (h - s));
}
__device__ __forceinline__ df df_neg(df a) { return mkdf(-a.hi, -a.lo); }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
// a * f for an FP32 factor f
__device__ __forceinline__ df df_mulf(df a, float f) {
  const float p = a.hi * f;
  float e = fmaf(a.hi, f, -p);
  e = fmaf(a.lo, f, e);
  const float h = p + e;
  return mkdf(h, e - (h - p));
}
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float h = p + e;
  return mkdf(h, e - (h - p));
}
// Conversions to/from FP64 (these use the FP64 pipe; only at the boundary of the sweep).
__device__ __forceinline__ df df_from_double(double x) {
  const float h = (float)x;
  return mkdf(h, (float)(x - (double)h));
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// x * 2^E exactly (unless the result leaves the FP32 range), for |E| <= 250.
__device__ __forceinline__ float scale2(float x, int E) {
  E = E < -250 ? -250 : (E > 250 ? 250 : E);
  const int E1 = E / 2, E2 = E - E1;
  return x * __int_as_float((E1 + 127) << 23) * __int_as_float((E2 + 127) << 23);
}

// round(f * 2^sh) as a 64-bit integer (ties away from zero); zero and subnormal f give 0.
// Requires |f| * 2^sh < 2^62.
__device__ __forceinline__ long long f2fix(float f, int sh) {
  const uint32_t u = __float_as_uint(f);
  const int ex = (int)((u >> 23) & 0xFFu);
  if (ex == 0) return 0;
  const long long m = (long long)((u & 0x7FFFFFu) | 0x800000u);
  const int s = ex - 150 + sh;
  long long r;
  if (s >= 0) r = m << (s > 38 ? 38 : s);
  else if (s < -25) r = 0;
  else r = (m + (1LL << (-s - 1))) >> (-s);
  return (u >> 31) ? -r : r;
}

// Exponent e with |x| < 2^e for x = hi + lo (from hi alone; 0 => -1000).
__device__ __forceinline__ int df_expo(float hi) {
  const uint32_t ex = (__float_as_uint(hi) >> 23) & 0xFFu;
  return ex == 0 ? -1000 : (int)ex - 126;
}

}  // namespace qtx
