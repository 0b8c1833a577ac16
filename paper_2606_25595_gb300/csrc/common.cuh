// Shared device helpers for the RGF library: complex arithmetic on (re, im) pairs and the
// batched-operation descriptors the host orchestration passes to the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qtx_rgf.h"

namespace qtx {

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> mk(T r, T i) {
  cx<T> z;
  z.re = r;
  z.im = i;
  return z;
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk(s * a.re, s * a.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> conj(cx<T> a) { return mk(a.re, -a.im); }
// acc += a * b  (four real FMAs)
template <typename T>
__device__ __forceinline__ void cfma(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// 1/a, scaled to avoid overflow (Smith's algorithm).
template <typename T>
__device__ __forceinline__ cx<T> crecip(cx<T> a) {
  T ar = a.re, ai = a.im;
  if (fabs(ar) >= fabs(ai)) {
    T r = ai / ar, d = ar + ai * r;
    return mk(T(1) / d, -r / d);
  } else {
    T r = ar / ai, d = ai + ar * r;
    return mk(r / d, T(-1) / d);
  }
}
template <typename T>
__device__ __forceinline__ T cabs1(cx<T> a) { return fabs(a.re) + fabs(a.im); }

// "df32" real: the unevaluated sum hi + lo of two FP32 values (|lo| <= ulp(hi)/2); arithmetic in df32.cuh.
struct df {
  float hi, lo;
};

// Conversions between FP64 and df32 (at the boundary of the sweep and in the observable
// reductions).  On the device they are done with integer operations -- GB300's FP64 pipe runs at
// 1/64 of the FP32 rate, and these conversions sit in HBM-bound kernels -- and give the same bits
// as the FP64 formulas (hi = RN(x), lo = RN(x - hi); x = RN(hi + lo)); values outside
// 2^-74 <= |x| < 2^127 (and subnormal or special df parts) take the FP64 formulas.
__host__ __device__ __forceinline__ df df_split_fp64(double x) {
  df r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
__host__ __device__ __forceinline__ double df_sum_fp64(df a) { return (double)a.hi + (double)a.lo; }
// The FP64 formulas for the rare operands the integer paths leave to them, kept out of line: inlined,
// the compiler may if-convert them, and then every element issues their FP64 instructions (1/64 rate).
static __device__ __noinline__ df df_split_fp64_rare(double x) { return df_split_fp64(x); }
static __device__ __noinline__ double df_sum_fp64_rare(df a) { return df_sum_fp64(a); }

__device__ __forceinline__ df df_split_int(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF) - 1023;  // x = +-M 2^(e-52), M in [2^52, 2^53)
  if ((u << 1) == 0ull) return df{__uint_as_float((unsigned)(u >> 32)), 0.f};  // +-0: (+-0, +0)
  if (e < -74 || e > 126) return df_split_fp64_rare(x);
  const unsigned long long M = (u & ((1ull << 52) - 1)) | (1ull << 52);
  unsigned long long q = M >> 29;  // hi's 24-bit significand, rounded to nearest even
  const unsigned long long rem = M & ((1ull << 29) - 1);
  if (rem > (1ull << 28) || (rem == (1ull << 28) && (q & 1ull))) ++q;
  const int R = (int)((long long)M - (long long)(q << 29));  // x - hi in units of 2^(e-52), |R| <= 2^28
  int eh = e;
  if (q == (1ull << 24)) {  // rounded up to the next power of two
    q >>= 1;
    ++eh;
  }
  const unsigned sgn = (unsigned)(u >> 63);
  df r;
  r.hi = __uint_as_float((sgn << 31) | ((unsigned)(eh + 127) << 23) | ((unsigned)q & 0x7FFFFFu));
  // lo = RN(R 2^(e-52)): the one rounding happens in the integer-to-float conversion; the scalings
  // by 2^-52 and 2^e are exact (|lo| >= 2^(e-52) >= 2^-126)
  const float lo = __int2float_rn(R) * __uint_as_float((unsigned)(127 - 52) << 23) *
                   __uint_as_float((unsigned)(e + 127) << 23);
  r.lo = R == 0 ? 0.f : (sgn ? -lo : lo);
  return r;
}

// RN(hi + lo) of a df32 pair: the significands aligned on lo's unit, T = Mh 2^d +- Ml (d = exponent
// gap), rounded to 53 bits, ties to even.  For d > 39, T is scaled down by 2^(d-39) first with an
// arithmetic (flooring) shift, and the bits shifted out only act as a sticky bit.  Pairs with
// d < 23 (|lo| > ulp(hi)), subnormal or special parts take the FP64 formula.
__device__ __forceinline__ double df_sum_int(df a) {
  const unsigned uh = __float_as_uint(a.hi), ul = __float_as_uint(a.lo);
  const int fh = (int)((uh >> 23) & 0xFF), fl = (int)((ul >> 23) & 0xFF);
  if (((uh | ul) << 1) == 0u)  // both parts +-0: RN(hi + lo) is -0 only if both are
    return __longlong_as_double((long long)((unsigned long long)(uh & ul & 0x80000000u) << 32));
  if (fh == 0 || fh == 0xFF || fl == 0xFF || (fl == 0 && (ul & 0x7FFFFFu))) return df_sum_fp64_rare(a);
  const unsigned long long sh = uh >> 31;
  const unsigned long long hi_mant = (unsigned long long)(uh & 0x7FFFFFu) << 29;
  if (fl == 0)  // lo = +-0: hi itself
    return __longlong_as_double((long long)((sh << 63) | ((unsigned long long)(fh - 127 + 1023) << 52) | hi_mant));
  const int d = fh - fl;
  if (d < 23 || d > 100) return df_sum_fp64_rare(a);
  const long long Mh = (long long)((uh & 0x7FFFFFu) | 0x800000u);
  const long long Ml = (long long)((ul & 0x7FFFFFu) | 0x800000u);
  const long long sMl = (ul >> 31) == sh ? Ml : -Ml;
  const int k = d > 39 ? d - 39 : 0;
  const long long S = (Mh << (d - k)) + (k < 63 ? (sMl >> k) : (sMl < 0 ? -1 : 0));
  const bool sticky = k > 0 && (k >= 63 || (sMl & ((1ll << k) - 1)) != 0);
  const int len = 64 - __clzll(S);  // S > 2^45: the hi term dominates
  int E = fl - 150 + k + len - 1;   // unbiased exponent of the result
  unsigned long long m;
  if (len <= 53) {                  // exact (k = 0 here: for k > 0, len >= 62)
    m = (unsigned long long)S << (53 - len);
  } else {
    const int sft = len - 53;
    m = (unsigned long long)S >> sft;
    const unsigned long long r = (unsigned long long)S & ((1ull << sft) - 1), half = 1ull << (sft - 1);
    if (r > half || (r == half && (sticky || (m & 1ull)))) ++m;
    if (m == (1ull << 53)) {
      m >>= 1;
      ++E;
    }
  }
  return __longlong_as_double((long long)((sh << 63) | ((unsigned long long)(E + 1023) << 52) | (m & ((1ull << 52) - 1))));
}

__host__ __device__ __forceinline__ double to_d(float x) { return (double)x; }
__host__ __device__ __forceinline__ double to_d(double x) { return x; }
__host__ __device__ __forceinline__ double to_d(df x) {
#ifdef __CUDA_ARCH__
  return df_sum_int(x);
#else
  return df_sum_fp64(x);
#endif
}
template <typename T>
__host__ __device__ __forceinline__ T from_d(double x);
template <>
__host__ __device__ __forceinline__ float from_d<float>(double x) { return (float)x; }
template <>
__host__ __device__ __forceinline__ double from_d<double>(double x) { return x; }
template <>
__host__ __device__ __forceinline__ df from_d<df>(double x) {
#ifdef __CUDA_ARCH__
  return df_split_int(x);
#else
  return df_split_fp64(x);
#endif
}

template <typename To, typename Ti>
__host__ __device__ __forceinline__ cx<To> cvt(cx<Ti> a) {
  cx<To> z;
  z.re = from_d<To>(to_d(a.re));
  z.im = from_d<To>(to_d(a.im));
  return z;
}

// Operation applied to a GEMM operand: as stored, or conjugate-transposed.
enum Op : int { OP_N = 0, OP_C = 1 };

// One batched GEMM  C[e] = alpha * op(A[e]) * op(B[e]) + beta * C0[e]  (e = batch index).
// Strides are in complex elements; a zero batch stride shares one matrix across the batch.
// `active` (optional) skips batch entries whose flag is 0.
template <typename T>
struct GemmArgs {
  int M, N, K;
  const cx<T>* A; long lda, sA; int opA;
  const cx<T>* B; long ldb, sB; int opB;
  const cx<T>* C0; long ldc0, sC0;
  cx<T>* C; long ldc, sC;
  double alpha, beta;
  int batch;
  const int* active;
};

// A digitised operand kept across products (digit planes and scale exponents in caller-owned
// memory of gemm_tc_operand_bytes): mode 1 digitises the operand into it, mode 2 uses the planes
// already there (the operand, its op and shape unchanged since the mode-1 product).
struct TcOperand {
  unsigned char* planes = nullptr;
  int* expo = nullptr;
  int mode = 0;
};

// Arguments of the tensor-core engine (complex df32 operands and result).
struct TcArgs {
  int M, N, K;
  const cx<df>* A; long lda, sA; int opA;
  const cx<df>* B; long ldb, sB; int opB;
  const cx<df>* C0; long ldc0, sC0;
  cx<df>* C; long ldc, sC;
  double alpha, beta;          // applied in df32 (split into hi + lo FP32 parts by the launcher)
  int batch;
  const int* active;
  TcOperand* opndA = nullptr;  // optional kept / reused digit planes of op(A), op(B)
  TcOperand* opndB = nullptr;
  bool f32 = false;            // A, B, C0, C point to cx<float> arrays (four digit planes only)
  int stages = 0;              // schedule: pipeline stages of the product kernel (0 = the variant's
                               // default; only sizes its shared memory allows are taken)
  int ctas = 0;                // schedule: persistent CTAs per launch (0 = one per SM)
};

}  // namespace qtx
