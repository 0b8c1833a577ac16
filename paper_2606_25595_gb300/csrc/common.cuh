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

// Conversions through FP64 (used at the boundary of the sweep and in the observable reductions).
__host__ __device__ __forceinline__ double to_d(float x) { return (double)x; }
__host__ __device__ __forceinline__ double to_d(double x) { return x; }
__host__ __device__ __forceinline__ double to_d(df x) { return (double)x.hi + (double)x.lo; }
template <typename T>
__host__ __device__ __forceinline__ T from_d(double x);
template <>
__host__ __device__ __forceinline__ float from_d<float>(double x) { return (float)x; }
template <>
__host__ __device__ __forceinline__ double from_d<double>(double x) { return x; }
template <>
__host__ __device__ __forceinline__ df from_d<df>(double x) {
  df r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
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

// Arguments of the tensor-core engine (complex df32 operands and result).
struct TcArgs {
  int M, N, K;
  const cx<df>* A; long lda, sA; int opA;
  const cx<df>* B; long ldb, sB; int opB;
  const cx<df>* C0; long ldc0, sC0;
  cx<df>* C; long ldc, sC;
  float alpha, beta;
  int batch;
  const int* active;
};

}  // namespace qtx
