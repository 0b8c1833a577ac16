// FPX storage codec (Sec. V: byte-aligned custom floating-point formats FPX, X in {56, 48, 40, 32,
// 24, 16} bits = sign + the 8-bit exponent of FP32 (bias 127) + X - 9 significand bits, written
// with IEEE-754 rounding so that FP32 is one of them bit for bit; Sec. III: a value cutoff below
// which magnitudes are stored as zero).
//
// Rounding is to nearest, ties to even, from the FP64 value; results beyond the largest finite
// value become +-inf, values below 2^-126 become FP32-style subnormals (exponent field 0, value
// q 2^(-126-m)); NaN is stored as the quiet NaN code, infinities stay infinite, a result that
// rounds to zero keeps its sign, and the cutoff gives +0.  A stream of n values is the
// concatenation of their X/8-byte little-endian codes.
//
// Kernels: one thread per group of 8 values -- it reads 8 consecutive reals (64 bytes of FP64)
// and writes the group's X bytes as X/8 aligned 64-bit words (the codes of the group laid end to
// end), so both sides are contiguous across a warp.  The plan uses the same kernels on its own
// sweep types (FP64, FP32 and df32 values, converted exactly to FP64 first) to keep the
// left-connected blocks compressed between the forward and the backward sweeps.
#include <type_traits>

#include "../../include/qtx_kernels.h"
#include "df32.cuh"
#include "kernels.cuh"

namespace qtx {
namespace {

template <int BITS>
__device__ __forceinline__ uint64_t fpx_encode(double x, double cutoff) {
  constexpr int m = BITS - 9;
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint64_t s = u >> 63;
  const int e = (int)((u >> 52) & 0x7FF);
  const uint64_t f = u & ((1ull << 52) - 1);
  if (e == 0x7FF) {  // infinity or NaN
    if (f) return (0xFFull << m) | (1ull << (m - 1));
    return (s << (BITS - 1)) | (0xFFull << m);
  }
  if (fabs(x) < cutoff) return 0;
  if (e == 0) return s << (BITS - 1);  // FP64 zero or subnormal: far below the smallest FPX value
  const int E = e - 1023 + 127;       // FPX biased exponent of the value
  const uint64_t F = (1ull << 52) | f;
  // q = F >> sh rounded to nearest even; sh = 52 - m for normal results, more for subnormal ones
  const int sh = E >= 1 ? 52 - m : 53 - m - E;
  uint64_t q;
  if (sh >= 64) {
    q = 0;
  } else {
    q = F >> sh;
    const uint64_t rem = F & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  // normal: q in [2^m, 2^(m+1)]; field = (E << m) + (q - 2^m) carries into the exponent on
  // round-up.  subnormal: field = q (q = 2^m becomes the smallest normal by itself).
  uint64_t field = E >= 1 ? ((uint64_t)E << m) + (q - (1ull << m)) : q;
  if (field >= (0xFFull << m)) field = 0xFFull << m;  // overflow to infinity
  return (s << (BITS - 1)) | field;
}

template <int BITS>
__device__ __forceinline__ double fpx_decode(uint64_t c) {
  constexpr int m = BITS - 9;
  const uint64_t s = (c >> (BITS - 1)) & 1ull;
  const int ef = (int)((c >> m) & 0xFF);
  const uint64_t q = c & ((1ull << m) - 1);
  uint64_t u;
  if (ef == 0xFF) {
    u = (s << 63) | (0x7FFull << 52) | (q ? (1ull << 51) : 0ull);
  } else if (ef == 0) {
    // q 2^(-126 - m): exact in FP64 (q < 2^47, no FP64 underflow)
    const double v = (double)q * __longlong_as_double((long long)((uint64_t)(1023 - 126 - m) << 52));
    u = (uint64_t)__double_as_longlong(v) | (s << 63);
  } else {
    u = (s << 63) | ((uint64_t)(ef - 127 + 1023) << 52) | (q << (52 - m));
  }
  return __longlong_as_double((long long)u);
}

// real value k of an FP64 array, or of an array of T-typed complex numbers viewed as 2n reals
__device__ __forceinline__ double real_at(const double* x, long k) { return x[k]; }
__device__ __forceinline__ void set_real(double* x, long k, double v) { x[k] = v; }
template <typename T>
__device__ __forceinline__ double real_at(const cx<T>* x, long k) {
  const T v = (k & 1) ? x[k >> 1].im : x[k >> 1].re;
  if constexpr (std::is_same<T, df>::value) return (double)v.hi + (double)v.lo;  // exact: |lo| <= ulp(hi)/2
  else return (double)v;
}
template <typename T>
__device__ __forceinline__ void set_real(cx<T>* x, long k, double v) {
  T t;
  if constexpr (std::is_same<T, df>::value) {
    const float hi = __double2float_rn(v);
    t = mkdf(hi, __double2float_rn(v - (double)hi));
  } else {
    t = (T)v;
  }
  if (k & 1) x[k >> 1].im = t;
  else x[k >> 1].re = t;
}

template <int BITS, typename P>
__global__ void __launch_bounds__(256) k_fpx_compress(const P* x, long n, double cutoff, uint64_t* out) {
  constexpr int W = BITS / 8;  // 64-bit words per group of 8 codes
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g * 8 >= n) return;
  uint64_t w[W];
#pragma unroll
  for (int i = 0; i < W; ++i) w[i] = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const long k = g * 8 + j;
    const uint64_t c = k < n ? fpx_encode<BITS>(real_at(x, k), cutoff) : 0ull;
    const int bit = j * BITS, wi = bit / 64, off = bit % 64;
    w[wi] |= c << off;
    if (off + BITS > 64) w[wi + 1] |= c >> (64 - off);
  }
#pragma unroll
  for (int i = 0; i < W; ++i) out[g * W + i] = w[i];
}

template <int BITS, typename P>
__global__ void __launch_bounds__(256) k_fpx_decompress(const uint64_t* in, long n, P* x) {
  constexpr int W = BITS / 8;
  constexpr uint64_t MASK = (1ull << BITS) - 1;
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g * 8 >= n) return;
  uint64_t w[W];
#pragma unroll
  for (int i = 0; i < W; ++i) w[i] = in[g * W + i];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const long k = g * 8 + j;
    if (k >= n) break;
    const int bit = j * BITS, wi = bit / 64, off = bit % 64;
    uint64_t c = w[wi] >> off;
    if (off + BITS > 64) c |= w[wi + 1] << (64 - off);
    set_real(x, k, fpx_decode<BITS>(c & MASK));
  }
}

template <typename P>
cudaError_t launch_compress(int bits, const P* x, long n, double cutoff, void* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long groups = (n + 7) / 8;
  const unsigned blocks = (unsigned)((groups + 255) / 256);
  uint64_t* o = reinterpret_cast<uint64_t*>(out);
  switch (bits) {
    case 56: k_fpx_compress<56, P><<<blocks, 256, 0, st>>>(x, n, cutoff, o); break;
    case 48: k_fpx_compress<48, P><<<blocks, 256, 0, st>>>(x, n, cutoff, o); break;
    case 40: k_fpx_compress<40, P><<<blocks, 256, 0, st>>>(x, n, cutoff, o); break;
    case 32: k_fpx_compress<32, P><<<blocks, 256, 0, st>>>(x, n, cutoff, o); break;
    case 24: k_fpx_compress<24, P><<<blocks, 256, 0, st>>>(x, n, cutoff, o); break;
    case 16: k_fpx_compress<16, P><<<blocks, 256, 0, st>>>(x, n, cutoff, o); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

template <typename P>
cudaError_t launch_decompress(int bits, const void* in, long n, P* x, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long groups = (n + 7) / 8;
  const unsigned blocks = (unsigned)((groups + 255) / 256);
  const uint64_t* i = reinterpret_cast<const uint64_t*>(in);
  switch (bits) {
    case 56: k_fpx_decompress<56, P><<<blocks, 256, 0, st>>>(i, n, x); break;
    case 48: k_fpx_decompress<48, P><<<blocks, 256, 0, st>>>(i, n, x); break;
    case 40: k_fpx_decompress<40, P><<<blocks, 256, 0, st>>>(i, n, x); break;
    case 32: k_fpx_decompress<32, P><<<blocks, 256, 0, st>>>(i, n, x); break;
    case 24: k_fpx_decompress<24, P><<<blocks, 256, 0, st>>>(i, n, x); break;
    case 16: k_fpx_decompress<16, P><<<blocks, 256, 0, st>>>(i, n, x); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace

bool fpx_width_ok(int bits) {
  return bits == 56 || bits == 48 || bits == 40 || bits == 32 || bits == 24 || bits == 16;
}
size_t fpx_bytes(int bits, long n_reals) { return n_reals <= 0 ? 0 : (size_t)((n_reals + 7) / 8) * (size_t)bits; }

template <typename T>
cudaError_t fpx_store(int bits, const cx<T>* x, long n_complex, void* out, cudaStream_t st) {
  return launch_compress<cx<T>>(bits, x, 2 * n_complex, 0.0, out, st);
}
template <typename T>
cudaError_t fpx_load(int bits, const void* in, long n_complex, cx<T>* x, cudaStream_t st) {
  return launch_decompress<cx<T>>(bits, in, 2 * n_complex, x, st);
}
template cudaError_t fpx_store<double>(int, const cx<double>*, long, void*, cudaStream_t);
template cudaError_t fpx_store<float>(int, const cx<float>*, long, void*, cudaStream_t);
template cudaError_t fpx_store<df>(int, const cx<df>*, long, void*, cudaStream_t);
template cudaError_t fpx_load<double>(int, const void*, long, cx<double>*, cudaStream_t);
template cudaError_t fpx_load<float>(int, const void*, long, cx<float>*, cudaStream_t);
template cudaError_t fpx_load<df>(int, const void*, long, cx<df>*, cudaStream_t);

}  // namespace qtx

using namespace qtx;

extern "C" {

size_t qtx_fpx_bytes(int bits, long n) { return fpx_width_ok(bits) ? fpx_bytes(bits, n) : 0; }

qtx_status qtx_fpx_compress(int bits, const double* x, long n, double cutoff, void* out, void* stream) {
  if (!fpx_width_ok(bits) || n < 0 || !(cutoff >= 0.0)) return QTX_ERR_INVALID_ARG;
  if (n == 0) return QTX_OK;
  if (!x || !out || (reinterpret_cast<uintptr_t>(x) & 7) || (reinterpret_cast<uintptr_t>(out) & 7))
    return QTX_ERR_INVALID_ARG;
  const cudaError_t e = launch_compress<double>(bits, x, n, cutoff, out, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? QTX_OK : QTX_ERR_CUDA;
}

qtx_status qtx_fpx_decompress(int bits, const void* in, long n, double* x, void* stream) {
  if (!fpx_width_ok(bits) || n < 0) return QTX_ERR_INVALID_ARG;
  if (n == 0) return QTX_OK;
  if (!x || !in || (reinterpret_cast<uintptr_t>(x) & 7) || (reinterpret_cast<uintptr_t>(in) & 7))
    return QTX_ERR_INVALID_ARG;
  const cudaError_t e = launch_decompress<double>(bits, in, n, x, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? QTX_OK : QTX_ERR_CUDA;
}

}  // extern "C"
