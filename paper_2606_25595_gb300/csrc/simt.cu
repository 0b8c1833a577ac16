// SIMT kernels of the RGF library (sm_103a): batched complex GEMM, batched leaf inverse by
// Gauss-Jordan elimination with partial pivoting, elementwise block combinations, assembly of
// the block rows of M, and the FP64 observable reductions of Sec. II-B.
#include <cmath>
#include <type_traits>

#include "df32.cuh"
#include "kernels.cuh"

namespace qtx {

std::atomic<long long> g_launches{0};

// ============================================================================ batched GEMM
// Tile BM x BN of C per CTA, K staged through shared memory BK at a time (two buffers: the next
// stage's global loads are issued into registers before the current stage's FMAs and stored to
// the other buffer after them, one barrier per stage); each thread owns a TM x TN sub-grid
// interleaved with stride (BM/TM, BN/TN) so smem reads of a warp are contiguous.
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_gemm(GemmArgs<T> g) {
  // FP32: two stage buffers (load latency hidden behind the FMAs); FP64 is bound by the FP64 pipe,
  // where one buffer with twice the K per stage (half the barriers) is faster
  constexpr int NBUF = sizeof(T) == 4 ? 2 : 1;
  constexpr int TX = BN / TN, TY = BM / TM, NT = TX * TY;
  constexpr int LA = (BM * BK + NT - 1) / NT, LB = (BK * BN + NT - 1) / NT;  // loads per thread
  const int e = blockIdx.z;
  if (g.active && !g.active[e]) return;
  __shared__ cx<T> As[NBUF][BK][BM + 1];
  __shared__ cx<T> Bs[NBUF][BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const cx<T>* A = g.A + (long)e * g.sA;
  const cx<T>* B = g.B + (long)e * g.sB;
  cx<T> acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = mk<T>(0, 0);

  cx<T> ra[LA], rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int idx = tid + l * NT;
      int mm, kk;
      if (g.opA == OP_N) { kk = idx % BK; mm = idx / BK; }
      else { mm = idx % BM; kk = idx / BM; }
      const int m = m0 + mm, k = k0 + kk;
      cx<T> v = mk<T>(0, 0);
      if (idx < BM * BK && m < g.M && k < g.K) v = (g.opA == OP_N) ? A[(long)m * g.lda + k] : conj(A[(long)k * g.lda + m]);
      ra[l] = v;
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int idx = tid + l * NT;
      int kk, nn;
      if (g.opB == OP_N) { nn = idx % BN; kk = idx / BN; }
      else { kk = idx % BK; nn = idx / BK; }
      const int k = k0 + kk, n = n0 + nn;
      cx<T> v = mk<T>(0, 0);
      if (idx < BK * BN && k < g.K && n < g.N) v = (g.opB == OP_N) ? B[(long)k * g.ldb + n] : conj(B[(long)n * g.ldb + k]);
      rb[l] = v;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int idx = tid + l * NT;
      if (idx < BM * BK) {
        if (g.opA == OP_N) As[buf][idx % BK][idx / BK] = ra[l];
        else As[buf][idx / BM][idx % BM] = ra[l];
      }
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int idx = tid + l * NT;
      if (idx < BK * BN) {
        if (g.opB == OP_N) Bs[buf][idx / BN][idx % BN] = rb[l];
        else Bs[buf][idx % BK][idx / BK] = rb[l];
      }
    }
  };
  auto fma_stage = [&](int buf) {
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cx<T> a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + i * TY];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[buf][kk][tx + j * TX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cfma(acc[i][j], a[i], bb[j]);
    }
  };
  if constexpr (NBUF == 2) {
    load(0);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < g.K; k0 += BK) {
      const bool more = k0 + BK < g.K;
      if (more) load(k0 + BK);
      fma_stage(buf);
      if (more) store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  } else {
    for (int k0 = 0; k0 < g.K; k0 += BK) {
      load(k0);
      store(0);
      __syncthreads();
      fma_stage(0);
      __syncthreads();
    }
  }
  cx<T>* C = g.C + (long)e * g.sC;
  const cx<T>* C0 = g.C0 ? g.C0 + (long)e * g.sC0 : nullptr;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty + i * TY;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + j * TX;
      if (n >= g.N) continue;
      cx<T> r = T(g.alpha) * acc[i][j];
      if (C0 && g.beta != 0.0) r = r + T(g.beta) * C0[(long)m * g.ldc0 + n];
      C[(long)m * g.ldc + n] = r;
    }
  }
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
static cudaError_t launch_gemm(const GemmArgs<T>& g, cudaStream_t st) {
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch);
  k_gemm<T, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(g);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t gemm_simt(const GemmArgs<T>& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.M <= 32 && g.N <= 32) return launch_gemm<T, 32, 32, 16, 2, 2>(g, st);
  if constexpr (sizeof(T) == 4) {
    if (g.M >= 128 && g.N >= 128) return launch_gemm<T, 128, 128, 8, 8, 8>(g, st);
  }
  return launch_gemm<T, 64, 64, 16, 4, 4>(g, st);
}
template cudaError_t gemm_simt<double>(const GemmArgs<double>&, cudaStream_t);
template cudaError_t gemm_simt<float>(const GemmArgs<float>&, cudaStream_t);

// ============================================================================ leaf inverse
// In-place Gauss-Jordan inverse with partial pivoting (pivot = first row of largest |Re|+|Im| among
// the rows not yet used, in the current column), one CTA per block, the block held in registers.
//
// Rows are not moved: step k pivots on (p_k, k) wherever row p_k sits.  With P the permutation
// (PA)[k] = A[p_k], the in-place sweep leaves B with B[p_k] = row k of (PA)^-1 = A^-1 P^T, i.e.
//     A^-1[k][p_j] = B[p_k][j],
// so each thread scatters its values to (step of its row, pivot row of its column's step).
//
// Layout: NMAX/8 warps; warp w owns rows w + (NMAX/8) m, m = 0..7; lane l owns columns l + 32 c,
// c < NMAX/32.  Entries outside the n x n block are zero and stay zero.  Each step needs one CTA
// barrier: at the end of step k every warp publishes, for column k+1, its best unused row already
// scaled by the inverse of its pivot entry (double-buffered in shared memory); after the barrier
// every thread picks the same winner (largest value, smallest row on ties) and reads the pivot row
// straight from the winner's slot.
template <typename T, int NMAX>
__global__ void __launch_bounds__(NMAX * 4) k_leaf_inverse(cx<T>* Ag, long lda, long sA, int n,
                                                          const int* active, int* status) {
  constexpr int WARPS = NMAX / 8, C = NMAX / 32;
  const int e = blockIdx.x;
  if (active && !active[e]) return;
  __shared__ T s_val[2][WARPS];
  __shared__ int s_row[2][WARPS];
  __shared__ cx<T> s_prow[2][WARPS][NMAX];
  cx<T>* A = Ag + (long)e * sA;
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  cx<T> a[8][C];
  int rowstep[8], colpiv[C];
  unsigned used = 0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int i = w + WARPS * m;
    rowstep[m] = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int j = lane + 32 * c;
      a[m][c] = (i < n && j < n) ? A[(long)i * lda + j] : mk<T>(T(0), T(0));
    }
  }
#pragma unroll
  for (int c = 0; c < C; ++c) colpiv[c] = 0;

  // publish this warp's pivot candidate for column kk into buffer b
  auto publish = [&](int kk, int b) {
    const int cc = kk / 32, owner = kk % 32;
    T best = T(-1);
    int bm = -1;
    if (lane == owner) {
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int i = w + WARPS * m;
        const cx<T> v = cc == 0 ? a[m][0] : a[m][C - 1];
        const T av = cabs1(v);
        if (i < n && !((used >> m) & 1u) && av > best) {
          best = av;
          bm = m;
        }
      }
    }
    best = __shfl_sync(0xffffffffu, best, owner);
    bm = __shfl_sync(0xffffffffu, bm, owner);
    if (bm >= 0) {
      cx<T> row[C];
#pragma unroll
      for (int c = 0; c < C; ++c) row[c] = mk<T>(T(0), T(0));
#pragma unroll
      for (int m = 0; m < 8; ++m)
        if (m == bm)
#pragma unroll
          for (int c = 0; c < C; ++c) row[c] = a[m][c];
      cx<T> pv = cc == 0 ? row[0] : row[C - 1];
      pv.re = __shfl_sync(0xffffffffu, pv.re, owner);
      pv.im = __shfl_sync(0xffffffffu, pv.im, owner);
      const cx<T> r = crecip(pv);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int j = lane + 32 * c;
        s_prow[b][w][j] = (j == kk) ? r : row[c] * r;
      }
    }
    if (lane == 0) {
      s_val[b][w] = best;
      s_row[b][w] = bm >= 0 ? w + WARPS * bm : -1;
    }
  };

  bool bad = false;
  if (n > 0) publish(0, 0);
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const int b = k & 1;
    T best = T(-1);
    int p = -1, ww = 0;
#pragma unroll
    for (int q = 0; q < WARPS; ++q) {
      const T v = s_val[b][q];
      const int ri = s_row[b][q];
      if (ri >= 0 && (v > best || (v == best && ri < p))) {
        best = v;
        p = ri;
        ww = q;
      }
    }
    if (!(best > T(0)) || !isfinite(best)) {
      bad = true;
      break;
    }
    const cx<T> r = s_prow[b][ww][k];
    cx<T> prow[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      prow[c] = s_prow[b][ww][lane + 32 * c];
      if (lane + 32 * c == k) colpiv[c] = p;
    }
    const int cc = k / 32, owner = k % 32;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int i = w + WARPS * m;
      cx<T> f = cc == 0 ? a[m][0] : a[m][C - 1];
      f.re = __shfl_sync(0xffffffffu, f.re, owner);
      f.im = __shfl_sync(0xffffffffu, f.im, owner);
      if (i == p) {
#pragma unroll
        for (int c = 0; c < C; ++c) a[m][c] = prow[c];
        used |= 1u << m;
        rowstep[m] = k;
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          if (lane + 32 * c == k) {
            a[m][c] = mk<T>(-(f.re * r.re - f.im * r.im), -(f.re * r.im + f.im * r.re));
          } else {
            cx<T> v = a[m][c];
            v.re = fma(-f.re, prow[c].re, v.re);
            v.re = fma(f.im, prow[c].im, v.re);
            v.im = fma(-f.re, prow[c].im, v.im);
            v.im = fma(-f.im, prow[c].re, v.im);
            a[m][c] = v;
          }
        }
      }
    }
    if (k + 1 < n) publish(k + 1, b ^ 1);
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0 && status) atomicCAS(status + e, 0, (int)QTX_ERR_SINGULAR);
    return;
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int i = w + WARPS * m;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int j = lane + 32 * c;
      if (i < n && j < n) A[(long)rowstep[m] * lda + colpiv[c]] = a[m][c];
    }
  }
}

template <typename T>
cudaError_t leaf_inverse(cx<T>* A, long lda, long sA, int n, int batch, const int* active, int* status,
                         cudaStream_t st) {
  if (n <= 0 || n > kLeafMax) return cudaErrorInvalidValue;
  if (n <= 32)
    k_leaf_inverse<T, 32><<<batch, 128, 0, st>>>(A, lda, sA, n, active, status);
  else
    k_leaf_inverse<T, 64><<<batch, 256, 0, st>>>(A, lda, sA, n, active, status);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t leaf_inverse<double>(cx<double>*, long, long, int, int, const int*, int*, cudaStream_t);
template cudaError_t leaf_inverse<float>(cx<float>*, long, long, int, int, const int*, int*, cudaStream_t);

// ============================================================================ elementwise
// Accumulator of a combination: FP64 when FP64 data is involved, df32 (error-free FP32 steps) when
// df32 data is, FP32 otherwise -- so the emulated and FP32 sweeps never touch the FP64 pipe here.
template <typename Tin, typename Tout>
struct AccSel {
  using type = float;
};
template <typename Tout>
struct AccSel<double, Tout> {
  using type = double;
};
template <>
struct AccSel<float, double> {
  using type = double;
};
template <>
struct AccSel<df, double> {  // df32 sums, converted to FP64 once (no FP64 arithmetic)
  using type = df;
};
template <>
struct AccSel<df, df> {
  using type = df;
};
template <>
struct AccSel<df, float> {
  using type = df;
};
template <>
struct AccSel<float, df> {
  using type = df;
};

__device__ __forceinline__ void acc_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void acc_zero(float& a) { a = 0.f; }
__device__ __forceinline__ void acc_zero(df& a) { a = mkdf(0.f, 0.f); }
__device__ __forceinline__ df as_df(float x) { return mkdf(x, 0.f); }
__device__ __forceinline__ df as_df(df x) { return x; }
__device__ __forceinline__ df as_df(double x) { return from_d<df>(x); }
template <typename X>
__device__ __forceinline__ void acc_axpy(double& a, double alpha, X x) { a += alpha * to_d(x); }
template <typename X>
__device__ __forceinline__ void acc_axpy(float& a, double alpha, X x) { a = fmaf((float)alpha, (float)to_d(x), a); }
__device__ __forceinline__ void acc_axpy(float& a, double alpha, float x) { a = fmaf((float)alpha, x, a); }
template <typename X>
__device__ __forceinline__ void acc_axpy(df& a, double alpha, X x) {
  const df v = as_df(x);
  a = df_add(a, alpha == 1.0 ? v : (alpha == -1.0 ? df_neg(v) : df_mulf(v, (float)alpha)));
}
// the same with the coefficient classified on the host (kind +1 / -1 / 0 = general, alpha in FP32)
template <typename X>
__device__ __forceinline__ void acc_axpy_k(df& a, int kind, float alpha_f, double, X x) {
  const df v = as_df(x);
  a = df_add(a, kind == 1 ? v : (kind == -1 ? df_neg(v) : df_mulf(v, alpha_f)));
}
template <typename X>
__device__ __forceinline__ void acc_axpy_k(float& a, int, float alpha_f, double, X x) {
  a = fmaf(alpha_f, (float)to_d(x), a);
}
__device__ __forceinline__ void acc_axpy_k(float& a, int, float alpha_f, double, float x) { a = fmaf(alpha_f, x, a); }
template <typename X>
__device__ __forceinline__ void acc_axpy_k(double& a, int, float, double alpha, X x) { a += alpha * to_d(x); }
__device__ __forceinline__ void acc_add_d(double& a, double z) { a += z; }
__device__ __forceinline__ void acc_add_d(float& a, double z) { a += (float)z; }
__device__ __forceinline__ void acc_add_d(df& a, double z) { a = df_add(a, from_d<df>(z)); }
template <typename Tout>
__device__ __forceinline__ Tout acc_out(double a) { return from_d<Tout>(a); }
template <typename Tout>
__device__ __forceinline__ Tout acc_out(float a);
template <>
__device__ __forceinline__ float acc_out<float>(float a) { return a; }
template <typename Tout>
__device__ __forceinline__ Tout acc_out(df a);
template <>
__device__ __forceinline__ df acc_out<df>(df a) { return a; }
template <>
__device__ __forceinline__ float acc_out<float>(df a) { return a.hi + a.lo; }
template <>
__device__ __forceinline__ double acc_out<double>(df a) { return to_d(a); }

// 32 x 32 output tiles; conjugate-transposed terms are staged through shared memory so that both
// the read and the write stay coalesced.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) k_combine(cx<Tout>* out, long sOut, Term<Tin> t0, Term<Tin> t1,
                                                 Term<Tin> t2, int b, const double* E, double eta,
                                                 double diag_coef, int has_diag, const int* active) {
  using Acc = typename AccSel<Tin, Tout>::type;
  const int e = blockIdx.z;
  if (active && !active[e]) return;
  __shared__ cx<Tin> tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  Acc accr[4], acci[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    acc_zero(accr[q]);
    acc_zero(acci[q]);
  }
  const Term<Tin> ts[3] = {t0, t1, t2};
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const Term<Tin>& T_ = ts[t];
    if (!T_.p) continue;
    const cx<Tin>* X = T_.p + (long)e * T_.s;
    if (T_.op == OP_N) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = r0 + ty + 8 * q, c = c0 + tx;
        if (r < b && c < b) {
          const cx<Tin> v = X[(long)r * b + c];
          acc_axpy_k(accr[q], T_.kind, T_.alpha_f, T_.alpha, v.re);
          acc_axpy_k(acci[q], T_.kind, T_.alpha_f, T_.alpha, v.im);
        }
      }
    } else {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) {  // tile[cc][rr] = X[c0+cc][r0+rr]
        const int rr = tx, cc = ty + 8 * q;
        const int xr = c0 + cc, xc = r0 + rr;
        if (xr < b && xc < b) tile[cc][rr] = X[(long)xr * b + xc];
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) {  // out(r, c) gets conj(X(c, r)) = conj(tile[c - c0][r - r0])
        const int r = r0 + ty + 8 * q, c = c0 + tx;
        if (r < b && c < b) {
          const cx<Tin> v = tile[tx][ty + 8 * q];
          acc_axpy_k(accr[q], T_.kind, T_.alpha_f, T_.alpha, v.re);
          acc_axpy_k(acci[q], -T_.kind, -T_.alpha_f, -T_.alpha, v.im);
        }
      }
    }
  }
  cx<Tout>* O = out + (long)e * sOut;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = r0 + ty + 8 * q, c = c0 + tx;
    if (r < b && c < b) {
      if (r == c && has_diag) {
        acc_add_d(accr[q], E ? diag_coef * E[e] : 0.0);
        acc_add_d(acci[q], diag_coef * eta);
      }
      cx<Tout> o;
      o.re = acc_out<Tout>(accr[q]);
      o.im = acc_out<Tout>(acci[q]);
      O[(long)r * b + c] = o;
    }
  }
}

// Without transposed terms every operand and the output are read and written in the same
// row-major order: one flat grid-stride pass per energy, with more bytes in flight per thread than
// the 32 x 32 tiles above (the tiled pass runs the output conversions at about half the HBM rate).
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) k_combine_flat(cx<Tout>* out, long sOut, Term<Tin> t0, Term<Tin> t1,
                                                      Term<Tin> t2, int b, const double* E, double eta,
                                                      double diag_coef, int has_diag, const int* active) {
  using Acc = typename AccSel<Tin, Tout>::type;
  const int e = blockIdx.y;
  if (active && !active[e]) return;
  const int bb = b * b;
  const cx<Tin>* X0 = t0.p ? t0.p + (long)e * t0.s : nullptr;
  const cx<Tin>* X1 = t1.p ? t1.p + (long)e * t1.s : nullptr;
  const cx<Tin>* X2 = t2.p ? t2.p + (long)e * t2.s : nullptr;
  cx<Tout>* O = out + (long)e * sOut;
  const double dre = has_diag ? (E ? diag_coef * E[e] : 0.0) : 0.0, dim_ = has_diag ? diag_coef * eta : 0.0;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < bb; idx += gridDim.x * blockDim.x) {
    Acc ar, ai;
    acc_zero(ar);
    acc_zero(ai);
    if (X0) {
      const cx<Tin> v = X0[idx];
      acc_axpy_k(ar, t0.kind, t0.alpha_f, t0.alpha, v.re);
      acc_axpy_k(ai, t0.kind, t0.alpha_f, t0.alpha, v.im);
    }
    if (X1) {
      const cx<Tin> v = X1[idx];
      acc_axpy_k(ar, t1.kind, t1.alpha_f, t1.alpha, v.re);
      acc_axpy_k(ai, t1.kind, t1.alpha_f, t1.alpha, v.im);
    }
    if (X2) {
      const cx<Tin> v = X2[idx];
      acc_axpy_k(ar, t2.kind, t2.alpha_f, t2.alpha, v.re);
      acc_axpy_k(ai, t2.kind, t2.alpha_f, t2.alpha, v.im);
    }
    if (has_diag && idx % (b + 1) == 0) {  // row == column
      acc_add_d(ar, dre);
      acc_add_d(ai, dim_);
    }
    cx<Tout> o;
    o.re = acc_out<Tout>(ar);
    o.im = acc_out<Tout>(ai);
    O[idx] = o;
  }
}
// CTAs along one energy's elements: about eight per SM over the whole batch, at least one per energy
static unsigned flat_ctas(long bb, int batch) {
  const long want = (8L * 152 + batch - 1) / batch, most = (bb + 255) / 256;
  return (unsigned)(want < 1 ? 1 : (want > most ? most : want));
}

template <typename Tin, typename Tout>
cudaError_t combine(cx<Tout>* out, long sOut, Term<Tin> t0, Term<Tin> t1, Term<Tin> t2, int b,
                    int batch, const double* E, double eta, double diag_coef, const int* active,
                    cudaStream_t st) {
  auto classify = [](Term<Tin>& t) {
    t.kind = t.alpha == 1.0 ? 1 : (t.alpha == -1.0 ? -1 : 0);
    t.alpha_f = (float)t.alpha;
  };
  classify(t0);
  classify(t1);
  classify(t2);
  auto direct = [](const Term<Tin>& t) { return !t.p || t.op != OP_C; };  // absent terms count as direct
  if (direct(t0) && direct(t1) && direct(t2)) {
    dim3 fgrid(flat_ctas((long)b * b, batch), batch);
    k_combine_flat<Tin, Tout><<<fgrid, 256, 0, st>>>(out, sOut, t0, t1, t2, b, E, eta, diag_coef, diag_coef != 0.0,
                                                     active);
    count_launch();
    return cudaGetLastError();
  }
  dim3 grid((b + 31) / 32, (b + 31) / 32, batch);
  k_combine<Tin, Tout><<<grid, 256, 0, st>>>(out, sOut, t0, t1, t2, b, E, eta, diag_coef, diag_coef != 0.0, active);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t combine<double, double>(cx<double>*, long, Term<double>, Term<double>, Term<double>, int, int, const double*, double, double, const int*, cudaStream_t);
template cudaError_t combine<float, float>(cx<float>*, long, Term<float>, Term<float>, Term<float>, int, int, const double*, double, double, const int*, cudaStream_t);
template cudaError_t combine<float, double>(cx<double>*, long, Term<float>, Term<float>, Term<float>, int, int, const double*, double, double, const int*, cudaStream_t);
template cudaError_t combine<double, float>(cx<float>*, long, Term<double>, Term<double>, Term<double>, int, int, const double*, double, double, const int*, cudaStream_t);
template cudaError_t combine<df, df>(cx<df>*, long, Term<df>, Term<df>, Term<df>, int, int, const double*, double, double, const int*, cudaStream_t);
template cudaError_t combine<df, double>(cx<double>*, long, Term<df>, Term<df>, Term<df>, int, int, const double*, double, double, const int*, cudaStream_t);
template cudaError_t combine<df, float>(cx<float>*, long, Term<df>, Term<df>, Term<df>, int, int, const double*, double, double, const int*, cudaStream_t);
template cudaError_t combine<float, df>(cx<df>*, long, Term<float>, Term<float>, Term<float>, int, int, const double*, double, double, const int*, cudaStream_t);
template cudaError_t combine<double, df>(cx<df>*, long, Term<double>, Term<double>, Term<double>, int, int, const double*, double, double, const int*, cudaStream_t);

template <typename T>
__global__ void k_assemble_diag(cx<T>* out, const cx<double>* H, const cx<double>* S,
                                const cx<double>* SigR, long sSig, const cx<double>* lead,
                                long sLead, const double* E, double eta, int b) {
  const int e = blockIdx.y;
  const int bb = b * b;  // b <= 4096: 32-bit indices (no 64-bit division per element)
  const double Er = E[e];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < bb; idx += gridDim.x * blockDim.x) {
    const int r = idx / b, c = idx - r * b;
    if constexpr (std::is_same<T, df>::value) {
      if (!S) {  // df32 arithmetic on the exactly split inputs: no FP64 operations
        df vr = r == c ? from_d<df>(Er) : mkdf(0.f, 0.f), vi = r == c ? from_d<df>(eta) : mkdf(0.f, 0.f);
        const cx<double> h = H[idx];
        vr = df_sub(vr, from_d<df>(h.re));
        vi = df_sub(vi, from_d<df>(h.im));
        if (SigR) {
          const cx<double> x = SigR[(long)e * sSig + idx];
          vr = df_sub(vr, from_d<df>(x.re));
          vi = df_sub(vi, from_d<df>(x.im));
        }
        if (lead) {
          const cx<double> x = lead[(long)e * sLead + idx];
          vr = df_sub(vr, from_d<df>(x.re));
          vi = df_sub(vi, from_d<df>(x.im));
        }
        cx<df> o;
        o.re = vr;
        o.im = vi;
        out[(long)e * bb + idx] = o;
        continue;
      }
    }
    cx<double> s = S ? S[idx] : mk<double>(r == c ? 1.0 : 0.0, 0.0);
    cx<double> v = mk<double>(Er * s.re - eta * s.im, Er * s.im + eta * s.re) - H[idx];
    if (SigR) v = v - SigR[(long)e * sSig + idx];
    if (lead) v = v - lead[(long)e * sLead + idx];
    out[(long)e * bb + idx] = cvt<T>(v);
  }
}
template <typename T>
cudaError_t assemble_diag(cx<T>* out, const cx<double>* H, const cx<double>* S,
                          const cx<double>* SigR, long sSig, const cx<double>* lead, long sLead,
                          const double* E, double eta, int b, int batch, cudaStream_t st) {
  const long bb = (long)b * b;
  dim3 grid((unsigned)((bb + 255) / 256 < 1024 ? (bb + 255) / 256 : 1024), batch);
  k_assemble_diag<T><<<grid, 256, 0, st>>>(out, H, S, SigR, sSig, lead, sLead, E, eta, b);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t assemble_diag<double>(cx<double>*, const cx<double>*, const cx<double>*, const cx<double>*, long, const cx<double>*, long, const double*, double, int, int, cudaStream_t);
template cudaError_t assemble_diag<float>(cx<float>*, const cx<double>*, const cx<double>*, const cx<double>*, long, const cx<double>*, long, const double*, double, int, int, cudaStream_t);
template cudaError_t assemble_diag<df>(cx<df>*, const cx<double>*, const cx<double>*, const cx<double>*, long, const cx<double>*, long, const double*, double, int, int, cudaStream_t);

template <typename T>
__global__ void k_axpby_from64(cx<T>* out, long sOut, const cx<double>* X, long sX, double c1,
                               const cx<double>* Y, long sY, double c2, int b, int k1, int k2) {
  const int e = blockIdx.y;
  const long bb = (long)b * b;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < bb; idx += (long)gridDim.x * blockDim.x) {
    if constexpr (std::is_same<T, df>::value) {  // df32 arithmetic: no FP64 operations
      // k = +1 / -1 / 0 (general coefficient, split to df32 once per element)
      auto scaled = [](int k, double c, double x) {
        const df v = from_d<df>(x);
        return k == 1 ? v : (k == -1 ? df_neg(v) : df_mul(v, from_d<df>(c)));
      };
      const cx<double> x = X[(long)e * sX + idx];
      df vr = scaled(k1, c1, x.re), vi = scaled(k1, c1, x.im);
      if (Y) {
        const cx<double> y = Y[(long)e * sY + idx];
        vr = df_add(vr, scaled(k2, c2, y.re));
        vi = df_add(vi, scaled(k2, c2, y.im));
      }
      cx<df> o;
      o.re = vr;
      o.im = vi;
      out[(long)e * sOut + idx] = o;
    } else {
      cx<double> v = c1 * X[(long)e * sX + idx];
      if (Y) v = v + c2 * Y[(long)e * sY + idx];
      out[(long)e * sOut + idx] = cvt<T>(v);
    }
  }
}
template <typename T>
cudaError_t axpby_from64(cx<T>* out, long sOut, const cx<double>* X, long sX, double c1,
                         const cx<double>* Y, long sY, double c2, int b, int batch, cudaStream_t st) {
  const long bb = (long)b * b;
  dim3 grid((unsigned)((bb + 255) / 256 < 1024 ? (bb + 255) / 256 : 1024), batch);
  const int k1 = c1 == 1.0 ? 1 : (c1 == -1.0 ? -1 : 0), k2 = c2 == 1.0 ? 1 : (c2 == -1.0 ? -1 : 0);
  k_axpby_from64<T><<<grid, 256, 0, st>>>(out, sOut, X, sX, c1, Y, sY, c2, b, k1, k2);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t axpby_from64<double>(cx<double>*, long, const cx<double>*, long, double, const cx<double>*, long, double, int, int, cudaStream_t);
template cudaError_t axpby_from64<float>(cx<float>*, long, const cx<double>*, long, double, const cx<double>*, long, double, int, int, cudaStream_t);
template cudaError_t axpby_from64<df>(cx<df>*, long, const cx<double>*, long, double, const cx<double>*, long, double, int, int, cudaStream_t);

// out[e] = src (one block shared by every energy) plus E[e] + i eta on the diagonal (E may be
// nullptr: no diagonal term).  The sweep's per-energy copy of a block whose FP64 -> df32 / FP32
// conversion was done once; only the writes remain.
__device__ __forceinline__ df add_t(df a, df c) { return df_add(a, c); }
__device__ __forceinline__ float add_t(float a, float c) { return a + c; }
template <typename T>
__global__ void __launch_bounds__(256) k_broadcast_diag(cx<T>* out, long sOut, const cx<T>* src, int b,
                                                        const double* E, double eta) {
  const int e = blockIdx.y;
  const int bb = b * b;
  cx<T> z;
  if (E) {
    z.re = from_d<T>(E[e]);
    z.im = from_d<T>(eta);
  }
  cx<T>* O = out + (long)e * sOut;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < bb; idx += gridDim.x * blockDim.x) {
    cx<T> v = src[idx];
    if (E && idx % (b + 1) == 0) {  // row == column
      v.re = add_t(v.re, z.re);
      v.im = add_t(v.im, z.im);
    }
    O[idx] = v;
  }
}
template <typename T>
cudaError_t broadcast_diag(cx<T>* out, long sOut, const cx<T>* src, int b, const double* E, double eta, int batch,
                           cudaStream_t st) {
  dim3 grid(flat_ctas((long)b * b, batch), batch);
  k_broadcast_diag<T><<<grid, 256, 0, st>>>(out, sOut, src, b, E, eta);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t broadcast_diag<float>(cx<float>*, long, const cx<float>*, int, const double*, double, int, cudaStream_t);
template cudaError_t broadcast_diag<df>(cx<df>*, long, const cx<df>*, int, const double*, double, int, cudaStream_t);

template <typename T>
__global__ void k_assemble_offdiag(cx<T>* U, cx<T>* V, const cx<double>* Hup, const cx<double>* Sup,
                                   const double* E, double eta, int b, const cx<double>* SRu,
                                   const cx<double>* SRl, long sSR) {
  const int e = blockIdx.z;
  __shared__ cx<double> tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  const double Er = E ? E[e] : 0.0, ei = E ? eta : 0.0;
  const long bb = (long)b * b;
  // U(r, c) = z S(r, c) - H(r, c)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = r0 + ty + 8 * q, c = c0 + tx;
    if (r < b && c < b) {
      const cx<double> s = Sup ? Sup[(long)r * b + c] : mk<double>(0, 0);
      cx<double> h = Hup[(long)r * b + c];
      if (SRu) h = h + SRu[(long)e * sSR + (long)r * b + c];  // U = z S - H - Sigma^R_{i,i+1}
      U[(long)e * bb + (long)r * b + c] = cvt<T>(mk<double>(Er * s.re - ei * s.im - h.re, Er * s.im + ei * s.re - h.im));
    }
  }
  // V(r, c) = z conj(S(c, r)) - conj(H(c, r))
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int cc = ty + 8 * q, rr = tx;
    const int xr = c0 + cc, xc = r0 + rr;
    if (xr < b && xc < b) {
      const cx<double> s = Sup ? Sup[(long)xr * b + xc] : mk<double>(0, 0);
      const cx<double> h = Hup[(long)xr * b + xc];
      // z * conj(s) - conj(h)
      tile[cc][rr] = mk<double>(Er * s.re + ei * s.im - h.re, -Er * s.im + ei * s.re + h.im);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = r0 + ty + 8 * q, c = c0 + tx;
    if (r < b && c < b) {
      cx<double> v = tile[tx][ty + 8 * q];
      if (SRl) v = v - SRl[(long)e * sSR + (long)r * b + c];  // V = z S^H - H^H - Sigma^R_{i+1,i}
      V[(long)e * bb + (long)r * b + c] = cvt<T>(v);
    }
  }
}
template <typename T>
cudaError_t assemble_offdiag(cx<T>* U, cx<T>* V, const cx<double>* Hup, const cx<double>* Sup,
                             const double* E, double eta, int b, int batch, cudaStream_t st,
                             const cx<double>* SRu, const cx<double>* SRl, long sSR) {
  dim3 grid((b + 31) / 32, (b + 31) / 32, batch);
  k_assemble_offdiag<T><<<grid, 256, 0, st>>>(U, V, Hup, Sup, E, eta, b, SRu, SRl, sSR);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t assemble_offdiag<double>(cx<double>*, cx<double>*, const cx<double>*, const cx<double>*, const double*, double, int, int, cudaStream_t, const cx<double>*, const cx<double>*, long);
template cudaError_t assemble_offdiag<float>(cx<float>*, cx<float>*, const cx<double>*, const cx<double>*, const double*, double, int, int, cudaStream_t, const cx<double>*, const cx<double>*, long);
template cudaError_t assemble_offdiag<df>(cx<df>*, cx<df>*, const cx<double>*, const cx<double>*, const double*, double, int, int, cudaStream_t, const cx<double>*, const cx<double>*, long);

__global__ void __launch_bounds__(256) k_residual_mask(const cx<df>* R, long sR, long nn, float tol2,
                                                       const int* active, int* next, int* status) {
  const int e = blockIdx.x;
  if (active && !active[e]) {
    if (threadIdx.x == 0) next[e] = 0;
    return;
  }
  const cx<df>* X = R + (long)e * sR;
  float s = 0.f;
  for (long i = threadIdx.x; i < nn; i += blockDim.x) s = fmaf(X[i].re.hi, X[i].re.hi, fmaf(X[i].im.hi, X[i].im.hi, s));
  __shared__ float red[8];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) s += red[w];
    // a NaN or infinite norm compares false against tol2: such an energy keeps refining, and its
    // block inverse has failed, so it is reported singular
    next[e] = (s <= tol2) ? 0 : 1;
    if (status && !(s <= 3.0e38f)) atomicCAS(status + e, 0, (int)QTX_ERR_SINGULAR);
  }
}
cudaError_t residual_mask(const cx<df>* R, long sR, int n, int batch, double tol, const int* active, int* next,
                          int* status, cudaStream_t st) {
  k_residual_mask<<<batch, 256, 0, st>>>(R, sR, (long)n * n, (float)(tol * tol), active, next, status);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void k_add_identity(cx<T>* X, long sX, int n, const int* active) {
  const int e = blockIdx.y;
  if (active && !active[e]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) X[(long)e * sX + (long)i * n + i].re += T(1);
}
template <typename T>
cudaError_t add_identity(cx<T>* X, long sX, int n, int batch, const int* active, cudaStream_t st) {
  dim3 grid((n + 127) / 128, batch);
  k_add_identity<T><<<grid, 128, 0, st>>>(X, sX, n, active);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t add_identity<double>(cx<double>*, long, int, int, const int*, cudaStream_t);
template cudaError_t add_identity<float>(cx<float>*, long, int, int, const int*, cudaStream_t);

// ============================================================================ strided conversion
template <typename Tin, typename Tout>
__global__ void k_convert(const cx<Tin>* in, long ldi, long si, cx<Tout>* out, long ldo, long so, int rows,
                          int cols) {
  const int e = blockIdx.z;
  const int r = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x)
    out[(long)e * so + (long)r * ldo + c] = cvt<Tout>(in[(long)e * si + (long)r * ldi + c]);
}
template <typename Tin, typename Tout>
cudaError_t convert_strided(const cx<Tin>* in, long ldi, long si, cx<Tout>* out, long ldo, long so, int rows,
                            int cols, int batch, cudaStream_t st) {
  if (rows <= 0 || cols <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((cols + 127) / 128 < 8 ? (cols + 127) / 128 : 8, rows, batch);
  k_convert<Tin, Tout><<<grid, 128, 0, st>>>(in, ldi, si, out, ldo, so, rows, cols);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t convert_strided<double, double>(const cx<double>*, long, long, cx<double>*, long, long, int, int, int, cudaStream_t);
template cudaError_t convert_strided<double, float>(const cx<double>*, long, long, cx<float>*, long, long, int, int, int, cudaStream_t);
template cudaError_t convert_strided<float, double>(const cx<float>*, long, long, cx<double>*, long, long, int, int, int, cudaStream_t);
template cudaError_t convert_strided<double, df>(const cx<double>*, long, long, cx<df>*, long, long, int, int, int, cudaStream_t);
template cudaError_t convert_strided<df, double>(const cx<df>*, long, long, cx<double>*, long, long, int, int, int, cudaStream_t);

// ============================================================================ observables
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) s += red[i];
  return s;  // valid in thread 0
}

// One energy's trace is split over `parts` CTAs (blockIdx.x) when the batch alone would leave most
// SMs idle (few energies of large blocks); each writes its partial sum (df32, or FP64 when FP64
// arithmetic is used) to `partial`, and k_obs_current_sum adds them in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_obs_current(double* cur, long ldcur, const cx<double>* Hup,
                                                     const cx<double>* Sup, const cx<T>* GLu, long sG,
                                                     const double* E, int b, int parts, double* partial) {
  const int e = blockIdx.y, part = blockIdx.x;
  const long bb = (long)b * b;
  const long chunk = (bb + parts - 1) / parts;
  const long i0 = (long)part * chunk, i1 = i0 + chunk < bb ? i0 + chunk : bb;
  const double Er = E[e];
  const cx<T>* G = GLu + (long)e * sG;
  double s = 0.0;
  if constexpr (std::is_same<T, df>::value) {
    if (!Sup) {  // df32 products and sums: no FP64 arithmetic per element
      df a = mkdf(0.f, 0.f);
      for (long idx = i0 + threadIdx.x; idx < i1; idx += blockDim.x) {
        const cx<double> x = Hup[idx];
        const cx<df> g = G[idx];
        a = df_add(a, df_add(df_mul(from_d<df>(x.re), g.re), df_mul(from_d<df>(x.im), g.im)));
      }
      __shared__ df red[8];
      for (int off = 16; off > 0; off >>= 1)
        a = df_add(a, mkdf(__shfl_down_sync(0xffffffffu, a.hi, off), __shfl_down_sync(0xffffffffu, a.lo, off)));
      if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = a;
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int i = 1; i < (int)blockDim.x / 32; ++i) a = df_add(a, red[i]);
        if (parts == 1) cur[(long)e * ldcur] = -2.0 * to_d(a);
        else reinterpret_cast<df*>(partial)[(long)e * parts + part] = a;
      }
      return;
    }
  }
  for (long idx = i0 + threadIdx.x; idx < i1; idx += blockDim.x) {
    cx<double> x = Hup[idx];
    if (Sup) x = x - Er * Sup[idx];
    const cx<double> gg = cvt<double>(G[idx]);
    s += x.re * gg.re + x.im * gg.im;  // Re(x * conj(g))
  }
  s = block_sum(s);
  // 2 Re Tr[X (-GLu^H)] = -2 sum_jk Re(X_jk conj(GLu_jk))
  if (threadIdx.x == 0) {
    if (parts == 1) cur[(long)e * ldcur] = -2.0 * s;
    else partial[(long)e * parts + part] = s;
  }
}
// the partial sums of one energy, in order (df32 partials: the df32 path of k_obs_current)
__global__ void k_obs_current_sum(double* cur, long ldcur, const double* partial, int parts, int df_parts) {
  const int e = blockIdx.x;
  if (threadIdx.x != 0) return;
  if (df_parts) {
    const df* pp = reinterpret_cast<const df*>(partial) + (long)e * parts;
    df a = pp[0];
    for (int k = 1; k < parts; ++k) a = df_add(a, pp[k]);
    cur[(long)e * ldcur] = -2.0 * to_d(a);
  } else {
    double a = 0.0;
    for (int k = 0; k < parts; ++k) a += partial[(long)e * parts + k];
    cur[(long)e * ldcur] = -2.0 * a;
  }
}
template <typename T>
cudaError_t obs_current(double* cur, long ldcur, const cx<double>* Hup, const cx<double>* Sup,
                        const cx<T>* GLu, long sG, const double* E, int b, int batch, cudaStream_t st,
                        double* scratch, long scratch_doubles) {
  // about two CTAs per SM in all; at least 64 K elements per CTA
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 1;
  }
  const long bb = (long)b * b;
  long parts = (2L * sms + batch - 1) / batch;
  const long by_size = bb / 65536 > 0 ? bb / 65536 : 1;
  if (parts > by_size) parts = by_size;
  if (parts > 1024) parts = 1024;
  if (!scratch || parts * batch > scratch_doubles) parts = 1;
  dim3 grid((unsigned)parts, batch);
  k_obs_current<T><<<grid, 256, 0, st>>>(cur, ldcur, Hup, Sup, GLu, sG, E, b, (int)parts, scratch);
  count_launch();
  if (parts > 1) {
    k_obs_current_sum<<<batch, 32, 0, st>>>(cur, ldcur, scratch, (int)parts, std::is_same<T, df>::value && !Sup);
    count_launch();
  }
  return cudaGetLastError();
}
template cudaError_t obs_current<double>(double*, long, const cx<double>*, const cx<double>*, const cx<double>*, long, const double*, int, int, cudaStream_t, double*, long);
template cudaError_t obs_current<float>(double*, long, const cx<double>*, const cx<double>*, const cx<float>*, long, const double*, int, int, cudaStream_t, double*, long);
template cudaError_t obs_current<df>(double*, long, const cx<double>*, const cx<double>*, const cx<df>*, long, const double*, int, int, cudaStream_t, double*, long);

template <typename T>
__global__ void k_obs_density(double* den, long ldden, const cx<T>* GL, long sG, int b) {
  const int e = blockIdx.x;
  const cx<T>* G = GL + (long)e * sG;
  double s = 0.0;
  for (int i = threadIdx.x; i < b; i += blockDim.x) s += to_d(G[(long)i * b + i].im);
  s = block_sum(s);
  if (threadIdx.x == 0) den[(long)e * ldden] = s;
}
template <typename T>
cudaError_t obs_density(double* den, long ldden, const cx<T>* GL, long sG, int b, int batch, cudaStream_t st) {
  k_obs_density<T><<<batch, 128, 0, st>>>(den, ldden, GL, sG, b);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t obs_density<double>(double*, long, const cx<double>*, long, int, int, cudaStream_t);
template cudaError_t obs_density<float>(double*, long, const cx<float>*, long, int, int, cudaStream_t);
template cudaError_t obs_density<df>(double*, long, const cx<df>*, long, int, int, cudaStream_t);

// scale * Part Tr[X Y - Z W],  Part = Re (part 0) or Im (part 1);  Tr[X Y] = sum_jk X_jk Y_kj
template <typename T>
__global__ void __launch_bounds__(256) k_obs_trace2(double* out, long ld, const cx<double>* X, long sX,
                                                    const cx<T>* Y, long sY, const cx<double>* Z, long sZ,
                                                    const cx<T>* W, long sW, int b, int part, double scale) {
  const int e = blockIdx.x;
  const long bb = (long)b * b;
  double s = 0.0;
  for (long idx = threadIdx.x; idx < bb; idx += blockDim.x) {
    const int j = (int)(idx / b), k = (int)(idx % b);
    const cx<double> x = X[(long)e * sX + idx];
    const cx<double> y = cvt<double>(Y[(long)e * sY + (long)k * b + j]);
    s += part ? x.re * y.im + x.im * y.re : x.re * y.re - x.im * y.im;
    if (Z) {
      const cx<double> z = Z[(long)e * sZ + idx];
      const cx<double> w = cvt<double>(W[(long)e * sW + (long)k * b + j]);
      s -= part ? z.re * w.im + z.im * w.re : z.re * w.re - z.im * w.im;
    }
  }
  s = block_sum(s);
  if (threadIdx.x == 0) out[(long)e * ld] = scale * s;
}
template <typename T>
cudaError_t obs_trace2(double* out, long ld, const cx<double>* X, long sX, const cx<T>* Y, long sY,
                       const cx<double>* Z, long sZ, const cx<T>* Wm, long sW, int b, int batch,
                       cudaStream_t st, int part, double scale) {
  k_obs_trace2<T><<<batch, 256, 0, st>>>(out, ld, X, sX, Y, sY, Z, sZ, Wm, sW, b, part, scale);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t obs_trace2<double>(double*, long, const cx<double>*, long, const cx<double>*, long, const cx<double>*, long, const cx<double>*, long, int, int, cudaStream_t, int, double);
template cudaError_t obs_trace2<float>(double*, long, const cx<double>*, long, const cx<float>*, long, const cx<double>*, long, const cx<float>*, long, int, int, cudaStream_t, int, double);
template cudaError_t obs_trace2<df>(double*, long, const cx<double>*, long, const cx<df>*, long, const cx<double>*, long, const cx<df>*, long, int, int, cudaStream_t, int, double);

// Local current balance of slice i (current conservation, Sec. II-B):
//   J = Re Tr[Sigma^< G^>] - Re Tr[Sigma^> G^<],  G^> = G^< + G - G^H,
//   Sigma^> = Sigma^< + Sigma^R - Sigma^R^H - 2 i eta I  (the broadening acts as a sink),
// with Tr[X Y] = sum_jk X_jk Y_kj; Sigma pointers may be null (no scattering), sSig their batch stride.
// scale = the absolute sum of J's terms, sum_jk |Sigma^<_jk| |G^>_kj| + |Sigma^>_jk| |G^<_kj|, plus,
// when the interface (i, i+1) exists (GLu = G^<_{i,i+1} non-null), that of its current,
// 2 sum_jk |(H - E S)_{i,i+1, jk}| |G^<_{i,i+1, jk}|: the size of the terms each balance cancels, hence
// the scale of its rounding error.
// gn[e * ld] = ||G_ii||_F^2 and hn[e * ld] = ||H_ii||_F + 2 ||H_{i,i+1}||_F (Hd = H_ii, Hu may be null): the
// pieces of the condition estimate ||M|| ||G|| of the escalation check.
template <typename T>
__global__ void __launch_bounds__(256) k_obs_balance(double* out, double* scale, double* gn, double* hn, long ld,
                                                     const cx<double>* SL, const cx<double>* SR, long sSig,
                                                     const cx<T>* G, const cx<T>* GL, long sG, double eta, int b,
                                                     const cx<double>* Hd, const cx<double>* Hu,
                                                     const cx<double>* Su, const double* E, const cx<T>* GLu) {
  const int e = blockIdx.x;
  const long bb = (long)b * b;
  const cx<T>* Ge = G + (long)e * sG;
  const cx<T>* GLe = GL + (long)e * sG;
  double s = 0.0, a = 0.0, g2 = 0.0, hd2 = 0.0, hu2 = 0.0;
  for (long idx = threadIdx.x; idx < bb; idx += blockDim.x) {
    const int j = (int)(idx / b), k = (int)(idx % b);
    const long kj = (long)k * b + j;
    const cx<double> gl = cvt<double>(GLe[kj]);
    const cx<double> gkj = cvt<double>(Ge[kj]), gjk = cvt<double>(Ge[idx]);
    const cx<double> gg = mk<double>(gl.re + gkj.re - gjk.re, gl.im + gkj.im + gjk.im);  // G^>_kj
    cx<double> sl = mk<double>(0.0, 0.0), sg = mk<double>(0.0, j == k ? -2.0 * eta : 0.0);
    if (SL) {
      sl = SL[(long)e * sSig + idx];
      sg.re += sl.re;
      sg.im += sl.im;
    }
    if (SR) {
      const cx<double> rjk = SR[(long)e * sSig + idx], rkj = SR[(long)e * sSig + kj];
      sg.re += rjk.re - rkj.re;  // Sigma^R - Sigma^R^H
      sg.im += rjk.im + rkj.im;
    }
    s += (sl.re * gg.re - sl.im * gg.im) - (sg.re * gl.re - sg.im * gl.im);
    a += hypot(sl.re, sl.im) * hypot(gg.re, gg.im) + hypot(sg.re, sg.im) * hypot(gl.re, gl.im);
    g2 += gjk.re * gjk.re + gjk.im * gjk.im;
    const cx<double> hd = Hd[idx];
    hd2 += hd.re * hd.re + hd.im * hd.im;
    if (Hu) hu2 += Hu[idx].re * Hu[idx].re + Hu[idx].im * Hu[idx].im;
    if (GLu) {
      const cx<double> u = cvt<double>(GLu[(long)e * sG + idx]);
      cx<double> h = Hu[idx];
      if (Su) {
        const double Ee = E[e];
        h.re -= Ee * Su[idx].re;
        h.im -= Ee * Su[idx].im;
      }
      a += 2.0 * hypot(h.re, h.im) * hypot(u.re, u.im);
    }
  }
  s = block_sum(s);
  a = block_sum(a);
  g2 = block_sum(g2);
  hd2 = block_sum(hd2);
  hu2 = block_sum(hu2);
  if (threadIdx.x == 0) {
    out[(long)e * ld] = s;
    scale[(long)e * ld] = a;
    gn[(long)e * ld] = g2;
    hn[(long)e * ld] = sqrt(hd2) + 2.0 * sqrt(hu2);
  }
}
template <typename T>
cudaError_t obs_balance(double* out, double* scale, double* gn, double* hn, long ld, const cx<double>* SL,
                        const cx<double>* SR, long sSig, const cx<T>* G, const cx<T>* GL, long sG, double eta, int b,
                        int batch, cudaStream_t st, const cx<double>* Hd, const cx<double>* Hu, const cx<double>* Su,
                        const double* E, const cx<T>* GLu) {
  k_obs_balance<T><<<batch, 256, 0, st>>>(out, scale, gn, hn, ld, SL, SR, sSig, G, GL, sG, eta, b, Hd, Hu, Su, E, GLu);
  count_launch();
  return cudaGetLastError();
}
#define QTX_BAL(T)                                                                                                   \
  template cudaError_t obs_balance<T>(double*, double*, double*, double*, long, const cx<double>*,                \
                                      const cx<double>*, long, const cx<T>*, const cx<T>*, long, double, int, int,  \
                                      cudaStream_t, const cx<double>*, const cx<double>*, const cx<double>*,        \
                                      const double*, const cx<T>*);
QTX_BAL(double)
QTX_BAL(float)
QTX_BAL(df)
#undef QTX_BAL

// Continuity residual per energy: the largest violation of I_{i-1} + J_i = I_i over the slices
// (I_{-1} = I_L, I_{N_B-1} = -I_R with contacts, else 0), relative to the largest balance scale
// (k_obs_balance).  flag[e] = 1 when it is not below tol (NaN included), or when the condition
// estimate kappa = (|E| + max_i hn_i) max_i ||G_ii||_F times eps_mode (the arithmetic's unit error,
// Eq. 6's model error ~ kappa eps) is not below tol.  One thread per energy.
__global__ void k_continuity(const double* cur, long ldc, const double* J, const double* Js, const double* gn,
                             const double* hn, long ldj, const double* con, const double* E, int nb, int ne, double tol,
                             double eps_mode, double* res, int* flag) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const double* I = cur + (long)e * ldc;
  const double* Je = J + (long)e * ldj;
  const double* Se = Js + (long)e * ldj;
  const double IL = con ? con[2L * e] : 0.0, IR = con ? con[2L * e + 1] : 0.0;
  double worst = 0.0, scale = 0.0;
  for (int i = 0; i < nb; ++i) {
    const double prev = i == 0 ? IL : I[i - 1];
    const double next = i == nb - 1 ? -IR : I[i];
    const double r = fabs(prev + Je[i] - next);
    worst = (r > worst || r != r) ? r : worst;
    scale = fmax(scale, Se[i]);
  }
  const double rel = worst / (scale > 0.0 ? scale : 1.0);
  double g2 = 0.0, h = 0.0;
  for (int i = 0; i < nb; ++i) {
    g2 = fmax(g2, gn[(long)e * ldj + i]);
    h = fmax(h, hn[(long)e * ldj + i]);
  }
  const double kest = (fabs(E[e]) + h) * sqrt(g2);
  res[e] = rel;
  flag[e] = (rel < tol && kest * eps_mode < tol) ? 0 : 1;
}
cudaError_t continuity(const double* cur, long ldc, const double* J, const double* Js, const double* gn,
                       const double* hn, long ldj, const double* con, const double* E, int nb, int ne, double tol,
                       double eps_mode, double* res, int* flag, cudaStream_t st) {
  k_continuity<<<(ne + 127) / 128, 128, 0, st>>>(cur, ldc, J, Js, gn, hn, ldj, con, E, nb, ne, tol, eps_mode, res, flag);
  count_launch();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_obs_frob_dot(double* out, long ld, const cx<double>* X, long sX,
                                                      const cx<double>* Y, long sY, double scale, int b) {
  const int e = blockIdx.x;
  const long bb = (long)b * b;
  double s = 0.0;
  for (long idx = threadIdx.x; idx < bb; idx += blockDim.x) {
    const cx<double> x = X[(long)e * sX + idx], y = Y[(long)e * sY + idx];
    s += x.re * y.re + x.im * y.im;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) out[(long)e * ld] += scale * s;
}
cudaError_t obs_frob_dot(double* out, long ld, const cx<double>* X, long sX, const cx<double>* Y,
                         long sY, double scale, int b, int batch, cudaStream_t st) {
  k_obs_frob_dot<<<batch, 256, 0, st>>>(out, ld, X, sX, Y, sY, scale, b);
  count_launch();
  return cudaGetLastError();
}

// ============================================================================ leads
__device__ __forceinline__ double fermi_dev(double E, double mu, double kT) {
  const double x = (E - mu) / kT;
  if (x > 0) {
    const double ex = exp(-x);
    return ex / (1.0 + ex);
  }
  return 1.0 / (1.0 + exp(x));
}

__global__ void k_lead_sigmas(const cx<double>* SR, cx<double>* Gam, cx<double>* SL, cx<double>* SG,
                              const double* E, double mu, double kT, int b) {
  const int e = blockIdx.y;
  const long bb = (long)b * b;
  const double f = fermi_dev(E[e], mu, kT);
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < bb; idx += (long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / b), c = (int)(idx % b);
    const cx<double> s = SR[(long)e * bb + idx];
    const cx<double> st = SR[(long)e * bb + (long)c * b + r];
    // Gamma = i (S - S^H):  (S - S^H)(r,c) = s - conj(st)
    const cx<double> d = mk<double>(s.re - st.re, s.im + st.im);
    const cx<double> g = mk<double>(-d.im, d.re);
    Gam[(long)e * bb + idx] = g;
    SL[(long)e * bb + idx] = mk<double>(-f * g.im, f * g.re);                   // i f Gamma
    SG[(long)e * bb + idx] = mk<double>((1.0 - f) * g.im, -(1.0 - f) * g.re);  // -i (1-f) Gamma
  }
}
cudaError_t lead_sigmas(const cx<double>* SR, cx<double>* Gam, cx<double>* SL, cx<double>* SG,
                        const double* E, double mu, double kT, int b, int batch, cudaStream_t st) {
  const long bb = (long)b * b;
  dim3 grid((unsigned)((bb + 255) / 256 < 1024 ? (bb + 255) / 256 : 1024), batch);
  k_lead_sigmas<<<grid, 256, 0, st>>>(SR, Gam, SL, SG, E, mu, kT, b);
  count_launch();
  return cudaGetLastError();
}

// out[0] = max |X_jk| over one b x b block (the decimation's tolerance scale, kept on the device)
__global__ void __launch_bounds__(256) k_max_modulus(const cx<double>* X, long n, double* out) {
  double m = 0.0;
  for (long idx = threadIdx.x; idx < n; idx += blockDim.x) m = fmax(m, hypot(X[idx].re, X[idx].im));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  __shared__ double red[8];
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < 8; ++i) m = fmax(m, red[i]);
    out[0] = m;
  }
}
cudaError_t max_modulus(const cx<double>* X, long n, double* out, cudaStream_t st) {
  k_max_modulus<<<1, 256, 0, st>>>(X, n, out);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_fill_int(int* p, int v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
cudaError_t fill_int(int* p, int v, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_fill_int<<<(n + 255) / 256, 256, 0, st>>>(p, v, n);
  count_launch();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_decim_converged(const cx<double>* X, const cx<double>* Y, int b,
                                                         double tol_rel, const double* scale, int* active,
                                                         int* sweeps) {
  const int e = blockIdx.x;
  if (!active[e]) return;
  const double tol = tol_rel * (*scale > 0.0 ? *scale : 1.0);
  const long bb = (long)b * b;
  double m = 0.0;
  for (long idx = threadIdx.x; idx < bb; idx += blockDim.x) {
    const cx<double> x = X[(long)e * bb + idx], y = Y[(long)e * bb + idx];
    m = fmax(m, fmax(hypot(x.re, x.im), hypot(y.re, y.im)));
  }
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  __shared__ double red[8];
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)blockDim.x / 32; ++i) m = fmax(m, red[i]);
    m = fmax(m, red[0]);
    sweeps[e] += 1;
    if (m < tol) active[e] = 0;
  }
}
cudaError_t decim_converged(const cx<double>* X, const cx<double>* Y, int b, double tol_rel, const double* scale,
                            int* active, int* sweeps, int batch, cudaStream_t st) {
  k_decim_converged<<<batch, 256, 0, st>>>(X, Y, b, tol_rel, scale, active, sweeps);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_flag_active(const int* active, int* status, int code, int batch) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < batch && active[e]) atomicCAS(status + e, 0, code);
}
cudaError_t flag_active(const int* active, int* status, int code, int batch, cudaStream_t st) {
  k_flag_active<<<(batch + 127) / 128, 128, 0, st>>>(active, status, code, batch);
  count_launch();
  return cudaGetLastError();
}

// ============================================================================ integration
__global__ void k_integrate_add(double* acc, const double* val, long ld, int n, const double* w,
                                const double* E, int e0, int nE, int batch, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int e = 0; e < batch; ++e) {
    double we;
    const int g = e0 + e;
    if (w) we = w[g];
    else {
      we = 0.0;
      if (g + 1 < nE) we += 0.5 * (E[g + 1] - E[g]);
      if (g > 0) we += 0.5 * (E[g] - E[g - 1]);
    }
    s += we * val[(long)e * ld + i];
  }
  acc[i] += scale * s;
}
cudaError_t integrate_add(double* acc, const double* val, long ld, int n, const double* w,
                          const double* E, int e0, int nE, int batch, double scale, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_integrate_add<<<(n + 127) / 128, 128, 0, st>>>(acc, val, ld, n, w, E, e0, nE, batch, scale);
  count_launch();
  return cudaGetLastError();
}

}  // namespace qtx
