// Contact self-energies by Sancho-Rubio decimation (Lopez Sancho et al., J. Phys. F 15, 851 (1985)),
// FP64, without host synchronisation.
//
// For a lead with principal layer H00 and coupling H01 (from a lead cell to the next one away from
// the device), per energy z = E + i eta:
//     alpha = H01, beta = H01^H, eps = eps_s = H00;
//     repeat:  g = (z - eps)^-1
//              eps_s += alpha g beta,  eps += alpha g beta + beta g alpha,
//              alpha = alpha g alpha,  beta = beta g beta
//     until max |alpha|, |beta| < tol max |H01|;  then g_s = (z - eps_s)^-1 and
//     Sigma^R = H01 g_s H01^H  (the device's end slice couples to the first lead cell by H01).
//
// k_decimate: the whole iteration of one energy in one CTA, every block in shared memory (b <= 32:
// eight b x b complex128 blocks, at most 128 KB).  The inverses are in-place Gauss-Jordan elimination
// with partial (row) pivoting on |re| + |im| (first maximum on ties), the row interchanges undone as
// column interchanges at the end.  The sweep count, the convergence test and the status are kept on
// the device: a contact costs one launch, and a solve with contacts makes no host synchronisation
// (so it can be captured in a CUDA graph).
#include "kernels.cuh"

namespace qtx {

namespace {

constexpr int kDecThreads = 256;

// C = A B for n x n blocks in shared memory with row stride NM (all threads; the caller syncs)
template <int NM>
__device__ __forceinline__ void mm_s(const cx<double>* A, const cx<double>* B, cx<double>* C, int n) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx % n;
    cx<double> acc = mk<double>(0.0, 0.0);
    for (int k = 0; k < n; ++k) cfma(acc, A[r * NM + k], B[k * NM + c]);
    C[r * NM + c] = acc;
  }
}

// In-place inverse of the n x n block A (row stride NM) by Gauss-Jordan elimination with partial
// pivoting.  colk[NM] and perm[NM] are shared scratch.  Returns false (uniformly) for a zero pivot.
template <int NM>
__device__ bool inv_s(cx<double>* A, int n, cx<double>* colk, int* perm, int* s_piv) {
  const int t = threadIdx.x;
  for (int k = 0; k < n; ++k) {
    if (t < 32) {
      double best = -1.0;
      int bi = -1;
      for (int i = k + t; i < n; i += 32) {
        const double v = cabs1(A[i * NM + k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi >= 0 && (bi < 0 || oi < bi))) {
          best = ov;
          bi = oi;
        }
      }
      if (t == 0) {
        *s_piv = best > 0.0 ? bi : -1;
        perm[k] = bi;
      }
    }
    __syncthreads();
    const int p = *s_piv;
    if (p < 0) return false;
    if (p != k)
      for (int j = t; j < n; j += blockDim.x) {
        const cx<double> x = A[k * NM + j];
        A[k * NM + j] = A[p * NM + j];
        A[p * NM + j] = x;
      }
    __syncthreads();
    const cx<double> r = crecip(A[k * NM + k]);
    for (int i = t; i < n; i += blockDim.x) colk[i] = A[i * NM + k];
    __syncthreads();
    for (int j = t; j < n; j += blockDim.x) A[k * NM + j] = (j == k) ? r : A[k * NM + j] * r;
    __syncthreads();
    for (int idx = t; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx % n;
      if (i == k) continue;
      const cx<double> f = colk[i];
      if (j == k) A[i * NM + k] = mk<double>(0.0, 0.0) - f * r;
      else A[i * NM + j] = A[i * NM + j] - f * A[k * NM + j];
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = t; i < n; i += blockDim.x) {
        const cx<double> x = A[i * NM + k];
        A[i * NM + k] = A[i * NM + p];
        A[i * NM + p] = x;
      }
    __syncthreads();
  }
  return true;
}

// largest modulus over the n x n blocks X and Y (all threads get it)
template <int NM>
__device__ double max_mod2(const cx<double>* X, const cx<double>* Y, int n, double* red) {
  double m = 0.0;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx % n;
    const cx<double> x = X[r * NM + c], y = Y[r * NM + c];
    m = fmax(m, fmax(hypot(x.re, x.im), hypot(y.re, y.im)));
  }
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < (int)blockDim.x / 32; ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

template <int NM>
__global__ void __launch_bounds__(kDecThreads) k_decimate(const cx<double>* H00, const cx<double>* H01,
                                                         const double* E, double eta, double tol_rel,
                                                         int max_iter, int n, cx<double>* SR, int* status) {
  extern __shared__ __align__(16) unsigned char dsm[];
  cx<double>* al = reinterpret_cast<cx<double>*>(dsm);
  cx<double>* be = al + NM * NM;
  cx<double>* ep = be + NM * NM;
  cx<double>* es = ep + NM * NM;
  cx<double>* G = es + NM * NM;
  cx<double>* AG = G + NM * NM;
  cx<double>* BG = AG + NM * NM;
  cx<double>* T = BG + NM * NM;
  cx<double>* colk = T + NM * NM;
  __shared__ int perm[NM];
  __shared__ int s_piv;
  __shared__ double red[kDecThreads / 32];
  const int e = blockIdx.x, t = threadIdx.x;
  const cx<double> z = mk<double>(E[e], eta);
  for (int idx = t; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx % n;
    al[r * NM + c] = H01[idx];
    be[r * NM + c] = conj(H01[(long)c * n + r]);
    ep[r * NM + c] = H00[idx];
    es[r * NM + c] = H00[idx];
  }
  __syncthreads();
  // tolerance relative to the coupling's largest modulus (al holds H01, be its adjoint)
  double scale = max_mod2<NM>(al, al, n, red);
  const double tol = tol_rel * (scale > 0.0 ? scale : 1.0);
  bool converged = false, singular = false;
  for (int it = 1; it <= max_iter; ++it) {
    for (int idx = t; idx < n * n; idx += blockDim.x) {
      const int r = idx / n, c = idx % n;
      const cx<double> x = ep[r * NM + c];
      G[r * NM + c] = mk<double>((r == c ? z.re : 0.0) - x.re, (r == c ? z.im : 0.0) - x.im);
    }
    __syncthreads();
    if (!inv_s<NM>(G, n, colk, perm, &s_piv)) {
      singular = true;
      break;
    }
    mm_s<NM>(al, G, AG, n);
    mm_s<NM>(be, G, BG, n);
    __syncthreads();
    mm_s<NM>(AG, be, T, n);  // alpha g beta
    __syncthreads();
    for (int idx = t; idx < n * n; idx += blockDim.x) {
      const int r = idx / n, c = idx % n;
      es[r * NM + c] = es[r * NM + c] + T[r * NM + c];
      ep[r * NM + c] = ep[r * NM + c] + T[r * NM + c];
    }
    __syncthreads();
    mm_s<NM>(BG, al, T, n);  // beta g alpha
    __syncthreads();
    for (int idx = t; idx < n * n; idx += blockDim.x) {
      const int r = idx / n, c = idx % n;
      ep[r * NM + c] = ep[r * NM + c] + T[r * NM + c];
    }
    __syncthreads();
    mm_s<NM>(AG, al, T, n);  // alpha g alpha
    mm_s<NM>(BG, be, G, n);  // beta g beta (G is free now)
    __syncthreads();
    for (int idx = t; idx < n * n; idx += blockDim.x) {
      const int r = idx / n, c = idx % n;
      al[r * NM + c] = T[r * NM + c];
      be[r * NM + c] = G[r * NM + c];
    }
    __syncthreads();
    if (max_mod2<NM>(al, be, n, red) < tol) {
      converged = true;
      break;
    }
  }
  int st = 0;
  if (singular) st = (int)QTX_ERR_SINGULAR;
  else if (!converged) st = (int)QTX_ERR_NOT_CONVERGED;
  // g_s = (z - eps_s)^-1 (also after a capped iteration, as the launched path does)
  if (!singular) {
    for (int idx = t; idx < n * n; idx += blockDim.x) {
      const int r = idx / n, c = idx % n;
      const cx<double> x = es[r * NM + c];
      G[r * NM + c] = mk<double>((r == c ? z.re : 0.0) - x.re, (r == c ? z.im : 0.0) - x.im);
      al[r * NM + c] = H01[idx];
      be[r * NM + c] = conj(H01[(long)c * n + r]);
    }
    __syncthreads();
    if (!inv_s<NM>(G, n, colk, perm, &s_piv)) singular = true;
  }
  cx<double>* out = SR + (long)e * n * n;
  if (singular) {
    st = (int)QTX_ERR_SINGULAR;
    for (int idx = t; idx < n * n; idx += blockDim.x) out[idx] = mk<double>(0.0, 0.0);
  } else {
    mm_s<NM>(al, G, T, n);  // H01 g_s
    __syncthreads();
    mm_s<NM>(T, be, AG, n);  // (H01 g_s) H01^H
    __syncthreads();
    for (int idx = t; idx < n * n; idx += blockDim.x) out[idx] = AG[(idx / n) * NM + idx % n];
  }
  if (t == 0 && st && status) atomicCAS(status + e, 0, st);
}

template <int NM>
constexpr size_t decim_smem() {
  return (size_t)(8 * NM * NM + NM) * sizeof(cx<double>);
}

}  // namespace

cudaError_t decimate_small(const cx<double>* H00, const cx<double>* H01, const double* E, double eta,
                           double tol_rel, int max_iter, int n, int batch, cx<double>* SR, int* status,
                           cudaStream_t st) {
  if (n < 1 || n > kDecimSmallMax) return cudaErrorInvalidValue;
  if (n <= 16) {
    k_decimate<16><<<batch, kDecThreads, decim_smem<16>(), st>>>(H00, H01, E, eta, tol_rel, max_iter, n, SR, status);
  } else {
    static bool attr = false;
    if (!attr) {
      const cudaError_t e = cudaFuncSetAttribute(k_decimate<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)decim_smem<32>());
      if (e != cudaSuccess) return e;
      attr = true;
    }
    k_decimate<32><<<batch, kDecThreads, decim_smem<32>(), st>>>(H00, H01, E, eta, tol_rel, max_iter, n, SR, status);
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace qtx
