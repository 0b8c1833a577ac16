// Allocation-free variant of the batched emulated-FP64 complex GEMM (qtx_zgemm_emu64_noalloc).
//
// Who needs it: callers that must not allocate device memory while they run -- e.g. code inside a
// real-time or latency-critical loop (cudaMalloc/cudaFree can synchronise the device), a plugin or
// progress thread hosted by another runtime that owns all device allocations, or a process whose
// memory budget is fixed up front.  qtx_zgemm_batched allocates its temporaries with cudaMallocAsync;
// this entry point instead keeps every temporary (df32 copies of the operands and of the result, the
// digit planes and their exponents, the wait flag) in one fixed device array that is part of the
// library image.  Every GPU that loads the library holds that array until the process exits.
//
// Set-up: a __device__ array's name in host code is only a host-side stand-in, not a device address.
// The first call on each device, with that device current, resolves the real address with
// cudaGetSymbolAddress (checked) and caches it per device together with the id of the context it
// belongs to; later calls reuse it while the device's current context is the same one (after
// cudaDeviceReset the runtime makes a new context, and the next call resolves the address again).
// Make the first call on a device, and the first after a reset, outside any stream capture.
//
// Sharing: all calls share the one array and it keeps the last call's contents.  The wait flag is
// cleared (cudaMemsetAsync) at the start of each call; everything else is fully rewritten.  Calls that
// overlap on the GPU (different streams, or different host threads without ordering) race on the
// array and must be serialised by the caller.
#include <cuda.h>

#include <mutex>

#include "../../include/qtx_kernels.h"
#include "kernels.cuh"

using namespace qtx;

namespace {

constexpr size_t kNoAllocBytes = QTX_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
unsigned long long g_ctx[kMaxDevices] = {};  // id of the context g_addr[dev] was resolved in

// Id of the current context (0 if none is current or the driver cannot say).  The two driver
// functions are looked up through the runtime, so the library has no link-time dependency on the
// driver library (it still loads on a machine without a GPU driver).
unsigned long long current_ctx_id() {
  typedef CUresult (*get_current_t)(CUcontext*);
  typedef CUresult (*get_id_t)(CUcontext, unsigned long long*);
  static get_current_t get_current = nullptr;
  static get_id_t get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult r1, r2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &r1) == cudaSuccess &&
        r1 == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<get_current_t>(f1);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &r2) == cudaSuccess &&
        r2 == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<get_id_t>(f2);
    cudaGetLastError();
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of the temporaries inside the fixed array for one call.
struct Carve {
  size_t flag, a, b, c0, c, tc, total;
};
Carve carve(int M, int N, int K, int batch, int nA, int nB, int nC0, int rA, int cA, int rB, int cB) {
  Carve c{};
  size_t off = 0;
  const size_t es = sizeof(cx<df>);
  c.flag = off; off = al256(off + sizeof(int));
  c.a = off; off = al256(off + es * (size_t)nA * rA * cA);
  c.b = off; off = al256(off + es * (size_t)nB * rB * cB);
  c.c0 = off; off = al256(off + es * (size_t)nC0 * M * N);
  c.c = off; off = al256(off + es * (size_t)batch * M * N);
  c.tc = off; off = al256(off + gemm_tc_scratch_bytes(M, N, K, batch, 6));
  c.total = off;
  return c;
}

}  // namespace

extern "C" {

qtx_status qtx_zgemm_emu64_noalloc(int M, int N, int K, int opA, const void* A, long lda, long sA, int opB,
                                   const void* B, long ldb, long sB, double alpha, double beta, const void* C0,
                                   long ldc0, long sC0, void* C, long ldc, long sC, int batch, void* stream) {
  if (M < 0 || N < 0 || K < 0 || batch < 1 || !A || !B || !C || (beta != 0.0 && !C0) ||
      (opA != QTX_OP_N && opA != QTX_OP_C) || (opB != QTX_OP_N && opB != QTX_OP_C))
    return QTX_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return QTX_OK;
  if (!tc_available()) return QTX_ERR_UNSUPPORTED;
  const int rA = opA == QTX_OP_N ? M : K, cA = opA == QTX_OP_N ? K : M;
  const int rB = opB == QTX_OP_N ? K : N, cB = opB == QTX_OP_N ? N : K;
  const int nA = sA ? batch : 1, nB = sB ? batch : 1, nC0 = (C0 && beta != 0.0) ? (sC0 ? batch : 1) : 0;
  const Carve cv = carve(M, N, K, batch, nA, nB, nC0, rA, cA, rB, cB);
  // the request must fit the fixed array: otherwise nothing is enqueued
  if (cv.total > kNoAllocBytes) return QTX_ERR_OOM;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QTX_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long ctx = current_ctx_id();
    if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the context current
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        g_addr[dev] = nullptr;
        return QTX_ERR_CUDA;
      }
      g_addr[dev] = p;
      g_ctx[dev] = current_ctx_id();
    }
    base = reinterpret_cast<unsigned char*>(g_addr[dev]);
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* flag = reinterpret_cast<int*>(base + cv.flag);
  cx<df>* a = reinterpret_cast<cx<df>*>(base + cv.a);
  cx<df>* b = reinterpret_cast<cx<df>*>(base + cv.b);
  cx<df>* c0 = reinterpret_cast<cx<df>*>(base + cv.c0);
  cx<df>* c = reinterpret_cast<cx<df>*>(base + cv.c);
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = convert_strided<double, df>((const cx<double>*)A, lda, sA, a, cA, (long)rA * cA, rA, cA, nA, st);
  if (e == cudaSuccess)
    e = convert_strided<double, df>((const cx<double>*)B, ldb, sB, b, cB, (long)rB * cB, rB, cB, nB, st);
  if (e == cudaSuccess && nC0)
    e = convert_strided<double, df>((const cx<double>*)C0, ldc0, sC0, c0, N, (long)M * N, M, N, nC0, st);
  if (e == cudaSuccess) {
    TcArgs t;
    t.M = M; t.N = N; t.K = K;
    t.A = a; t.lda = cA; t.sA = nA > 1 ? (long)rA * cA : 0; t.opA = opA;
    t.B = b; t.ldb = cB; t.sB = nB > 1 ? (long)rB * cB : 0; t.opB = opB;
    t.C0 = nC0 ? c0 : nullptr; t.ldc0 = N; t.sC0 = nC0 > 1 ? (long)M * N : 0;
    t.C = c; t.ldc = N; t.sC = (long)M * N;
    t.alpha = alpha; t.beta = nC0 ? beta : 0.0;
    t.batch = batch; t.active = nullptr;
    e = gemm_tc(t, 6, base + cv.tc, kNoAllocBytes - cv.tc, flag, st);
  }
  if (e == cudaSuccess)
    e = convert_strided<df, double>(c, N, (long)M * N, (cx<double>*)C, ldc, sC, M, N, batch, st);
  int hflag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();  // leave no error pending in the runtime for the caller's next call
    return QTX_ERR_CUDA;
  }
  if (hflag) return QTX_ERR_TIMEOUT;
  return QTX_OK;
}

}  // extern "C"
