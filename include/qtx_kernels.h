/*
 * qtx_kernels.h -- component-level C ABI of the RGF library: the three building blocks of the sweep
 * exposed on their own, on complex128 device arrays, for testing and for callers that assemble their
 * own solvers.  Same conventions as qtx_rgf.h: device pointers owned by the caller, interleaved
 * (re, im) doubles, row-major blocks, asynchronous on `stream` (a cudaStream_t), status codes from
 * qtx_status.  Each call allocates its temporaries with stream-ordered cudaMallocAsync and frees them
 * before returning.  Nothing falls back to the CPU.
 */
#ifndef QTX_KERNELS_H
#define QTX_KERNELS_H

#include "qtx_rgf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Operand operations for qtx_zgemm_batched. */
enum { QTX_OP_N = 0, QTX_OP_C = 1 /* conjugate transpose */ };

/* Batched complex GEMM, the product kernel of the sweep (the paper's ZGEMM, Sec. IV):
 *     C[e] = alpha * op(A[e]) * op(B[e]) + beta * C0[e],   e = 0 .. batch-1,
 * op(A) is M x K, op(B) is K x N, C and C0 are M x N.  lda/ldb/ldc0/ldc are row strides and
 * strideA/B/C0/C batch strides in complex elements (0 shares one matrix across the batch).
 * precision: QTX_FP64 / QTX_FP32 on the CUDA cores; QTX_EMU64 / QTX_BF16X3 on the tcgen05 tensor cores
 * with 6 (7 when K > 512) / 2 bf16 digit planes per operand (Ozaki-style slicing, Sec. II-D), inputs
 * and outputs rounded to df32 (hi + lo FP32 pairs) on the way in and out; alpha and beta are applied as
 * df32 pairs as well (~48 bits: a scalar such as 0.1 adds no FP32-sized error).  C0 may be NULL when beta == 0; C may
 * alias C0 (same layout).  Errors: QTX_ERR_INVALID_ARG (sizes < 0, NULL operands),
 * QTX_ERR_UNSUPPORTED (tensor-core modes on a GPU other than sm_103), QTX_ERR_CUDA, QTX_ERR_TIMEOUT
 * (a bounded wait inside the tensor-core kernel expired; the context stays usable). */
qtx_status qtx_zgemm_batched(int precision, int M, int N, int K, int opA, const void *A, long lda,
                             long strideA, int opB, const void *B, long ldb, long strideB, double alpha,
                             double beta, const void *C0, long ldc0, long strideC0, void *C, long ldc,
                             long strideC, int batch, void *stream);

/* Batched inverse of n x n complex blocks, in place (A[e] -> A[e]^-1, batch stride strideA), as used
 * by the forward sweep (g_i = (A_i - V g U)^-1): Gauss-Jordan with partial pivoting on blocks of at
 * most 64, a 2 x 2 Schur-complement recursion above that, plus one Newton step X += X (I - A X) for
 * recursed FP32/FP64 blocks; QTX_EMU64 / QTX_BF16X3 start from the FP32 inverse and apply
 * `refine_iter` Newton sweeps with tensor-core products.  status[e] (device, may be NULL) receives
 * QTX_ERR_SINGULAR for a zero pivot. */
qtx_status qtx_zinv_batched(int precision, int n, void *A, long strideA, int batch, int refine_iter,
                            int *status, void *stream);

/* Retarded contact self-energy Sigma^R(E) = H01 g_s H01^H of a semi-infinite lead by Sancho-Rubio
 * decimation in FP64, batched over energies: H00, H01 are n x n (H01 couples a lead cell to the next
 * one away from the device), energies[n_energies] a device array, z = E + i eta.  Output
 * SigR[n_energies][n][n]; status[e] = QTX_ERR_NOT_CONVERGED when max|alpha|,|beta| did not fall below
 * tol * max|H01| within max_iter sweeps (convergence is tested on the device).  Synchronises `stream`
 * once before returning (the call's temporary plan is freed). */
qtx_status qtx_lead_self_energy(int n, const void *H00, const void *H01, const double *energies,
                                int n_energies, double eta, double tol, int max_iter, void *SigR,
                                int *status, void *stream);

/* FPX storage codec (Sec. V): byte-aligned floating-point formats of X = bits in {56, 48, 40, 32,
 * 24, 16} bits -- a sign bit, the 8-bit exponent and bias of FP32, and X - 9 significand bits
 * (FP32 itself for X = 32, bfloat16 for X = 16) -- used to store the simulation's blocks in less
 * memory.  Compression rounds each FP64 value to nearest (ties to even); values beyond the largest
 * finite one become +-inf, values below 2^-126 FP32-style subnormals, NaN the quiet-NaN code, and
 * magnitudes below `cutoff` (Sec. III's value cutoff; 0 = none) +0.  The stream of n values is the
 * concatenation of their X/8-byte little-endian codes, padded with zero codes to a multiple of 8
 * values: qtx_fpx_bytes(bits, n) = ceil(n / 8) * bits bytes.  Decompression is exact (every FPX
 * value is an FP64 value).  x, in and out are device pointers, 8-byte aligned; complex arrays are
 * passed as 2n reals.  Asynchronous on `stream`.  Errors: QTX_ERR_INVALID_ARG (bits not one of the
 * six widths, n < 0, cutoff < 0 or NaN, NULL or misaligned pointers with n > 0), QTX_ERR_CUDA. */
size_t qtx_fpx_bytes(int bits, long n);
qtx_status qtx_fpx_compress(int bits, const double *x, long n, double cutoff, void *out, void *stream);
qtx_status qtx_fpx_decompress(int bits, const void *in, long n, double *x, void *stream);

/* Test switch of the bounded device-side waits (the paper has no counterpart; it exists to test the
 * QTX_ERR_TIMEOUT path without faulting or hanging a GPU).  While enabled (enable != 0), every
 * tensor-core product launch first makes its MMA-issuing thread wait on a barrier that nothing arrives
 * at, with every wait of the launch limited to 100 us: the wait gives up before any MMA is issued,
 * the launch raises its wait flag, drains the bulk copies it has issued, frees its tensor memory and
 * returns, and the call that launched it reports QTX_ERR_TIMEOUT (qtx_zgemm_batched, or
 * qtx_rgf_status after a solve; the products' outputs are then not valid).  The context stays usable
 * and the next call after disabling the switch computes normally.  Process-wide; not for production
 * use.  Always returns QTX_OK. */
qtx_status qtx_tc_wait_test(int enable);

/* Size in bytes of the fixed device array behind qtx_zgemm_emu64_noalloc (48 MiB per GPU). */
#define QTX_NOALLOC_SCRATCH_BYTES ((size_t)48 << 20)

/* Allocation-free variant of qtx_zgemm_batched with precision QTX_EMU64 (same arguments and result,
 * same tensor-core kernels).  The paper has no counterpart: this serves callers that must not allocate
 * device memory while they run -- a latency-critical loop (cudaMalloc/cudaFree can synchronise the
 * device), a plugin or progress thread inside another runtime that owns all device memory, or a process
 * with a fixed memory budget.  All temporaries (df32 copies of A, B, C0 and of the result, the digit
 * planes and exponents, a wait flag) live in one array of QTX_NOALLOC_SCRATCH_BYTES that is part of the
 * library image; every GPU that loads the library holds it until the process exits.  No cudaMalloc,
 * cudaFree or allocating library routine is called.
 *   - The first call on each device (with that device current) resolves the array's device address
 *     with cudaGetSymbolAddress and caches it for that device's context; a call that finds another
 *     context current (after cudaDeviceReset) resolves it again.  Make the first call on a device,
 *     and the first after a reset, outside any stream capture.
 *   - On QTX_ERR_CUDA the runtime's last error has been cleared (cudaGetLastError).
 *   - Calls share the array and it keeps the last call's contents: the wait flag is cleared at the
 *     start of every call and everything else is rewritten.  Calls that overlap on the GPU (other
 *     streams, other host threads) race on it; serialise them.
 *   - The call synchronises `stream` before returning (it reads the wait flag).
 * Errors: QTX_ERR_OOM when the call needs more scratch than QTX_NOALLOC_SCRATCH_BYTES -- about
 * 16 B x (M K + K N + 2 M N) + the digit planes (6 planes x (4 M_pad K_pad + 6 N_pad K_pad) bytes with
 * M_pad = 128-multiple, N_pad = 48-multiple, K_pad = 32-multiple) per batch entry, e.g. at most 5
 * entries of 256 x 256 x 256 -- nothing is enqueued then; QTX_ERR_INVALID_ARG, QTX_ERR_UNSUPPORTED,
 * QTX_ERR_CUDA, QTX_ERR_TIMEOUT as for qtx_zgemm_batched. */
qtx_status qtx_zgemm_emu64_noalloc(int M, int N, int K, int opA, const void *A, long lda, long strideA,
                                   int opB, const void *B, long ldb, long strideB, double alpha,
                                   double beta, const void *C0, long ldc0, long strideC0, void *C,
                                   long ldc, long strideC, int batch, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* QTX_KERNELS_H */
