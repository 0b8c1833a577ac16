// Launchers of the SIMT kernels (simt.cu) and of the tensor-core engine (tc_engine.cu), called by the
// host orchestration (rgf.cu).  All launchers are asynchronous on `st` and return the launch status.
#pragma once
#include <atomic>

#include "common.cuh"

namespace qtx {

// Running count of kernel launches issued by this library (read by qtx_kernel_launches()).
extern std::atomic<long long> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---- batched complex GEMM on the CUDA cores (T = double: DFMA, T = float: FFMA)
template <typename T>
cudaError_t gemm_simt(const GemmArgs<T>& g, cudaStream_t st);

// ---- in-place inverse of n x n blocks (n <= kLeafMax) by Gauss-Jordan elimination with partial
// (row) pivoting, one CTA per block.  A zero pivot stores QTX_ERR_SINGULAR into status[e].
constexpr int kLeafMax = 64;
template <typename T>
cudaError_t leaf_inverse(cx<T>* A, long lda, long sA, int n, int batch, const int* active,
                         int* status, cudaStream_t st);

// ---- elementwise combination of b x b blocks (batched over energies):
//   out[e] = sum_t alpha_t * op_t(X_t[e])  +  diag_coef * (E[e] + i eta) * I
// op_t = OP_N or OP_C (conjugate transpose).  Up to 3 terms; a term with p == nullptr is skipped.
template <typename T>
struct Term {
  const cx<T>* p = nullptr;
  long s = 0;     // batch stride (complex elements); 0 shares one block
  int op = OP_N;
  double alpha = 0.0;
  // set by combine() on the host from alpha: +1 / -1 / general (with alpha rounded to FP32), so the
  // df32 and FP32 accumulations make no per-element FP64 comparisons (GB300's FP64 pipe is 1/64 rate)
  int kind = 0;
  float alpha_f = 0.f;
};
template <typename Tin, typename Tout>
cudaError_t combine(cx<Tout>* out, long sOut, Term<Tin> t0, Term<Tin> t1, Term<Tin> t2, int b,
                    int batch, const double* E, double eta, double diag_coef, const int* active,
                    cudaStream_t st);

// out[e](r, c) = in[e](r, c) converted between storage types (row strides ldi/ldo, batch si/so)
template <typename Tin, typename Tout>
cudaError_t convert_strided(const cx<Tin>* in, long ldi, long si, cx<Tout>* out, long ldo, long so, int rows,
                            int cols, int batch, cudaStream_t st);

// X[e] += I
template <typename T>
cudaError_t add_identity(cx<T>* X, long sX, int n, int batch, const int* active, cudaStream_t st);
// next[e] = active[e] (1 when active is nullptr) and ||R[e]||_F > tol, from the hi parts in FP32; a
// non-finite norm also sets status[e] = QTX_ERR_SINGULAR (status may be nullptr)
cudaError_t residual_mask(const cx<df>* R, long sR, int n, int batch, double tol, const int* active, int* next,
                          int* status, cudaStream_t st);

// ---- assemble a diagonal block of M (step 1 of the sweep), in T precision from complex128 inputs:
//   out[e] = (E[e] + i eta) S - H - SigR[e] - lead[e]     (S == nullptr => identity)
template <typename T>
cudaError_t assemble_diag(cx<T>* out, const cx<double>* H, const cx<double>* S,
                          const cx<double>* SigR, long sSig, const cx<double>* lead, long sLead,
                          const double* E, double eta, int b, int batch, cudaStream_t st);
// out[e] = c1 * X[e] + c2 * Y[e]  with complex128 inputs (Y may be nullptr), converted to T
template <typename T>
cudaError_t axpby_from64(cx<T>* out, long sOut, const cx<double>* X, long sX, double c1,
                         const cx<double>* Y, long sY, double c2, int b, int batch,
                         cudaStream_t st);
// out[e] = src + (E[e] + i eta) on the diagonal, for e < batch (src one shared block; E may be nullptr)
template <typename T>
cudaError_t broadcast_diag(cx<T>* out, long sOut, const cx<T>* src, int b, const double* E, double eta, int batch,
                           cudaStream_t st);
// off-diagonal rows of M: U[e] = z_e S_up - H_up - SRu[e],  V[e] = z_e S_up^H - H_up^H - SRl[e]
// (S_up, SRu, SRl may be nullptr; SRu/SRl advance by sSR per batch entry, 0 = shared)
template <typename T>
cudaError_t assemble_offdiag(cx<T>* U, cx<T>* V, const cx<double>* Hup, const cx<double>* Sup,
                             const double* E, double eta, int b, int batch, cudaStream_t st,
                             const cx<double>* SRu = nullptr, const cx<double>* SRl = nullptr, long sSR = 0);

// ---- observables, FP64 accumulation
// cur[e * ldcur] = 2 Re Tr[(H_up - E S_up) G^<_{i+1,i}],  G^<_{i+1,i} = -(GLu)^H.  With a device
// scratch of scratch_doubles doubles, one energy's trace may be split over several CTAs.
template <typename T>
cudaError_t obs_current(double* cur, long ldcur, const cx<double>* Hup, const cx<double>* Sup,
                        const cx<T>* GLu, long sG, const double* E, int b, int batch,
                        cudaStream_t st, double* scratch = nullptr, long scratch_doubles = 0);
// den[e * ldden] = Im Tr GL[e]
template <typename T>
cudaError_t obs_density(double* den, long ldden, const cx<T>* GL, long sG, int b, int batch,
                        cudaStream_t st);
// out[e * ld] = scale * Part(Tr[X[e] Y[e]] - Tr[Z[e] W[e]])  (Z, W may be nullptr; X, Z complex128),
// Part = Re for part == 0, Im for part == 1.
template <typename T>
cudaError_t obs_trace2(double* out, long ld, const cx<double>* X, long sX, const cx<T>* Y, long sY,
                       const cx<double>* Z, long sZ, const cx<T>* Wm, long sW, int b, int batch,
                       cudaStream_t st, int part = 0, double scale = 1.0);
// out[e * ld] = Re Tr[X[e] op(Y[e])] with op = conj-transpose-conj, i.e. sum_jk X_jk conj(Y_jk),
// scaled by `scale` and added to `add[e*ld]` if add != nullptr.
cudaError_t obs_frob_dot(double* out, long ld, const cx<double>* X, long sX, const cx<double>* Y,
                         long sY, double scale, int b, int batch, cudaStream_t st);

// out[e * ld] = J = Re Tr[Sigma^< G^>] - Re Tr[Sigma^> G^<] of one slice (G^> = G^< + G - G^H,
// Sigma^> = Sigma^< + Sigma^R - Sigma^R^H - 2 i eta I; SL, SR complex128 or null, batch stride sSig);
// scale[e * ld] = the absolute sum of its terms plus, with GLu = G^<_{i,i+1} given, that of the
// interface's current (Hu, Su: H_{i,i+1}, S_{i,i+1} or null; E the energies); gn[e * ld] = ||G_ii||_F^2,
// hn[e * ld] = ||H_ii||_F + 2 ||H_{i,i+1}||_F (Hd = H_ii)
template <typename T>
cudaError_t obs_balance(double* out, double* scale, double* gn, double* hn, long ld, const cx<double>* SL,
                        const cx<double>* SR, long sSig, const cx<T>* G, const cx<T>* GL, long sG, double eta, int b,
                        int batch, cudaStream_t st, const cx<double>* Hd, const cx<double>* Hu, const cx<double>* Su,
                        const double* E, const cx<T>* GLu);
// res[e] = max_i |I_{i-1} + J_i - I_i| / max_i scale_i per energy (con: [ne][2] contact currents or
// null); flag[e] = !(res[e] < tol) or !(kappa_est eps_mode < tol), kappa_est = (|E| + max hn) sqrt(max gn)
cudaError_t continuity(const double* cur, long ldc, const double* J, const double* Js, const double* gn,
                       const double* hn, long ldj, const double* con, const double* E, int nb, int ne, double tol,
                       double eps_mode, double* res, int* flag, cudaStream_t st);

// ---- lead post-processing: from Sigma^R (complex128) build Gamma, Sigma^<, Sigma^>
cudaError_t lead_sigmas(const cx<double>* SR, cx<double>* Gam, cx<double>* SL, cx<double>* SG,
                        const double* E, double mu, double kT, int b, int batch, cudaStream_t st);
// per batch entry: if the largest modulus over X and Y is < tol_rel * max(*scale, or 1 if 0), clear
// active[e]; count sweeps (scale is a device scalar, e.g. from max_modulus)
cudaError_t decim_converged(const cx<double>* X, const cx<double>* Y, int b, double tol_rel,
                            const double* scale, int* active, int* sweeps, int batch, cudaStream_t st);
// out[0] = largest modulus of the n complex values X[0..n) (device scalar)
cudaError_t max_modulus(const cx<double>* X, long n, double* out, cudaStream_t st);
// p[0..n) = v
cudaError_t fill_int(int* p, int v, int n, cudaStream_t st);
// The whole decimation of a lead block of size n <= kDecimSmallMax per energy in one CTA (decim.cu):
// SR[e] = H01 g_s(E[e] + i eta) H01^H; status[e] = QTX_ERR_NOT_CONVERGED / QTX_ERR_SINGULAR (only
// raised from 0).  No host synchronisation.
constexpr int kDecimSmallMax = 32;
cudaError_t decimate_small(const cx<double>* H00, const cx<double>* H01, const double* E, double eta,
                           double tol_rel, int max_iter, int n, int batch, cx<double>* SR, int* status,
                           cudaStream_t st);
// set status[e] = code for entries still active (decimation not converged)
cudaError_t flag_active(const int* active, int* status, int code, int batch, cudaStream_t st);

// ---- energy integration: acc[i] += scale * sum_{e<batch} w[e] * val[e * ld + i]
//      (w == nullptr: trapezoid weights of the full grid E[0..nE), entries e0 .. e0+batch)
cudaError_t integrate_add(double* acc, const double* val, long ld, int n, const double* w,
                          const double* E, int e0, int nE, int batch, double scale,
                          cudaStream_t st);

// ---- tensor-core engine (tc_engine.cu): emulated-precision batched complex GEMM on sm_103a.
// `digits` bf16 digit planes per operand (6: ~41-bit products from 21 digit products, 7 of them
// taken for K > 512; 2: ~13-bit products from 3; 4 with a.f32: ~27-bit products from 10 for FP32
// operands and results).  `scratch` holds the digit planes and scale exponents.
// `ev` (optional, two events) brackets the tensor-core GEMM kernel itself (not the digitiser).
cudaError_t gemm_tc(const TcArgs& a, int digits, void* scratch, size_t scratch_bytes, int* err_flag,
                    cudaStream_t st, cudaEvent_t* ev = nullptr);
// Kernel parameters of one tensor-core product (filled by gemm_tc_prepare).
struct TcParams {
  const unsigned char* pa;  // A plane tiles [batch'][S][M_pad/128][nks][128 x 32 B]
  const unsigned char* pb;  // B plane sub-tiles [batch'][S][N_pad/48][K_pad/16][3][48 x 32 B]: Re, Im, -Im
  const int* eA;   // [batch][M_pad] row exponents of op(A)
  const int* eB;   // [batch][N_pad] column exponents of op(B)
  int M_pad, N_pad, nks;  // nks: K-stages of 16 over the embedded K (2 * K_pad)
  int M, N;
  int bn_last;     // complex columns the last column tile computes: N - 48 (NBt - 1), rounded up to 8
  void* C; long ldc, sC;         // cx<df>, or cx<float> for the FP32 products
  const void* C0; long ldc0, sC0;
  df alpha, beta;  // as df32 pairs; the kinds say how they enter the epilogue:
  int akind;       //   alpha: 0 = +1, 1 = -1, 2 = general (df32 product)
  int bkind;       //   beta:  0 = +1, 1 = -1, 2 = general, 3 = no beta * C0 term
  int escale;      // exponent shift of the recombined sum: 2 l1 - 2
  int a_batched, b_batched;  // 0: the operand is shared by the whole batch (digitized once)
  const int* active;
  int* err;
};
// A product whose operands are digitised (on the preparing stream) and whose kernel parameters are
// filled, ready to launch alone or with other products of the same variant.
struct TcPrepared {
  int variant = -1;  // gemm_tc_variant
  int ctas = 0;      // persistent CTAs of its launch (0 = one per SM)
  int NBt = 0, MBt = 0;
  long tiles = 0;    // output tiles: column tiles x row tiles x batch
  TcParams p{};
};
// Kernel variant of a product: digits used, IO type and pipeline stages; -1 for products split along K.
int gemm_tc_variant(const TcArgs& a, int digits);
// Digitise a product's operands on `st` (not one split along K) and fill *out.
cudaError_t gemm_tc_prepare(const TcArgs& a, int digits, void* scratch, size_t scratch_bytes, int* err_flag,
                            cudaStream_t st, TcPrepared* out);
// One persistent launch over the tiles of 1..kTcMaxGroup prepared products of one variant (each
// product's tiles computed exactly as in a launch of its own: the results are bit-identical).
constexpr int kTcMaxGroup = 8;
cudaError_t gemm_tc_launch(const TcPrepared* const* p, int n, cudaStream_t st, cudaEvent_t* ev = nullptr);
// digit products (pairs i + j <= digits + 1) the engine issues per real product
inline int tc_pairs(int digits) { return digits * (digits + 1) / 2; }
size_t gemm_tc_scratch_bytes(int M, int N, int K, int batch, int digits);
// Bytes of a TcOperand for op(A) (side 0, R = M rows) or op(B) (side 1, R = N columns) of K; 0 when
// the product would be split along K (operands cannot be kept then).  tc_operand_at carves one.
size_t gemm_tc_operand_bytes(int side, int R, int K, int batch, int digits);
TcOperand tc_operand_at(void* base, int side, int R, int K, int batch, int digits);
bool tc_available();

// ---- FPX storage codec (fpx.cu): n_complex T-typed complex values <-> their FPX codes
bool fpx_width_ok(int bits);
size_t fpx_bytes(int bits, long n_reals);
template <typename T>
cudaError_t fpx_store(int bits, const cx<T>* x, long n_complex, void* out, cudaStream_t st);
template <typename T>
cudaError_t fpx_load(int bits, const void* in, long n_complex, cx<T>* x, cudaStream_t st);

}  // namespace qtx
