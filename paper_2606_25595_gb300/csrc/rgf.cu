// Host orchestration and C ABI of the RGF selected inversion (declared in include/qtx_rgf.h).
//
// Per chunk of energies (all kernels batched over the chunk, one stream):
//   1. contacts: Sancho-Rubio decimation in FP64 -> Sigma^R_L,R, Gamma, Sigma^<, Sigma^>
//   2. forward sweep i = 0..N_B-1:  g_i = (A_i - V_{i-1} g_{i-1} U_{i-1})^-1,
//                                   g^<_i = g_i (Sigma^<_i + V_{i-1} g^<_{i-1} V_{i-1}^H) g_i^H
//   3. backward sweep i = N_B-2..0 for G^R, G^< blocks (formulas at `backward`), G^> = G^< + G^R - G^A
//   4. FP64 observables and their energy integrals.
// The sweep is the block Gaussian elimination of the paper's Sec. IV-A applied to Eq. 2 (Table I,
// G-row); the block inverse is a recursive 2 x 2 Schur-complement inversion over leaf blocks of at
// most 64 that are inverted with partial pivoting.  Elimination without pivoting between blocks is
// safe here for the same reason it is safe between slices: the anti-Hermitian part of M,
// eta S + Gamma/2, is positive definite, so every leading principal block and every Schur
// complement is nonsingular.
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/qtx_kernels.h"
#include "kernels.cuh"

using namespace qtx;

namespace {
thread_local std::string g_create_error;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Byte-offset allocator for the single workspace allocation.
struct Arena {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  }
};

// U_i, V_i differ per energy when z multiplies an overlap block or Sigma^R_{i,i+1} depends on E.
inline bool uv_per_energy(const qtx_rgf_desc& d) {
  return d.has_S || d.system_input || (d.offdiag_sigma && d.energy_dependent_sigma);
}

struct Layout {
  size_t g, gl, gl2, zk, xk, gfx, glfx, fx_slot, sig_stage, opnd[3], opnd_bytes[3], refine_act, tmp, inv_tmp, U, V, ident, ident_df, shared_blk, ref, f32a, f32tmp, dec, lead, obs, flags, dscale, bal, bscale, bgn, bhn, cres, cflag,
      tc_scratch, total;
  int n_tmp, n_dec;
  size_t tc_bytes;
};
}  // namespace

struct qtx_rgf_group_s;

struct qtx_rgf_plan_s {
  qtx_rgf_desc d{};
  qtx_rgf_group_s* group = nullptr;  // set while the plan solves as a member of a group
  int member = -1;
  int b = 0, nb = 0, Ec = 0;
  long bb = 0;
  size_t esz = 0;  // bytes per complex element of the sweep workspace
  Layout L{};
  unsigned char* ws = nullptr;
  std::string err;
  cudaStream_t last = nullptr;
  int* d_err_flag = nullptr;    // tensor-core engine wait/limit flag
  int worst = 0;                // worst per-energy status after the last synchronising call
  int* h_status = nullptr;      // pinned host copy of the chunk status
  int* h_flag = nullptr;        // pinned host copy of the chunk's escalation flags
  std::vector<int> status_host;
  const int* out_status = nullptr;  // caller's per-energy status array of the last solve
  int out_status_n = 0;
  // GEMM profiling (qtx_rgf_set_profiling): event pairs around each product-kernel launch
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  double pipe_flops = 0.0, useful_flops = 0.0;
  cudaEvent_t* next_events() {
    if (ev_used + 2 > ev_pool.size()) {
      for (int k = 0; k < 256; ++k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ev_pool.push_back(e);
      }
    }
    cudaEvent_t* r = &ev_pool[ev_used];
    ev_used += 2;
    return r;
  }
};

namespace {

Layout make_layout(const qtx_rgf_desc& d) {
  Layout L{};
  const long b = d.block_size, nb = d.n_blocks, Ec = d.max_energies_in_flight;
  const size_t bb = (size_t)b * b;
  // FP32 plans that escalate energies to FP64 lay out complex128 blocks (the FP64 re-solve runs on
  // the same workspace); df32 blocks are complex128-sized anyway
  const size_t es = (d.precision == QTX_FP32 && !(d.escalate_tol > 0)) ? sizeof(cx<float>) : sizeof(cx<double>);
  Arena a;
  // 12, 13: Sigma^<_{i,i+1} in the sweep's type and g_i Sigma^<_{i,i+1}; 14: g_i B2_{i,i+1} (second_rhs)
  L.n_tmp = d.offdiag_sigma ? (d.second_rhs ? 15 : 14) : 12;
  if (d.storage_bits) {
    // two working blocks per kind in the sweep's type (slices i and i-1 / i+1), every slice's
    // left-connected blocks in FPX: a slot of fx_slot bytes per slice and kind
    L.g = a.take(2 * Ec * bb * es);
    L.gl = a.take(2 * Ec * bb * es);
    L.fx_slot = fpx_bytes(d.storage_bits, 2 * Ec * bb);
    L.gfx = a.take(nb * L.fx_slot);
    L.glfx = a.take(nb * L.fx_slot);
  } else {
    L.g = a.take(nb * Ec * bb * es);
    L.gl = a.take(nb * Ec * bb * es);
  }
  L.gl2 = a.take(d.second_rhs ? nb * Ec * bb * es : 0);  // left-connected blocks of the second right-hand side
  // Z_i = V_i g_i of every slice but the last, formed in the forward sweep and kept for the
  // backward one (without FPX storage, whose point is to keep fewer full blocks)
  L.zk = a.take(!d.storage_bits && nb > 1 ? (nb - 1) * Ec * bb * es : 0);
  // and X_i = V_i g^<_i of every right-hand side, the backward sweep's Q_i
  L.xk = a.take(!d.storage_bits && nb > 1 ? (size_t)(d.second_rhs ? 2 : 1) * (nb - 1) * Ec * bb * es : 0);
  L.tmp = a.take((size_t)L.n_tmp * Ec * bb * es);
  L.sig_stage = a.take(d.sigma_stream ? 2 * Ec * bb * sizeof(cx<double>) : 0);  // Sigma^R_ii, Sigma^<_ii
  L.inv_tmp = a.take(Ec * bb * es + 4096);
  const size_t ou = uv_per_energy(d) ? (size_t)(nb > 1 ? nb - 1 : 0) * Ec * bb * es : (size_t)(nb > 1 ? nb - 1 : 0) * bb * es;
  L.U = a.take(ou);
  L.V = a.take(ou);
  L.ident = a.take(bb * sizeof(cx<double>));
  L.ident_df = a.take(bb * sizeof(cx<double>));
  // one block shared by every energy (the slice's -(H + Sigma^R) or Sigma^<, converted once)
  L.shared_blk = a.take(d.precision == QTX_FP64 ? 0 : bb * sizeof(cx<double>));
  const bool mixed = d.precision == QTX_EMU64 || d.precision == QTX_BF16X3;
  L.ref = a.take((mixed || b > kLeafMax) ? 3 * Ec * bb * sizeof(cx<double>) : 0);
  L.f32a = a.take(mixed ? Ec * bb * sizeof(cx<float>) : 0);
  L.f32tmp = a.take(mixed ? Ec * bb * sizeof(cx<float>) + 4096 : 0);
  L.n_dec = 9;
  L.dec = a.take(d.leads ? (size_t)L.n_dec * Ec * bb * sizeof(cx<double>) : 0);
  L.lead = a.take(d.leads ? 8 * Ec * bb * sizeof(cx<double>) : 0);
  // per-energy observables: current, density, contact(2), transmission, scratch(2)
  L.obs = a.take((size_t)Ec * (2 * nb + 8) * sizeof(double));
  L.flags = a.take((size_t)Ec * 3 * sizeof(int) + 64);
  L.dscale = a.take(64);  // device scalars (the decimation's tolerance scale)
  // continuity check: per-slice balances J [Ec][nb], residuals [Ec], escalation flags [Ec]
  const bool cont = (d.outputs & QTX_OUT_CONTINUITY) || d.escalate_tol > 0;
  L.bal = a.take(cont ? (size_t)Ec * nb * sizeof(double) : 0);
  L.bscale = a.take(cont ? (size_t)Ec * nb * sizeof(double) : 0);
  L.bgn = a.take(cont ? (size_t)Ec * nb * sizeof(double) : 0);
  L.bhn = a.take(cont ? (size_t)Ec * nb * sizeof(double) : 0);
  L.cres = a.take(cont ? (size_t)Ec * sizeof(double) : 0);
  L.cflag = a.take(cont ? (size_t)Ec * sizeof(int) + 64 : 0);
  L.refine_act = a.take((size_t)Ec * 2 * sizeof(int) + 64);  // per-energy sweep masks (ping-pong)
  L.tc_bytes = 0;
  if (mixed) L.tc_bytes = gemm_tc_scratch_bytes((int)b, (int)b, (int)b, (int)Ec, d.precision == QTX_EMU64 ? 6 : 2);
  if (d.precision == QTX_EMU64)  // the Newton correction's four-plane products
    L.tc_bytes = std::max(L.tc_bytes, gemm_tc_scratch_bytes((int)b, (int)b, (int)b, (int)Ec, 4));
  // the FP32 mode's products of 96 and more (four digit planes; the recursive inverse's halves too)
  if (d.precision == QTX_FP32 && b >= 96 && b <= 1024) L.tc_bytes = gemm_tc_scratch_bytes((int)b, (int)b, (int)b, (int)Ec, 4);
  L.tc_scratch = a.take(L.tc_bytes);
  // kept digitised operands (emulated modes): two left operands and one right operand, b x b, E_c
  // energies (none when the products are split along K)
  for (int k = 0; k < 3; ++k) {
    L.opnd_bytes[k] = mixed ? gemm_tc_operand_bytes(k < 2 ? 0 : 1, (int)b, (int)b, (int)Ec, d.precision == QTX_EMU64 ? 6 : 2) : 0;
    L.opnd[k] = a.take(L.opnd_bytes[k]);
  }
  L.total = a.off;
  return L;
}

const char* cuda_msg(cudaError_t e) { return cudaGetErrorString(e); }

#define QTX_CK(call)                                                      \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) {                                              \
      P->err = std::string(#call) + ": " + cuda_msg(e_);                  \
      return QTX_ERR_CUDA;                                                \
    }                                                                     \
  } while (0)

// ----------------------------------------------------------------------------- solver context
template <typename T>
struct Ctx {
  qtx_rgf_plan_s* P;
  cudaStream_t st;
  int ne;                 // energies in this chunk
  const double* E;        // device energies of this chunk
  int* status;            // device status of this chunk [ne]
  long bb;
  int b;

  cx<T>* blk(size_t base, long i) const {
    return reinterpret_cast<cx<T>*>(P->ws + base) + (size_t)i * P->Ec * bb;
  }
  cx<T>* tmp(int k) const { return blk(P->L.tmp, k); }
  // left-connected / full blocks of slice i: slot i, or with FPX storage working block i % 2
  cx<T>* g(int i) const { return blk(P->L.g, P->d.storage_bits ? i % 2 : i); }
  cx<T>* gl(int i) const { return blk(P->L.gl, P->d.storage_bits ? i % 2 : i); }
  // lesser-type blocks of right-hand side k (k = 1: second_rhs, never FPX-stored)
  cx<T>* glk(int k, int i) const { return k ? blk(P->L.gl2, i) : gl(i); }
  // Z_i = V_i g_i kept from the forward sweep (nullptr without: FPX storage or one slice)
  bool keep_z() const { return !P->d.storage_bits && P->nb > 1; }
  cx<T>* zk(int i) const { return blk(P->L.zk, i); }
  // X_i = V_i g^<_i of right-hand side k, kept from the forward sweep as the backward sweep's Q_i
  cx<T>* xk(int k, int i) const { return blk(P->L.xk, (long)k * (P->nb - 1) + i); }
  void* gfx(int i) const { return P->ws + P->L.gfx + (size_t)i * P->L.fx_slot; }
  void* glfx(int i) const { return P->ws + P->L.glfx + (size_t)i * P->L.fx_slot; }
};

template <typename T>
GemmArgs<T> gargs(int M, int N, int K, const cx<T>* A, long lda, long sA, int opA, const cx<T>* B,
                  long ldb, long sB, int opB, const cx<T>* C0, long ldc0, long sC0, cx<T>* C, long ldc,
                  long sC, double alpha, double beta, int batch, const int* active) {
  GemmArgs<T> g;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.sA = sA; g.opA = opA;
  g.B = B; g.ldb = ldb; g.sB = sB; g.opB = opB;
  g.C0 = C0; g.ldc0 = ldc0; g.sC0 = sC0;
  g.C = C; g.ldc = ldc; g.sC = sC;
  g.alpha = alpha; g.beta = beta; g.batch = batch; g.active = active;
  return g;
}

// GEMM dispatch by the plan's precision (FP32 and FP64: SIMT; EMU64 / BF16X3: tensor-core engine).
// Which kept digitised operands (tensor-core modes) a product uses: slot 0, 1 (left operands) or
// 2 (right operand), mode KEEP (digitise into the slot) or REUSE (take the slot's planes: the operand,
// its op and its shape are unchanged since the KEEP product).  Ignored by the SIMT modes.
enum { DG_NONE = 0, DG_KEEP = 1, DG_REUSE = 2 };
struct DigitHint {
  int a_slot = -1, a_mode = DG_NONE, b_slot = -1, b_mode = DG_NONE;
  int digits = 0;  // digit planes of a tensor-core product (0: the plan's)
};
inline DigitHint keepA(int slot) { DigitHint h; h.a_slot = slot; h.a_mode = DG_KEEP; return h; }
inline DigitHint reuseA(int slot) { DigitHint h; h.a_slot = slot; h.a_mode = DG_REUSE; return h; }
inline DigitHint keepB(int slot) { DigitHint h; h.b_slot = slot; h.b_mode = DG_KEEP; return h; }
inline DigitHint planes(int digits) { DigitHint h; h.digits = digits; return h; }

template <typename T>
qtx_status gemm(qtx_rgf_plan_s* P, const GemmArgs<T>& g, cudaStream_t st, bool force_simt = false,
                DigitHint hint = DigitHint{});

// A tensor-core product of a plan that solves as a group member: posted to the group, launched
// together with the other members' products (defined with the group below).
cudaError_t group_gemm(qtx_rgf_plan_s* P, const TcArgs& a, int digits, cudaStream_t st);

// The profiled product kernel is the plan's own: the SIMT GEMM in the FP64 / FP32 modes, the
// tensor-core GEMM in the emulated modes (whose FP32 starting-guess inverse also calls GEMMs -- SIMT,
// or the tensor cores' four-plane FP32 instance -- which are not counted).
template <typename T>
qtx_status gemm_simt_prof(qtx_rgf_plan_s* P, const GemmArgs<T>& g, cudaStream_t st) {
  const bool mine = P->d.precision == QTX_FP64 || P->d.precision == QTX_FP32;
  cudaEvent_t* ev = (P->prof && mine) ? P->next_events() : nullptr;
  if (ev) cudaEventRecord(ev[0], st);
  QTX_CK(gemm_simt<T>(g, st));
  if (ev) {
    cudaEventRecord(ev[1], st);
    const double f = 8.0 * g.M * g.N * g.K * g.batch;
    P->pipe_flops += f;
    P->useful_flops += f;
  }
  return QTX_OK;
}
// complex64 products (the FP32 mode, and the emulated-FP64 mode's FP32 starting inverse): those of
// at least kTcF32Min in every dimension run on the tensor cores with four digit planes (~27-bit
// products, at least FP32's precision; every digit group exact), the smaller ones on the SIMT GEMM.
constexpr int kTcF32Min = 96;
inline bool f32_on_tc(const qtx_rgf_desc& d) { return d.precision == QTX_EMU64 || d.precision == QTX_FP32; }
template <>
qtx_status gemm<float>(qtx_rgf_plan_s* P, const GemmArgs<float>& g, cudaStream_t st, bool, DigitHint) {
  if (f32_on_tc(P->d) && g.M >= kTcF32Min && g.N >= kTcF32Min && g.K >= kTcF32Min && g.K <= 1024 &&
      gemm_tc_scratch_bytes(g.M, g.N, g.K, g.batch, 4) <= P->L.tc_bytes) {
    TcArgs a;
    a.f32 = true;
    a.M = g.M; a.N = g.N; a.K = g.K;
    a.A = reinterpret_cast<const cx<df>*>(g.A); a.lda = g.lda; a.sA = g.sA; a.opA = g.opA;
    a.B = reinterpret_cast<const cx<df>*>(g.B); a.ldb = g.ldb; a.sB = g.sB; a.opB = g.opB;
    a.C0 = reinterpret_cast<const cx<df>*>(g.C0); a.ldc0 = g.ldc0; a.sC0 = g.sC0;
    a.C = reinterpret_cast<cx<df>*>(g.C); a.ldc = g.ldc; a.sC = g.sC;
    a.alpha = g.alpha; a.beta = g.beta;
    a.batch = g.batch; a.active = g.active;
    a.stages = P->d.tc_stages; a.ctas = P->d.tc_ctas;
    // in the FP32 mode these are the plan's own products (profiled); in the emulated mode they
    // belong to the starting inverse (not counted)
    if (P->group && gemm_tc_variant(a, 4) >= 0) {
      QTX_CK(group_gemm(P, a, 4, st));
      return QTX_OK;
    }
    cudaEvent_t* ev = (P->prof && P->d.precision == QTX_FP32) ? P->next_events() : nullptr;
    QTX_CK(gemm_tc(a, 4, P->ws + P->L.tc_scratch, P->L.tc_bytes, P->d_err_flag, st, ev));
    if (ev) {
      const double f = 8.0 * g.M * g.N * g.K * g.batch;
      P->pipe_flops += f * tc_pairs(4);
      P->useful_flops += f;
    }
    return QTX_OK;
  }
  return gemm_simt_prof<float>(P, g, st);
}
template <>
qtx_status gemm<double>(qtx_rgf_plan_s* P, const GemmArgs<double>& g, cudaStream_t st, bool, DigitHint) {
  return gemm_simt_prof<double>(P, g, st);
}
inline int tc_digits(const qtx_rgf_desc& d) { return d.precision == QTX_EMU64 ? 6 : 2; }
template <>
qtx_status gemm<df>(qtx_rgf_plan_s* P, const GemmArgs<df>& g, cudaStream_t st, bool, DigitHint hint) {
  TcArgs a;
  const int digits = hint.digits > 0 ? hint.digits : tc_digits(P->d);
  // kept operands: only for the plan's b x b x b products at the plan's digit count, when slots exist
  TcOperand oa, ob;
  const bool square = g.M == P->b && g.N == P->b && g.K == P->b && g.batch <= P->Ec && digits == tc_digits(P->d);
  if (square && hint.a_mode != DG_NONE && P->L.opnd_bytes[hint.a_slot]) {
    oa = tc_operand_at(P->ws + P->L.opnd[hint.a_slot], 0, P->b, P->b, P->Ec, tc_digits(P->d));
    oa.mode = hint.a_mode;
    a.opndA = &oa;
  }
  if (square && hint.b_mode != DG_NONE && P->L.opnd_bytes[hint.b_slot]) {
    ob = tc_operand_at(P->ws + P->L.opnd[hint.b_slot], 1, P->b, P->b, P->Ec, tc_digits(P->d));
    ob.mode = hint.b_mode;
    a.opndB = &ob;
  }
  a.M = g.M; a.N = g.N; a.K = g.K;
  a.A = g.A; a.lda = g.lda; a.sA = g.sA; a.opA = g.opA;
  a.B = g.B; a.ldb = g.ldb; a.sB = g.sB; a.opB = g.opB;
  a.C0 = g.C0; a.ldc0 = g.ldc0; a.sC0 = g.sC0;
  a.C = g.C; a.ldc = g.ldc; a.sC = g.sC;
  a.alpha = g.alpha; a.beta = g.beta;
  a.batch = g.batch; a.active = g.active;
  a.stages = P->d.tc_stages; a.ctas = P->d.tc_ctas;
  if (P->group && gemm_tc_variant(a, digits) >= 0) {
    QTX_CK(group_gemm(P, a, digits, st));
    return QTX_OK;
  }
  // the profile times the products at the plan's digit count (one kernel instance)
  cudaEvent_t* ev = (P->prof && digits == tc_digits(P->d)) ? P->next_events() : nullptr;
  QTX_CK(gemm_tc(a, digits, P->ws + P->L.tc_scratch, P->L.tc_bytes, P->d_err_flag, st, ev));
  if (ev) {
    const double f = 8.0 * g.M * g.N * g.K * g.batch;
    P->pipe_flops += f * tc_pairs(digits);
    P->useful_flops += f;
  }
  return QTX_OK;
}

// Plain (non-refined) recursive inverse of n x n blocks stored with leading dimension lda.
// T12/T21 scratch for each recursion level is carved from `scratch` (>= 0.7 n^2 per batch entry).
template <typename T>
qtx_status inverse_rec(qtx_rgf_plan_s* P, cx<T>* A, long lda, long sA, int n, int batch,
                       const int* active, int* status, cx<T>* scratch, long sScr, cudaStream_t st,
                       bool force_simt) {
  if (n <= kLeafMax) {
    QTX_CK(leaf_inverse<T>(A, lda, sA, n, batch, active, status, st));
    return QTX_OK;
  }
  const int h = (n + 1) / 2, r = n - h;
  cx<T>* A11 = A;
  cx<T>* A12 = A + h;
  cx<T>* A21 = A + (long)h * lda;
  cx<T>* A22 = A + (long)h * lda + h;
  cx<T>* T12 = scratch;              // h x r, ld r
  cx<T>* T21 = scratch + (long)h * r; // r x h, ld h
  cx<T>* next = scratch + 2L * h * r;
  qtx_status s;
  if ((s = inverse_rec<T>(P, A11, lda, sA, h, batch, active, status, next, sScr, st, force_simt))) return s;
  // T12 = X11 A12 ; T21 = A21 X11
  if ((s = gemm<T>(P, gargs<T>(h, r, h, A11, lda, sA, OP_N, A12, lda, sA, OP_N, nullptr, 0, 0, T12, r, sScr, 1.0, 0.0, batch, active), st, force_simt))) return s;
  if ((s = gemm<T>(P, gargs<T>(r, h, h, A21, lda, sA, OP_N, A11, lda, sA, OP_N, nullptr, 0, 0, T21, h, sScr, 1.0, 0.0, batch, active), st, force_simt))) return s;
  // A22 <- A22 - A21 T12 (Schur complement), then invert it in place
  if ((s = gemm<T>(P, gargs<T>(r, r, h, A21, lda, sA, OP_N, T12, r, sScr, OP_N, A22, lda, sA, A22, lda, sA, -1.0, 1.0, batch, active), st, force_simt))) return s;
  if ((s = inverse_rec<T>(P, A22, lda, sA, r, batch, active, status, next, sScr, st, force_simt))) return s;
  // A12 <- -T12 Y ; A21 <- -Y T21 ; A11 <- X11 - T12 A21
  if ((s = gemm<T>(P, gargs<T>(h, r, r, T12, r, sScr, OP_N, A22, lda, sA, OP_N, nullptr, 0, 0, A12, lda, sA, -1.0, 0.0, batch, active), st, force_simt))) return s;
  if ((s = gemm<T>(P, gargs<T>(r, h, r, A22, lda, sA, OP_N, T21, h, sScr, OP_N, nullptr, 0, 0, A21, lda, sA, -1.0, 0.0, batch, active), st, force_simt))) return s;
  if ((s = gemm<T>(P, gargs<T>(h, h, r, T12, r, sScr, OP_N, A21, lda, sA, OP_N, A11, lda, sA, A11, lda, sA, -1.0, 1.0, batch, active), st, force_simt))) return s;
  return QTX_OK;
}

// Recursive inverse followed, when the recursion splits the block (n > kLeafMax), by one Newton
// step X <- X + X (I - A X) in the same precision: elimination without pivoting between the two
// halves can lose digits on ill-conditioned leading blocks (e.g. the decimation's z - eps), and one
// step brings the result back to the accuracy of a pivoted inverse.
template <typename T>
qtx_status inverse_refined(qtx_rgf_plan_s* P, cx<T>* A, int n, int batch, const int* active,
                           int* status, cudaStream_t st) {
  const long nn = (long)n * n;
  cx<T>* scr = reinterpret_cast<cx<T>*>(P->ws + P->L.inv_tmp);
  if (n <= kLeafMax) return inverse_rec<T>(P, A, n, nn, n, batch, active, status, scr, nn, st, true);
  cx<T>* Acopy = reinterpret_cast<cx<T>*>(P->ws + P->L.ref);
  cx<T>* R = Acopy + (size_t)P->Ec * nn;
  cx<T>* Xn = R + (size_t)P->Ec * nn;
  Term<T> tA; tA.p = A; tA.s = nn; tA.alpha = 1.0;
  Term<T> none;
  QTX_CK((combine<T, T>(Acopy, nn, tA, none, none, n, batch, nullptr, 0.0, 0.0, active, st)));
  qtx_status s = inverse_rec<T>(P, A, n, nn, n, batch, active, status, scr, nn, st, true);
  if (s) return s;
  // R = I - Acopy X  (identity via the diagonal term of combine), Xn = X + X R, X <- Xn
  if ((s = gemm<T>(P, gargs<T>(n, n, n, Acopy, n, nn, OP_N, A, n, nn, OP_N, nullptr, 0, 0, R, n, nn, -1.0, 0.0, batch, active), st, true))) return s;
  QTX_CK(add_identity<T>(R, nn, n, batch, active, st));
  if ((s = gemm<T>(P, gargs<T>(n, n, n, A, n, nn, OP_N, R, n, nn, OP_N, A, n, nn, Xn, n, nn, 1.0, 1.0, batch, active), st, true))) return s;
  Term<T> tX; tX.p = Xn; tX.s = nn; tX.alpha = 1.0;
  QTX_CK((combine<T, T>(A, nn, tX, none, none, n, batch, nullptr, 0.0, 0.0, active, st)));
  return QTX_OK;
}

// FP32 inverse used as the emulated modes' starting guess (the df32 Newton sweeps that follow only
// need ||I - A X0|| < 1); its scratch lives in the FP32 area so the df32 buffers stay intact.
qtx_status inverse_refined_f32(qtx_rgf_plan_s* P, cx<float>* A, int n, int batch, const int* active,
                               int* status, cudaStream_t st) {
  const long nn = (long)n * n;
  cx<float>* scr = reinterpret_cast<cx<float>*>(P->ws + P->L.f32tmp);
  return inverse_rec<float>(P, A, n, nn, n, batch, active, status, scr, nn, st, true);
}

// Block inverse used by the sweep.  FP64 / FP32: recursive inverse in the sweep precision.
// EMU64 / BF16X3: X0 from the recursive inverse in FP32, then Newton refinement
// X <- X + X (I - A X) with both products on the tensor-core engine (the residual I - A X is
// formed in emulated FP64 before it is rounded for the correction product).
template <typename T>
qtx_status block_inverse(qtx_rgf_plan_s* P, cx<T>* A, int n, int batch, const int* active,
                         int* status, cudaStream_t st);

template <>
qtx_status block_inverse<float>(qtx_rgf_plan_s* P, cx<float>* A, int n, int batch, const int* active,
                                int* status, cudaStream_t st) {
  return inverse_refined<float>(P, A, n, batch, active, status, st);
}

template <>
qtx_status block_inverse<double>(qtx_rgf_plan_s* P, cx<double>* A, int n, int batch, const int* active,
                                 int* status, cudaStream_t st) {
  return inverse_refined<double>(P, A, n, batch, active, status, st);
}

// Emulated modes (df32 storage): X0 from the FP32 inverse of the leading parts, then Newton sweeps
// X <- X + X (I - A X) with both products on the tensor-core engine; the residual I - A X is formed
// by the engine's ~38-bit products with I added exactly in the epilogue.
template <>
qtx_status block_inverse<df>(qtx_rgf_plan_s* P, cx<df>* A, int n, int batch, const int* active,
                             int* status, cudaStream_t st) {
  const long nn = (long)n * n;
  cx<float>* A32 = reinterpret_cast<cx<float>*>(P->ws + P->L.f32a);
  cx<df>* Acopy = reinterpret_cast<cx<df>*>(P->ws + P->L.ref);
  cx<df>* R = Acopy + (size_t)P->Ec * nn;
  cx<df>* Xn = R + (size_t)P->Ec * nn;
  const cx<df>* I = reinterpret_cast<const cx<df>*>(P->ws + P->L.ident_df);
  Term<df> tA; tA.p = A; tA.s = nn; tA.alpha = 1.0;
  Term<df> none;
  QTX_CK((combine<df, float>(A32, nn, tA, none, none, n, batch, nullptr, 0.0, 0.0, active, st)));
  QTX_CK((combine<df, df>(Acopy, nn, tA, none, none, n, batch, nullptr, 0.0, 0.0, active, st)));
  qtx_status s = inverse_refined_f32(P, A32, n, batch, active, status, st);
  if (s) return s;
  Term<float> tX; tX.p = A32; tX.s = nn; tX.alpha = 1.0;
  Term<float> none32;
  QTX_CK((combine<float, df>(A, nn, tX, none32, none32, n, batch, nullptr, 0.0, 0.0, active, st)));
  // With refine_tol > 0 an energy leaves the sweeps once ||I - A X||_F <= refine_tol: the masks
  // (ping-pong in refine_act) make every later product, digitisation and combination skip it.
  int* masks = reinterpret_cast<int*>(P->ws + P->L.refine_act);
  const int* act = active;
  for (int it = 0; it < P->d.refine_max_iter; ++it) {
    // Acopy's digit planes serve every sweep
    if ((s = gemm<df>(P, gargs<df>(n, n, n, Acopy, n, nn, OP_N, A, n, nn, OP_N, I, n, 0, R, n, nn, -1.0, 1.0, batch, act), st,
                      false, it == 0 ? keepA(0) : reuseA(0)))) return s;
    int* next = nullptr;
    if (P->d.refine_tol > 0.0 && it + 1 < P->d.refine_max_iter) {
      next = masks + (it & 1) * P->Ec;
      QTX_CK(residual_mask(R, nn, n, batch, P->d.refine_tol, act, next, status, st));
    }
    // The correction X R is small (||R|| <= 2^-12 once an energy is refined, and typically near the
    // FP32 inverse's kappa 2^-24), so four digit planes (~27-bit operands, every digit group exact)
    // keep its error near 2^-27 |X| |R|, far below the 2^-40 the sweep keeps; R itself, where A X
    // cancels against I, takes the plan's six.
    const DigitHint xr = tc_digits(P->d) == 6 ? planes(4) : DigitHint{};
    if (n <= 1024) {
      // X <- X + X R in place: the product reads X only through its digit planes (made before the
      // launch) and, element by element in the epilogue, as C0 right before writing C
      if ((s = gemm<df>(P, gargs<df>(n, n, n, A, n, nn, OP_N, R, n, nn, OP_N, A, n, nn, A, n, nn, 1.0, 1.0, batch, act), st,
                        false, xr))) return s;
    } else {
      // split along K: a later K-chunk digitises columns of X an earlier chunk would have overwritten
      if ((s = gemm<df>(P, gargs<df>(n, n, n, A, n, nn, OP_N, R, n, nn, OP_N, A, n, nn, Xn, n, nn, 1.0, 1.0, batch, act), st,
                        false, xr))) return s;
      Term<df> tXn; tXn.p = Xn; tXn.s = nn; tXn.alpha = 1.0;
      QTX_CK((combine<df, df>(A, nn, tXn, none, none, n, batch, nullptr, 0.0, 0.0, act, st)));
    }
    if (next) act = next;
  }
  return QTX_OK;
}

// ----------------------------------------------------------------------------- contacts
// Batched Sancho-Rubio decimation for one contact (FP64); result Sigma^R = H01 g_s H01^H in SR.
// Nothing here reads back to the host: for lead blocks of at most kDecimSmallMax the whole iteration
// of an energy runs in one CTA (decimate_small); larger blocks run decim_max_iter sweeps of batched
// launches in which converged energies are masked off on the device (their launches return at once),
// with the tolerance scale max|H01| computed on the device too.  A solve with contacts therefore
// makes no host synchronisation and can be captured in a CUDA graph.
template <typename T>
qtx_status contact(const Ctx<T>& c, const cx<double>* H00, const cx<double>* H01, double eta,
                   cx<double>* SR) {
  qtx_rgf_plan_s* P = c.P;
  const int b = c.b, ne = c.ne;
  const long bb = c.bb;
  cudaStream_t st = c.st;
  if (b <= kDecimSmallMax) {
    QTX_CK(decimate_small(H00, H01, c.E, eta, P->d.decim_tol, P->d.decim_max_iter, b, ne, SR, c.status, st));
    return QTX_OK;
  }
  cx<double>* D = reinterpret_cast<cx<double>*>(P->ws + P->L.dec);
  auto buf = [&](int k) { return D + (size_t)k * P->Ec * bb; };
  cx<double>*alpha = buf(0), *beta = buf(1), *eps = buf(2), *eps_s = buf(3), *g = buf(4), *ag = buf(5),
  *bg = buf(6), *t1 = buf(7), *t2 = buf(8);
  int* flags = reinterpret_cast<int*>(P->ws + P->L.flags);
  int* active = flags;
  int* sweeps = flags + P->Ec;
  double* scale = reinterpret_cast<double*>(P->ws + P->L.dscale);
  QTX_CK(max_modulus(H01, bb, scale, st));

  Term<double> none;
  Term<double> t01; t01.p = H01; t01.s = 0; t01.alpha = 1.0;
  Term<double> t01h = t01; t01h.op = OP_C;
  Term<double> t00; t00.p = H00; t00.s = 0; t00.alpha = 1.0;
  QTX_CK((combine<double, double>(alpha, bb, t01, none, none, b, ne, nullptr, 0, 0, nullptr, st)));
  QTX_CK((combine<double, double>(beta, bb, t01h, none, none, b, ne, nullptr, 0, 0, nullptr, st)));
  QTX_CK((combine<double, double>(eps, bb, t00, none, none, b, ne, nullptr, 0, 0, nullptr, st)));
  QTX_CK((combine<double, double>(eps_s, bb, t00, none, none, b, ne, nullptr, 0, 0, nullptr, st)));
  QTX_CK(fill_int(active, 1, ne, st));
  QTX_CK(cudaMemsetAsync(sweeps, 0, ne * sizeof(int), st));
  qtx_status s;
  auto G = [&](const cx<double>* A, const cx<double>* B, cx<double>* C) {
    return gemm<double>(P, gargs<double>(b, b, b, A, b, bb, OP_N, B, b, bb, OP_N, nullptr, 0, 0, C, b, bb, 1.0, 0.0, ne, active), st, true);
  };
  for (int it = 1; it <= P->d.decim_max_iter; ++it) {
    Term<double> te; te.p = eps; te.s = bb; te.alpha = -1.0;
    QTX_CK((combine<double, double>(g, bb, te, none, none, b, ne, c.E, eta, 1.0, active, st)));  // z - eps
    if ((s = inverse_refined<double>(P, g, b, ne, active, c.status, st))) return s;
    if ((s = G(alpha, g, ag))) return s;
    if ((s = G(beta, g, bg))) return s;
    if ((s = G(ag, beta, t1))) return s;   // alpha g beta
    if ((s = G(bg, alpha, t2))) return s;  // beta g alpha
    Term<double> ts; ts.p = eps_s; ts.s = bb; ts.alpha = 1.0;
    Term<double> ta; ta.p = t1; ta.s = bb; ta.alpha = 1.0;
    Term<double> tb; tb.p = t2; tb.s = bb; tb.alpha = 1.0;
    Term<double> tep; tep.p = eps; tep.s = bb; tep.alpha = 1.0;
    QTX_CK((combine<double, double>(eps_s, bb, ts, ta, none, b, ne, nullptr, 0, 0, active, st)));
    QTX_CK((combine<double, double>(eps, bb, tep, ta, tb, b, ne, nullptr, 0, 0, active, st)));
    if ((s = G(ag, alpha, t1))) return s;  // alpha g alpha
    if ((s = G(bg, beta, t2))) return s;   // beta g beta
    Term<double> tt1; tt1.p = t1; tt1.s = bb; tt1.alpha = 1.0;
    Term<double> tt2; tt2.p = t2; tt2.s = bb; tt2.alpha = 1.0;
    QTX_CK((combine<double, double>(alpha, bb, tt1, none, none, b, ne, nullptr, 0, 0, active, st)));
    QTX_CK((combine<double, double>(beta, bb, tt2, none, none, b, ne, nullptr, 0, 0, active, st)));
    QTX_CK(decim_converged(alpha, beta, b, P->d.decim_tol, scale, active, sweeps, ne, st));
  }
  QTX_CK(flag_active(active, c.status, (int)QTX_ERR_NOT_CONVERGED, ne, st));
  Term<double> tes; tes.p = eps_s; tes.s = bb; tes.alpha = -1.0;
  QTX_CK((combine<double, double>(g, bb, tes, none, none, b, ne, c.E, eta, 1.0, nullptr, st)));  // z - eps_s
  if ((s = inverse_refined<double>(P, g, b, ne, nullptr, c.status, st))) return s;
  // Sigma^R = H01 g_s H01^H
  if ((s = gemm<double>(P, gargs<double>(b, b, b, H01, b, 0, OP_N, g, b, bb, OP_N, nullptr, 0, 0, t1, b, bb, 1.0, 0.0, ne, nullptr), st, true))) return s;
  if ((s = gemm<double>(P, gargs<double>(b, b, b, t1, b, bb, OP_N, H01, b, 0, OP_C, nullptr, 0, 0, SR, b, bb, 1.0, 0.0, ne, nullptr), st, true))) return s;
  return QTX_OK;
}

// Copy/convert a sweep block (batch stride bb) into a complex128 output [e][slice] layout.
template <typename T>
qtx_status emit(qtx_rgf_plan_s* P, void* out, long nslices, long slice, int e0, const cx<T>* src,
                int b, int ne, cudaStream_t st, const cx<T>* plus = nullptr, const cx<T>* minus_h = nullptr) {
  if (!out) return QTX_OK;
  const long bb = (long)b * b;
  cx<double>* o = reinterpret_cast<cx<double>*>(out) + ((long)e0 * nslices + slice) * bb;
  Term<T> t0; t0.p = src; t0.s = bb; t0.alpha = 1.0;
  Term<T> t1; t1.p = plus; t1.s = bb; t1.alpha = 1.0;
  Term<T> t2; t2.p = minus_h; t2.s = bb; t2.alpha = -1.0; t2.op = OP_C;
  QTX_CK((combine<T, double>(o, nslices * bb, t0, t1, t2, b, ne, nullptr, 0.0, 0.0, nullptr, st)));
  return QTX_OK;
}

template <typename T>
qtx_status solve_chunk(qtx_rgf_plan_s* P, const qtx_rgf_inputs* in, const qtx_rgf_outputs* out,
                       int e0, int ne, int* status, cudaStream_t st) {
  const qtx_rgf_desc& d = P->d;
  const int b = P->b, nb = P->nb;
  const long bb = P->bb;
  Ctx<T> c{P, st, ne, in->energies + e0, status, bb, b};
  const double eta = in->eta;
  const cx<double>* Hd = reinterpret_cast<const cx<double>*>(in->H_diag);
  const cx<double>* Hu = reinterpret_cast<const cx<double>*>(in->H_upper);
  const cx<double>* Sd = d.has_S ? reinterpret_cast<const cx<double>*>(in->S_diag) : nullptr;
  const cx<double>* Su = d.has_S ? reinterpret_cast<const cx<double>*>(in->S_upper) : nullptr;
  const cx<double>* SRd = d.has_scattering ? reinterpret_cast<const cx<double>*>(in->SigR_diag) : nullptr;
  const cx<double>* SLd = d.has_scattering ? reinterpret_cast<const cx<double>*>(in->SigL_diag) : nullptr;
  const long sSig = d.energy_dependent_sigma ? (long)nb * bb : 0;
  const long sigE0 = d.energy_dependent_sigma ? (long)e0 * nb * bb : 0;
  auto sigR = [&](int i) { return SRd ? SRd + sigE0 + (long)i * bb : nullptr; };
  auto sigL = [&](int i) { return SLd ? SLd + sigE0 + (long)i * bb : nullptr; };
  // second right-hand side (second_rhs): B2 in the layout of Sigma^<
  const int nrhs = d.second_rhs ? 2 : 1;
  const cx<double>* SGd = d.second_rhs ? reinterpret_cast<const cx<double>*>(in->SigG_diag) : nullptr;
  auto sigG = [&](int i) { return SGd ? SGd + sigE0 + (long)i * bb : nullptr; };
  // off-diagonal scattering blocks [N_E or 1][N_B-1][b][b]
  const bool odg = d.offdiag_sigma && nb > 1;
  const long sSigU = d.energy_dependent_sigma ? (long)(nb - 1) * bb : 0;
  const long sigUE0 = d.energy_dependent_sigma ? (long)e0 * (nb - 1) * bb : 0;
  const cx<double>* SRu = odg && !d.system_input ? reinterpret_cast<const cx<double>*>(in->SigR_upper) + sigUE0 : nullptr;
  const cx<double>* SRl = odg && !d.system_input ? reinterpret_cast<const cx<double>*>(in->SigR_lower) + sigUE0 : nullptr;
  const cx<double>* SLu = odg ? reinterpret_cast<const cx<double>*>(in->SigL_upper) + sigUE0 : nullptr;
  const cx<double>* SGu = odg && d.second_rhs ? reinterpret_cast<const cx<double>*>(in->SigG_upper) + sigUE0 : nullptr;
  // Sigma^<_{i,i+1} in the sweep's type (tmp 12): one block shared by the chunk, or one per energy
  const int nLt = d.energy_dependent_sigma ? ne : 1;
  const long sLt = d.energy_dependent_sigma ? bb : 0;
  // right-hand side k's upper block of slice i (k = 1: B2_{i,i+1})
  auto load_L = [&](int k, int i) -> cx<T>* {
    cx<T>* Lt = c.tmp(12);
    if (axpby_from64<T>(Lt, bb, (k ? SGu : SLu) + (long)i * bb, sSigU, 1.0, nullptr, 0, 0.0, b, nLt, st) != cudaSuccess) return nullptr;
    return Lt;
  };
  qtx_status s;
  Term<T> none;

  // ---- 1. contacts
  cx<double>* LB = reinterpret_cast<cx<double>*>(P->ws + P->L.lead);
  auto lb = [&](int k) { return LB + (size_t)k * P->Ec * bb; };
  cx<double>*SR_L = lb(0), *Gam_L = lb(1), *SL_L = lb(2), *SG_L = lb(3);
  cx<double>*SR_R = lb(4), *Gam_R = lb(5), *SL_R = lb(6), *SG_R = lb(7);
  if (d.leads) {
    if ((s = contact<T>(c, (const cx<double>*)in->lead_H00_L, (const cx<double>*)in->lead_H01_L, eta, SR_L))) return s;
    if ((s = contact<T>(c, (const cx<double>*)in->lead_H00_R, (const cx<double>*)in->lead_H01_R, eta, SR_R))) return s;
    QTX_CK(lead_sigmas(SR_L, Gam_L, SL_L, SG_L, c.E, in->mu_L, in->kT, b, ne, st));
    QTX_CK(lead_sigmas(SR_R, Gam_R, SL_R, SG_R, c.E, in->mu_R, in->kT, b, ne, st));
  }

  // ---- off-diagonal blocks of M
  cx<T>* Ub = reinterpret_cast<cx<T>*>(P->ws + P->L.U);
  cx<T>* Vb = reinterpret_cast<cx<T>*>(P->ws + P->L.V);
  const bool uvE = uv_per_energy(d);
  const long sUV = uvE ? bb : 0;
  auto U = [&](int i) { return Ub + (size_t)i * (uvE ? P->Ec * bb : bb); };
  auto V = [&](int i) { return Vb + (size_t)i * (uvE ? P->Ec * bb : bb); };
  // system input (M given): per-energy blocks [N_E][N_B(-1)][b][b]
  const cx<double>* Md = d.system_input ? reinterpret_cast<const cx<double>*>(in->M_diag) + (long)e0 * nb * bb : nullptr;
  const cx<double>* Mu = d.system_input && nb > 1 ? reinterpret_cast<const cx<double>*>(in->M_upper) + (long)e0 * (nb - 1) * bb : nullptr;
  const cx<double>* Ml = d.system_input && nb > 1 ? reinterpret_cast<const cx<double>*>(in->M_lower) + (long)e0 * (nb - 1) * bb : nullptr;
  for (int i = 0; i + 1 < nb; ++i) {
    if (d.system_input) {
      QTX_CK(axpby_from64<T>(U(i), bb, Mu + (long)i * bb, (long)(nb - 1) * bb, 1.0, nullptr, 0, 0.0, b, ne, st));
      QTX_CK(axpby_from64<T>(V(i), bb, Ml + (long)i * bb, (long)(nb - 1) * bb, 1.0, nullptr, 0, 0.0, b, ne, st));
      continue;
    }
    const cx<double>* sru = SRu ? SRu + (long)i * bb : nullptr;
    const cx<double>* srl = SRl ? SRl + (long)i * bb : nullptr;
    if (uvE) QTX_CK(assemble_offdiag<T>(U(i), V(i), Hu + (long)i * bb, Su ? Su + (long)i * bb : nullptr, c.E, eta, b, ne, st, sru, srl, sSigU));
    else QTX_CK(assemble_offdiag<T>(U(i), V(i), Hu + (long)i * bb, nullptr, nullptr, 0.0, b, 1, st, sru, srl, 0));
  }

  // ---- 2. forward sweep
  for (int i = 0; i < nb; ++i) {
    cx<T>* gi = c.g(i);
    const cx<double>* lead = nullptr;
    if (d.leads && i == 0) lead = SR_L;
    else if (d.leads && i == nb - 1) lead = SR_R;
    // streamed self-energies: this slice's blocks of the chunk's energies, host -> staging area
    const cx<double>* sRi = sigR(i);
    const cx<double>* sLi = sigL(i);
    long sS = sSig;
    if (d.sigma_stream) {
      cx<double>* stR = reinterpret_cast<cx<double>*>(P->ws + P->L.sig_stage);
      cx<double>* stL = stR + (size_t)P->Ec * bb;
      const size_t row = (size_t)bb * sizeof(cx<double>), pitch = (size_t)nb * row;
      if (pitch < ((size_t)1 << 31)) {  // one strided copy per kind
        QTX_CK(cudaMemcpy2DAsync(stR, row, sRi, pitch, row, ne, cudaMemcpyHostToDevice, st));
        QTX_CK(cudaMemcpy2DAsync(stL, row, sLi, pitch, row, ne, cudaMemcpyHostToDevice, st));
      } else {                          // pitches beyond the 2D copy's range: one copy per energy
        for (int e = 0; e < ne; ++e) {
          QTX_CK(cudaMemcpyAsync(stR + (size_t)e * bb, sRi + (size_t)e * nb * bb, row, cudaMemcpyHostToDevice, st));
          QTX_CK(cudaMemcpyAsync(stL + (size_t)e * bb, sLi + (size_t)e * nb * bb, row, cudaMemcpyHostToDevice, st));
        }
      }
      sRi = stR;
      sLi = stL;
      sS = bb;
    }
    cx<T>* shared_blk = reinterpret_cast<cx<T>*>(P->ws + P->L.shared_blk);
    if (d.system_input) QTX_CK(axpby_from64<T>(gi, bb, Md + (long)i * bb, (long)nb * bb, 1.0, nullptr, 0, 0.0, b, ne, st));
    else if (!std::is_same<T, double>::value && !Sd && (sS == 0 || !sRi) && !lead) {
      // Sigma^R shared by the energies: -(H_ii + Sigma^R_ii) converted once, then E + i eta added
      // on each energy's diagonal
      QTX_CK(axpby_from64<T>(shared_blk, 0, Hd + (long)i * bb, 0, -1.0, sRi, 0, -1.0, b, 1, st));
      QTX_CK(broadcast_diag<T>(gi, bb, shared_blk, b, c.E, eta, ne, st));
    } else QTX_CK(assemble_diag<T>(gi, Hd + (long)i * bb, Sd ? Sd + (long)i * bb : nullptr, sRi, sS, lead, bb, c.E, eta, b, ne, st));
    if (d.leads && nb == 1) {  // one slice touches both contacts
      Term<T> tg; tg.p = gi; tg.s = bb; tg.alpha = 1.0;
      QTX_CK((combine<T, T>(c.tmp(0), bb, tg, none, none, b, ne, nullptr, 0, 0, nullptr, st)));
      QTX_CK(axpby_from64<T>(c.tmp(1), bb, SR_R, bb, -1.0, nullptr, 0, 0.0, b, ne, st));
      Term<T> t0; t0.p = c.tmp(0); t0.s = bb; t0.alpha = 1.0;
      Term<T> t1; t1.p = c.tmp(1); t1.s = bb; t1.alpha = 1.0;
      QTX_CK((combine<T, T>(gi, bb, t0, t1, none, b, ne, nullptr, 0, 0, nullptr, st)));
    }
    if (i > 0 && c.keep_z()) {
      // V g U as (V g) U: Z_{i-1} = V_{i-1} g_{i-1} is kept for the backward sweep
      // (G_{i,i-1} = -G_ii Z_{i-1}), which then needs one product less per slice
      cx<T>* Zp = c.zk(i - 1);
      if ((s = gemm<T>(P, gargs<T>(b, b, b, V(i - 1), b, sUV, OP_N, c.g(i - 1), b, bb, OP_N, nullptr, 0, 0, Zp, b, bb, 1.0, 0.0, ne, nullptr), st)))
        return s;
      if ((s = gemm<T>(P, gargs<T>(b, b, b, Zp, b, bb, OP_N, U(i - 1), b, sUV, OP_N, gi, b, bb, gi, b, bb, -1.0, 1.0, ne, nullptr), st))) return s;
    } else if (i > 0) {
      cx<T>* Tm = c.tmp(0);
      // g_{i-1} was the left operand of the previous slice's g_{i-1} Sigma^<: its digit planes are kept
      if ((s = gemm<T>(P, gargs<T>(b, b, b, c.g(i - 1), b, bb, OP_N, U(i - 1), b, sUV, OP_N, nullptr, 0, 0, Tm, b, bb, 1.0, 0.0, ne, nullptr), st,
                       false, reuseA(1)))) return s;
      if ((s = gemm<T>(P, gargs<T>(b, b, b, V(i - 1), b, sUV, OP_N, Tm, b, bb, OP_N, gi, b, bb, gi, b, bb, -1.0, 1.0, ne, nullptr), st))) return s;
    }
    if ((s = block_inverse<T>(P, gi, b, ne, nullptr, status, st))) return s;
    // block-tridiagonal right-hand sides: V_{i-1} g_{i-1} of the cross term, shared by both
    cx<T>* Zf = i > 0 && c.keep_z() ? c.zk(i - 1) : c.tmp(2);
    if (i > 0 && odg && !c.keep_z() &&
        (s = gemm<T>(P, gargs<T>(b, b, b, V(i - 1), b, sUV, OP_N, c.g(i - 1), b, bb, OP_N, nullptr, 0, 0, Zf, b, bb, 1.0, 0.0, ne, nullptr), st)))
      return s;
    for (int k = 0; k < nrhs; ++k) {
      // Sigma^<_ii (+ contacts; or B2_ii), then the left-connected lesser function of right-hand side k
      cx<T>* SLi = c.tmp(1);
      const cx<double>* sl = k ? sigG(i) : sLi;
      const cx<double>* lsl = nullptr;
      if (k == 0 && d.leads && i == 0) lsl = SL_L;
      else if (k == 0 && d.leads && i == nb - 1) lsl = SL_R;
      if (sl && !lsl && sS == 0 && !std::is_same<T, double>::value) {  // shared: converted once
        QTX_CK(axpby_from64<T>(shared_blk, 0, sl, 0, 1.0, nullptr, 0, 0.0, b, 1, st));
        QTX_CK(broadcast_diag<T>(SLi, bb, shared_blk, b, nullptr, 0.0, ne, st));
      } else if (sl) QTX_CK(axpby_from64<T>(SLi, bb, sl, sS, 1.0, lsl, bb, 1.0, b, ne, st));
      else if (lsl) QTX_CK(axpby_from64<T>(SLi, bb, lsl, bb, 1.0, nullptr, 0, 0.0, b, ne, st));
      else QTX_CK(cudaMemsetAsync(SLi, 0, (size_t)ne * bb * sizeof(cx<T>), st));
      if (k == 0 && d.leads && nb == 1) {
        QTX_CK(axpby_from64<T>(c.tmp(2), bb, SL_R, bb, 1.0, nullptr, 0, 0.0, b, ne, st));
        Term<T> t0; t0.p = SLi; t0.s = bb; t0.alpha = 1.0;
        Term<T> t1; t1.p = c.tmp(2); t1.s = bb; t1.alpha = 1.0;
        QTX_CK((combine<T, T>(SLi, bb, t0, t1, none, b, ne, nullptr, 0, 0, nullptr, st)));
      }
      if (i > 0) {
        cx<T>* X = c.keep_z() ? c.xk(k, i - 1) : c.tmp(0);  // V_{i-1} g^<_{i-1}
        if ((s = gemm<T>(P, gargs<T>(b, b, b, V(i - 1), b, sUV, OP_N, c.glk(k, i - 1), b, bb, OP_N, nullptr, 0, 0, X, b, bb, 1.0, 0.0, ne, nullptr), st))) return s;
        if ((s = gemm<T>(P, gargs<T>(b, b, b, X, b, bb, OP_N, V(i - 1), b, sUV, OP_C, SLi, b, bb, SLi, b, bb, 1.0, 1.0, ne, nullptr), st))) return s;
        if (odg) {  // block-tridiagonal Sigma^<: bracket += -Y + Y^H, Y = V_{i-1} g_{i-1} Sigma^<_{i-1,i}
          cx<T>* Yf = c.tmp(3);
          cx<T>* Lt = load_L(k, i - 1);
          if (!Lt) return QTX_ERR_CUDA;
          if ((s = gemm<T>(P, gargs<T>(b, b, b, Zf, b, bb, OP_N, Lt, b, sLt, OP_N, nullptr, 0, 0, Yf, b, bb, 1.0, 0.0, ne, nullptr), st))) return s;
          Term<T> t0; t0.p = SLi; t0.s = bb; t0.alpha = 1.0;
          Term<T> t1; t1.p = Yf; t1.s = bb; t1.alpha = -1.0;
          Term<T> t2; t2.p = Yf; t2.s = bb; t2.alpha = 1.0; t2.op = OP_C;
          QTX_CK((combine<T, T>(SLi, bb, t0, t1, t2, b, ne, nullptr, 0, 0, nullptr, st)));
        }
      }
      cx<T>* Y = c.tmp(0);
      if ((s = gemm<T>(P, gargs<T>(b, b, b, gi, b, bb, OP_N, SLi, b, bb, OP_N, nullptr, 0, 0, Y, b, bb, 1.0, 0.0, ne, nullptr), st,
                       false, k ? reuseA(1) : keepA(1)))) return s;
      if ((s = gemm<T>(P, gargs<T>(b, b, b, Y, b, bb, OP_N, gi, b, bb, OP_C, nullptr, 0, 0, c.glk(k, i), b, bb, 1.0, 0.0, ne, nullptr), st))) return s;
    }  // right-hand sides
    // FPX storage: slices the backward sweep reads back from memory (the last two stay in the
    // working blocks) are kept compressed
    if (d.storage_bits && i < nb - 2) {
      QTX_CK(fpx_store<T>(d.storage_bits, gi, (long)ne * bb, c.gfx(i), st));
      QTX_CK(fpx_store<T>(d.storage_bits, c.gl(i), (long)ne * bb, c.glfx(i), st));
    }
  }

  // ---- 3. backward sweep.  With P = g_i U_i, Z = V_i g_i, Q = V_i g^<_i:
  //   G_{i+1,i} = -G_{i+1,i+1} Z,  G_{i,i+1} = -P G_{i+1,i+1},  G_ii = g_i - P G_{i+1,i}
  //   K = P G_{i+1,i+1} Q = -G_{i,i+1} Q   (block-tridiagonal Sigma^<: Q += (g_i Sigma^<_{i,i+1})^H)
  //   G^<_ii = g^<_i + (P G^<_{i+1,i+1}) P^H + K - K^H
  //   G^<_{i,i+1} = -P G^<_{i+1,i+1} + (G_{i+1,i+1} Q)^H     [= -P G^< - g^< V^H G^A]
  double* obs = reinterpret_cast<double*>(P->ws + P->L.obs);
  const int ncur = nb > 1 ? nb - 1 : 1;
  double* cur = obs;                           // [ne][nb-1]
  double* den = cur + (size_t)P->Ec * ncur;    // [ne][nb]
  double* con = den + (size_t)P->Ec * nb;      // [ne][2]
  double* tra = con + (size_t)P->Ec * 2;       // [ne]
  const unsigned m = d.outputs;
  auto want = [&](unsigned bit, const void* p) { return (m & bit) && p; };
  // current conservation (Sec. II-B): per-slice balances J_i, checked after the sweep
  const bool cont = (m & QTX_OUT_CONTINUITY) || d.escalate_tol > 0;
  double* bal = reinterpret_cast<double*>(P->ws + P->L.bal);        // [ne][nb]
  double* bscale = reinterpret_cast<double*>(P->ws + P->L.bscale);  // [ne][nb]
  double* bgn = reinterpret_cast<double*>(P->ws + P->L.bgn);        // [ne][nb]
  double* bhn = reinterpret_cast<double*>(P->ws + P->L.bhn);        // [ne][nb]
  {
    const int i = nb - 1;
    if (want(QTX_OUT_GR_DIAG, out->GR_diag) && (s = emit<T>(P, out->GR_diag, nb, i, e0, c.g(i), b, ne, st))) return s;
    if (want(QTX_OUT_GL_DIAG, out->GL_diag) && (s = emit<T>(P, out->GL_diag, nb, i, e0, c.gl(i), b, ne, st))) return s;
    if (want(QTX_OUT_GG_DIAG, out->GG_diag) &&
        (s = d.second_rhs ? emit<T>(P, out->GG_diag, nb, i, e0, c.glk(1, i), b, ne, st)
                          : emit<T>(P, out->GG_diag, nb, i, e0, c.gl(i), b, ne, st, c.g(i), c.g(i))))
      return s;
    QTX_CK(obs_density<T>(den + i, nb, c.gl(i), bb, b, ne, st));
    if (cont)
      QTX_CK(obs_balance<T>(bal + i, bscale + i, bgn + i, bhn + i, nb, sigL(i), sigR(i), sSig, c.g(i), c.gl(i), bb,
                            eta, b, ne, st, Hd + (long)i * bb, nullptr, nullptr, c.E, nullptr));
    if (d.leads) {  // right contact current on slice N_B-1:  G^> = G^< + G^R - G^A
      cx<T>* GG = c.tmp(0);
      Term<T> t0; t0.p = c.gl(i); t0.s = bb; t0.alpha = 1.0;
      Term<T> t1; t1.p = c.g(i); t1.s = bb; t1.alpha = 1.0;
      Term<T> t2; t2.p = c.g(i); t2.s = bb; t2.alpha = -1.0; t2.op = OP_C;
      QTX_CK((combine<T, T>(GG, bb, t0, t1, t2, b, ne, nullptr, 0, 0, nullptr, st)));
      QTX_CK(obs_trace2<T>(con + 1, 2, SL_R, bb, GG, bb, SG_R, bb, c.gl(i), bb, b, ne, st));
    }
  }
  for (int i = nb - 2; i >= 0; --i) {
    cx<T>* GRn = c.g(i + 1);
    cx<T>* Pm = c.tmp(2);
    cx<T>* Z = c.keep_z() ? c.zk(i) : c.tmp(3);  // V_i g_i
    cx<T>* GRl = c.tmp(4);
    cx<T>* GRu = c.tmp(5);
    cx<T>* Qw = c.tmp(6);
    cx<T>* K = c.tmp(7);
    cx<T>* PGL = c.tmp(8);
    cx<T>* X2 = c.tmp(9);
    cx<T>* GLu = c.tmp(10);
    cx<T>* gi = c.g(i);
    if (d.storage_bits && i < nb - 2) {  // g_i, g^<_i back from FPX into the working blocks
      QTX_CK(fpx_load<T>(d.storage_bits, c.gfx(i), (long)ne * bb, gi, st));
      QTX_CK(fpx_load<T>(d.storage_bits, c.glfx(i), (long)ne * bb, c.gl(i), st));
    }
    auto MM = [&](const cx<T>* A, long sA_, int opA, const cx<T>* B, long sB_, int opB, const cx<T>* C0, cx<T>* C, double al, double be,
                  DigitHint h = DigitHint{}) {
      return gemm<T>(P, gargs<T>(b, b, b, A, b, sA_, opA, B, b, sB_, opB, C0, b, bb, C, b, bb, al, be, ne, nullptr), st, false, h);
    };
    // kept digit planes (tensor-core modes): slot 0 = P (left operand of three products), slot 1 =
    // G_{i+1,i+1} (left operand of two), slot 2 = Q (right operand of two)
    DigitHint x2;
    x2.a_slot = 1; x2.a_mode = DG_REUSE; x2.b_slot = 2; x2.b_mode = DG_REUSE;
    if ((s = MM(gi, bb, OP_N, U(i), sUV, OP_N, nullptr, Pm, 1.0, 0.0))) return s;
    if (!c.keep_z() && (s = MM(V(i), sUV, OP_N, gi, bb, OP_N, nullptr, Z, 1.0, 0.0))) return s;
    // block-tridiagonal right-hand side k: g_i L_k with L_k its upper block (g_i still left-connected)
    auto Rl = [&](int k) { return odg ? c.tmp(13 + k) : nullptr; };
    if (odg) {
      for (int k = 0; k < nrhs; ++k) {
        cx<T>* Lt = load_L(k, i);
        if (!Lt) return QTX_ERR_CUDA;
        if ((s = MM(gi, bb, OP_N, Lt, sLt, OP_N, nullptr, Rl(k), 1.0, 0.0))) return s;
      }
    }
    if ((s = MM(GRn, bb, OP_N, Z, bb, OP_N, nullptr, GRl, -1.0, 0.0, keepA(1)))) return s;
    if ((s = MM(Pm, bb, OP_N, GRn, bb, OP_N, nullptr, GRu, -1.0, 0.0, keepA(0)))) return s;
    if ((s = MM(Pm, bb, OP_N, GRl, bb, OP_N, gi, gi, -1.0, 1.0, reuseA(0)))) return s;   // g_i <- G_ii
    if (want(QTX_OUT_GR_DIAG, out->GR_diag) && (s = emit<T>(P, out->GR_diag, nb, i, e0, gi, b, ne, st))) return s;
    if (want(QTX_OUT_GR_UPPER, out->GR_upper) && (s = emit<T>(P, out->GR_upper, nb - 1, i, e0, GRu, b, ne, st))) return s;
    if (want(QTX_OUT_GR_LOWER, out->GR_lower) && (s = emit<T>(P, out->GR_lower, nb - 1, i, e0, GRl, b, ne, st))) return s;
    // lesser-type blocks of each right-hand side on the shared retarded ones
    for (int k = 0; k < nrhs; ++k) {
      cx<T>* gli = c.glk(k, i);
      cx<T>* GLn = c.glk(k, i + 1);
      // Q = V_i g^<_i: the forward sweep's X of slice i + 1 when kept
      cx<T>* Q = c.keep_z() ? c.xk(k, i) : Qw;
      if (!c.keep_z() && (s = MM(V(i), sUV, OP_N, gli, bb, OP_N, nullptr, Q, 1.0, 0.0))) return s;
      if (odg) {  // Q = V_i g^<_i + (g_i Sigma^<_{i,i+1})^H
        Term<T> t0; t0.p = Q; t0.s = bb; t0.alpha = 1.0;
        Term<T> t1; t1.p = Rl(k); t1.s = bb; t1.alpha = 1.0; t1.op = OP_C;
        QTX_CK((combine<T, T>(Q, bb, t0, t1, none, b, ne, nullptr, 0, 0, nullptr, st)));
      }
      if ((s = MM(GRu, bb, OP_N, Q, bb, OP_N, nullptr, K, -1.0, 0.0, keepB(2)))) return s;
      if ((s = MM(Pm, bb, OP_N, GLn, bb, OP_N, nullptr, PGL, 1.0, 0.0, reuseA(0)))) return s;
      if ((s = MM(PGL, bb, OP_N, Pm, bb, OP_C, gli, gli, 1.0, 1.0))) return s;   // g^<_i + PGL P^H
      if ((s = MM(GRn, bb, OP_N, Q, bb, OP_N, nullptr, X2, 1.0, 0.0, x2))) return s;
      {
        Term<T> t0; t0.p = gli; t0.s = bb; t0.alpha = 1.0;
        Term<T> t1; t1.p = K; t1.s = bb; t1.alpha = 1.0;
        Term<T> t2; t2.p = K; t2.s = bb; t2.alpha = -1.0; t2.op = OP_C;
        QTX_CK((combine<T, T>(gli, bb, t0, t1, t2, b, ne, nullptr, 0, 0, nullptr, st)));   // G^<_ii
        Term<T> u0; u0.p = PGL; u0.s = bb; u0.alpha = -1.0;
        Term<T> u1; u1.p = X2; u1.s = bb; u1.alpha = 1.0; u1.op = OP_C;
        QTX_CK((combine<T, T>(GLu, bb, u0, u1, none, b, ne, nullptr, 0, 0, nullptr, st)));  // G^<_{i,i+1}
      }
      if (k == 1) {  // the second right-hand side's blocks are the GG outputs
        if (want(QTX_OUT_GG_DIAG, out->GG_diag) && (s = emit<T>(P, out->GG_diag, nb, i, e0, gli, b, ne, st))) return s;
        if (want(QTX_OUT_GG_UPPER, out->GG_upper) && (s = emit<T>(P, out->GG_upper, nb - 1, i, e0, GLu, b, ne, st))) return s;
        continue;
      }
      if (want(QTX_OUT_GL_DIAG, out->GL_diag) && (s = emit<T>(P, out->GL_diag, nb, i, e0, gli, b, ne, st))) return s;
      if (want(QTX_OUT_GL_UPPER, out->GL_upper) && (s = emit<T>(P, out->GL_upper, nb - 1, i, e0, GLu, b, ne, st))) return s;
      if (!d.second_rhs) {
        if (want(QTX_OUT_GG_DIAG, out->GG_diag) && (s = emit<T>(P, out->GG_diag, nb, i, e0, gli, b, ne, st, gi, gi))) return s;
        if (want(QTX_OUT_GG_UPPER, out->GG_upper) && (s = emit<T>(P, out->GG_upper, nb - 1, i, e0, GLu, b, ne, st, GRu, GRl))) return s;
      }
      if (!d.system_input)
        QTX_CK(obs_current<T>(cur + i, ncur, Hu + (long)i * bb, Su ? Su + (long)i * bb : nullptr, GLu, bb, c.E, b, ne, st,
                              reinterpret_cast<double*>(c.tmp(0)), (long)ne * bb * (long)sizeof(cx<T>) / (long)sizeof(double)));
      QTX_CK(obs_density<T>(den + i, nb, gli, bb, b, ne, st));
      if (cont)
        QTX_CK(obs_balance<T>(bal + i, bscale + i, bgn + i, bhn + i, nb, sigL(i), sigR(i), sSig, gi, gli, bb, eta, b,
                              ne, st, Hd + (long)i * bb, Hu + (long)i * bb, Su ? Su + (long)i * bb : nullptr, c.E, GLu));
    }
  }
  if (d.leads) {  // left contact current and transmission on slice 0
    cx<T>* GG = c.tmp(0);
    Term<T> t0; t0.p = c.gl(0); t0.s = bb; t0.alpha = 1.0;
    Term<T> t1; t1.p = c.g(0); t1.s = bb; t1.alpha = 1.0;
    Term<T> t2; t2.p = c.g(0); t2.s = bb; t2.alpha = -1.0; t2.op = OP_C;
    QTX_CK((combine<T, T>(GG, bb, t0, t1, t2, b, ne, nullptr, 0, 0, nullptr, st)));
    QTX_CK(obs_trace2<T>(con, 2, SL_L, bb, GG, bb, SG_L, bb, c.gl(0), bb, b, ne, st));
    // T = Tr[Gam A_00] - Tr[Gam G Gam G^H] with A = i (G - G^H): Tr[Gam A] = -Im Tr[Gam (G - G^H)],
    // and Tr[Gam G Gam G^H] = sum_jk (Gam G)_jk conj((G Gam)_jk) since Gam is Hermitian (FP64).
    cx<double>* D = reinterpret_cast<cx<double>*>(P->ws + P->L.dec);
    cx<double>* G64 = D;
    cx<double>* X1 = D + (size_t)P->Ec * bb;
    cx<double>* X2 = X1 + (size_t)P->Ec * bb;
    cx<double>* Dm = X2 + (size_t)P->Ec * bb;
    Term<T> tg; tg.p = c.g(0); tg.s = bb; tg.alpha = 1.0;
    QTX_CK((combine<T, double>(G64, bb, tg, none, none, b, ne, nullptr, 0, 0, nullptr, st)));
    Term<double> a0; a0.p = G64; a0.s = bb; a0.alpha = 1.0;
    Term<double> a1; a1.p = G64; a1.s = bb; a1.alpha = -1.0; a1.op = OP_C;
    Term<double> nn;
    QTX_CK((combine<double, double>(Dm, bb, a0, a1, nn, b, ne, nullptr, 0, 0, nullptr, st)));
    QTX_CK(obs_trace2<double>(tra, 1, Gam_L, bb, Dm, bb, nullptr, 0, nullptr, 0, b, ne, st, 1, -1.0));
    if ((s = gemm<double>(P, gargs<double>(b, b, b, Gam_L, b, bb, OP_N, G64, b, bb, OP_N, nullptr, 0, 0, X1, b, bb, 1.0, 0.0, ne, nullptr), st, true))) return s;
    if ((s = gemm<double>(P, gargs<double>(b, b, b, G64, b, bb, OP_N, Gam_L, b, bb, OP_N, nullptr, 0, 0, X2, b, bb, 1.0, 0.0, ne, nullptr), st, true))) return s;
    QTX_CK(obs_frob_dot(tra, 1, X1, bb, X2, bb, -1.0, b, ne, st));
  }
  // ---- continuity residual per energy (and the escalation flags)
  if (cont) {
    double* cres = reinterpret_cast<double*>(P->ws + P->L.cres);
    int* cflag = reinterpret_cast<int*>(P->ws + P->L.cflag);
    // unit error of the products in this mode (Eq. 6: error ~ kappa eps): 6 (7) bf16 digits ~41 bits,
    // 2 digits ~13 bits, complex64 24 bits, FP64 53
    const double eps_mode = std::is_same<T, double>::value ? 0x1p-53
                            : std::is_same<T, float>::value  ? 0x1p-24
                            : (d.precision == QTX_BF16X3 ? 0x1p-13 : 0x1p-40);
    QTX_CK(continuity(cur, ncur, bal, bscale, bgn, bhn, nb, d.leads ? con : nullptr, c.E, nb, ne,
                      d.escalate_tol > 0 ? d.escalate_tol : 1e300, eps_mode, cres, cflag, st));
    if (want(QTX_OUT_CONTINUITY, out->continuity))
      QTX_CK(cudaMemcpyAsync(out->continuity + e0, cres, (size_t)ne * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  // ---- 4. outputs of the per-energy observables and their integrals
  const int nbm1 = nb - 1;
  if (want(QTX_OUT_CURRENT, out->current) && nbm1 > 0)
    QTX_CK(cudaMemcpyAsync(out->current + (size_t)e0 * nbm1, cur, (size_t)ne * nbm1 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (want(QTX_OUT_DENSITY, out->density))
    QTX_CK(cudaMemcpyAsync(out->density + (size_t)e0 * nb, den, (size_t)ne * nb * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (d.leads && want(QTX_OUT_CONTACT, out->contact))
    QTX_CK(cudaMemcpyAsync(out->contact + (size_t)e0 * 2, con, (size_t)ne * 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (d.leads && want(QTX_OUT_TRANSMISSION, out->transmission))
    QTX_CK(cudaMemcpyAsync(out->transmission + e0, tra, (size_t)ne * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (m & QTX_OUT_INTEGRALS) {
    if (out->current_int && nbm1 > 0)
      QTX_CK(integrate_add(out->current_int, cur, nbm1, nbm1, in->weights, in->energies, e0, in->n_energies, ne, 1.0, st));
    if (out->density_int)
      QTX_CK(integrate_add(out->density_int, den, nb, nb, in->weights, in->energies, e0, in->n_energies, ne, 1.0 / (2.0 * 3.14159265358979323846), st));
  }
  return QTX_OK;
}

template <typename T>
qtx_status solve_all(qtx_rgf_plan_s* P, const qtx_rgf_inputs* in, const qtx_rgf_outputs* out, cudaStream_t st) {
  const int nb = P->nb;
  const unsigned m = P->d.outputs;
  if ((m & QTX_OUT_INTEGRALS) && out->current_int && nb > 1)
    QTX_CK(cudaMemsetAsync(out->current_int, 0, (size_t)(nb - 1) * sizeof(double), st));
  if ((m & QTX_OUT_INTEGRALS) && out->density_int)
    QTX_CK(cudaMemsetAsync(out->density_int, 0, (size_t)nb * sizeof(double), st));
  int* chunk_status = reinterpret_cast<int*>(P->ws + P->L.flags) + 2 * P->Ec;
  P->status_host.assign(in->n_energies, 0);
  for (int e0 = 0; e0 < in->n_energies; e0 += P->Ec) {
    const int ne = std::min(P->Ec, in->n_energies - e0);
    int* status = out->status_per_energy ? out->status_per_energy + e0 : chunk_status;
    QTX_CK(cudaMemsetAsync(status, 0, (size_t)ne * sizeof(int), st));
    if (out->escalated) QTX_CK(cudaMemsetAsync(out->escalated + e0, 0, (size_t)ne * sizeof(int), st));
    qtx_status s = solve_chunk<T>(P, in, out, e0, ne, status, st);
    if (s) return s;
    if (!std::is_same<T, double>::value && P->d.escalate_tol > 0) {
      // energies whose current is not conserved to escalate_tol are solved again in FP64
      QTX_CK(cudaMemcpyAsync(P->h_flag, P->ws + P->L.cflag, sizeof(int) * ne, cudaMemcpyDeviceToHost, st));
      QTX_CK(cudaStreamSynchronize(st));
      std::vector<int> redo;
      for (int k = 0; k < ne; ++k)
        if (P->h_flag[k]) redo.push_back(k);
      if (!redo.empty()) {
        // take their integral contributions back out first (the chunk's per-energy values are still
        // in the observable buffers; each FP64 re-solve adds its own)
        const int nbm1 = nb - 1, ncur = nb > 1 ? nb - 1 : 1;
        double* cur = reinterpret_cast<double*>(P->ws + P->L.obs);
        double* den = cur + (size_t)P->Ec * ncur;
        if ((m & QTX_OUT_INTEGRALS) && out->current_int && nbm1 > 0)
          for (int k : redo)
            QTX_CK(integrate_add(out->current_int, cur + (size_t)k * ncur, ncur, nbm1, in->weights, in->energies, e0 + k,
                                 in->n_energies, 1, -1.0, st));
        if ((m & QTX_OUT_INTEGRALS) && out->density_int)
          for (int k : redo)
            QTX_CK(integrate_add(out->density_int, den + (size_t)k * nb, nb, nb, in->weights, in->energies, e0 + k,
                                 in->n_energies, 1, -1.0 / (2.0 * 3.14159265358979323846), st));
        for (int k : redo) {
          QTX_CK(cudaMemsetAsync(status + k, 0, sizeof(int), st));
          if ((s = solve_chunk<double>(P, in, out, e0 + k, 1, status + k, st))) return s;
          if (out->escalated) QTX_CK(fill_int(out->escalated + e0 + k, 1, 1, st));
        }
      }
    }
    if (!out->status_per_energy) {
      // keep the worst chunk status without a host sync: fold into the error flag word
      QTX_CK(cudaMemcpyAsync(P->h_status, status, sizeof(int) * ne, cudaMemcpyDeviceToHost, st));
      QTX_CK(cudaStreamSynchronize(st));
      for (int k = 0; k < ne; ++k) P->worst = std::max(P->worst, P->h_status[k]);
    }
  }
  return QTX_OK;
}

qtx_status validate(const qtx_rgf_desc* d, std::string& err) {
  if (!d) { err = "desc is NULL"; return QTX_ERR_INVALID_ARG; }
  if (d->n_blocks < 1) { err = "n_blocks must be >= 1"; return QTX_ERR_INVALID_ARG; }
  if (d->block_size < 1 || d->block_size > 4096) { err = "block_size must be in [1, 4096]"; return QTX_ERR_INVALID_ARG; }
  if (d->max_energies_in_flight < 1) { err = "max_energies_in_flight must be >= 1"; return QTX_ERR_INVALID_ARG; }
  if (d->precision < QTX_FP64 || d->precision > QTX_EMU64) { err = "unknown precision"; return QTX_ERR_INVALID_ARG; }
  if (d->leads && (d->decim_max_iter < 1 || !(d->decim_tol > 0))) { err = "leads need decim_max_iter >= 1 and decim_tol > 0"; return QTX_ERR_INVALID_ARG; }
  if (d->refine_max_iter < 0) { err = "refine_max_iter must be >= 0"; return QTX_ERR_INVALID_ARG; }
  if (!(d->refine_tol >= 0.0)) { err = "refine_tol must be >= 0"; return QTX_ERR_INVALID_ARG; }
  if (d->offdiag_sigma && !d->has_scattering) { err = "offdiag_sigma needs has_scattering"; return QTX_ERR_INVALID_ARG; }
  if (d->storage_bits && !fpx_width_ok(d->storage_bits)) { err = "storage_bits must be 0, 56, 48, 40, 32, 24 or 16"; return QTX_ERR_INVALID_ARG; }
  if (d->sigma_stream && (!d->has_scattering || !d->energy_dependent_sigma || d->offdiag_sigma)) { err = "sigma_stream needs has_scattering and energy_dependent_sigma, without offdiag_sigma"; return QTX_ERR_INVALID_ARG; }
  if (d->second_rhs && (!d->system_input || d->storage_bits)) { err = "second_rhs needs system_input and storage_bits = 0"; return QTX_ERR_INVALID_ARG; }
  if (!(d->escalate_tol >= 0.0)) { err = "escalate_tol must be >= 0"; return QTX_ERR_INVALID_ARG; }
  if (d->tc_stages < 0 || d->tc_ctas < 0) { err = "tc_stages and tc_ctas must be >= 0"; return QTX_ERR_INVALID_ARG; }
  if ((d->escalate_tol > 0 || (d->outputs & QTX_OUT_CONTINUITY)) && (d->offdiag_sigma || d->system_input || d->sigma_stream)) {
    err = "the continuity check (escalate_tol, QTX_OUT_CONTINUITY) needs block-diagonal Sigma, no system_input and no sigma_stream";
    return QTX_ERR_INVALID_ARG;
  }
  if (d->system_input) {
    const unsigned bad = (d->second_rhs ? 0u : QTX_OUT_GG_DIAG | QTX_OUT_GG_UPPER) | QTX_OUT_CURRENT | QTX_OUT_CONTACT | QTX_OUT_TRANSMISSION | QTX_OUT_INTEGRALS;
    if (d->has_S || d->leads || d->sigma_stream) { err = "system_input needs has_S = 0, leads = 0, sigma_stream = 0"; return QTX_ERR_INVALID_ARG; }
    if (d->outputs & bad) { err = "system_input produces no G^> (without second_rhs), current, contact, transmission or integrals outputs"; return QTX_ERR_INVALID_ARG; }
  }
  if ((d->precision == QTX_EMU64 || d->precision == QTX_BF16X3) && !tc_available()) {
    err = "tensor-core engine not compiled into the library";
    return QTX_ERR_UNSUPPORTED;
  }
  return QTX_OK;
}

}  // namespace

// ----------------------------------------------------------------------------- W-system assembly
// Table I, W row: per energy the BT blocks of M = I - V P^R and B^<> = V P^<> V^H from the exact
// block products of the BT factors.  Row i of V P is (V P)_ij = sum_k V_ik P_kj over k = i-1..i+1
// with |k - j| <= 1 (j = i-1..i+1 for M; i-2..i+2 for B, whose blocks B_ij = sum_l (V P)_il
// (V_jl)^H need l up to j+1).  Each block product is one batched launch over the chunk's energies,
// V shared (batch stride 0).  Temporaries: 0-4 V blocks, 5 one P block, 6-10 row i of V P, 11 B.
template <typename T>
qtx_status w_assemble_chunk(qtx_rgf_plan_s* P, const qtx_w_inputs* in, const qtx_w_outputs* out, int nb,
                            int e0, int ne, cudaStream_t st) {
  const int b = P->b;
  const long bb = P->bb, nu = nb - 1;
  Ctx<T> c{P, st, ne, nullptr, nullptr, bb, b};
  const cx<double>* Vd = reinterpret_cast<const cx<double>*>(in->V_diag);
  const cx<double>* Vu = reinterpret_cast<const cx<double>*>(in->V_upper);
  // block j of a per-energy array [N_E][n][b][b], first energy of the chunk
  auto pe = [&](const void* X, long n, long j) {
    return reinterpret_cast<const cx<double>*>(X) + ((long)e0 * n + j) * bb;
  };
  // V slots: 0 V_ii, 1 V_{i+1,i+1}, 2 V_{i-1,i}, 3 V_{i,i+1}, 4 V_{i+1,i+2}
  cx<T>* Vt[5] = {c.tmp(0), c.tmp(1), c.tmp(2), c.tmp(3), c.tmp(4)};
  cx<T>* Pt = c.tmp(5);
  cx<T>* acc[5] = {c.tmp(6), c.tmp(7), c.tmp(8), c.tmp(9), c.tmp(10)};  // (V P)_{i,i-2} .. (V P)_{i,i+2}
  cx<T>* Bt = c.tmp(11);
  auto toT = [&](cx<T>* dst, const cx<double>* src, long sSrc, int batch) {
    return axpby_from64<T>(dst, bb, src, sSrc, 1.0, nullptr, 0, 0.0, b, batch, st);
  };
  auto mm = [&](const cx<T>* A, long sA, int opA, const cx<T>* B, long sB, int opB, cx<T>* C, double al,
                bool first) {
    return gemm<T>(P, gargs<T>(b, b, b, A, b, sA, opA, B, b, sB, opB, first ? nullptr : C, b, bb, C, b, bb, al,
                               first ? 0.0 : 1.0, ne, nullptr), st);
  };
  // out[e][j] = alpha X (+ I), complex128, n blocks per energy
  auto emit64 = [&](void* dst, long n, long j, const cx<T>* X, double alpha, bool ident) -> qtx_status {
    cx<double>* o = reinterpret_cast<cx<double>*>(dst) + ((long)e0 * n + j) * bb;
    Term<T> t0; t0.p = X; t0.s = bb; t0.alpha = alpha;
    Term<T> none;
    QTX_CK((combine<T, double>(o, n * bb, t0, none, none, b, ne, nullptr, 0.0, 0.0, nullptr, st)));
    if (ident) QTX_CK(add_identity<double>(o, n * bb, b, ne, nullptr, st));
    return QTX_OK;
  };
  qtx_status s;
  for (int i = 0; i < nb; ++i) {
    QTX_CK(toT(Vt[0], Vd + (long)i * bb, 0, 1));
    if (i + 1 < nb) QTX_CK(toT(Vt[1], Vd + (long)(i + 1) * bb, 0, 1));
    if (i >= 1) QTX_CK(toT(Vt[2], Vu + (long)(i - 1) * bb, 0, 1));
    if (i + 1 < nb) QTX_CK(toT(Vt[3], Vu + (long)i * bb, 0, 1));
    if (i + 2 < nb) QTX_CK(toT(Vt[4], Vu + (long)(i + 1) * bb, 0, 1));
    // row i of V P for j = i-W .. i+W.  V_ik: k = i-1 -> V_{i-1,i}^H, k = i -> V_ii, k = i+1 -> V_{i,i+1}.
    // P_kj: diagonal, upper (j = k+1), lower (j = k-1): given, or -(P_{j,j+1})^H for anti-Hermitian P.
    auto row = [&](const void* Pd, const void* Pu, const void* Pl, int W) -> qtx_status {
      for (int dj = -W; dj <= W; ++dj) {
        const int j = i + dj;
        if (j < 0 || j >= nb) continue;
        bool first = true;
        for (int k = i - 1; k <= i + 1; ++k) {
          if (k < 0 || k >= nb || k - j > 1 || j - k > 1) continue;
          const cx<T>* Vk = k == i ? Vt[0] : (k == i + 1 ? Vt[3] : Vt[2]);
          const int opV = k == i - 1 ? OP_C : OP_N;
          int opP = OP_N;
          double al = 1.0;
          if (k == j) QTX_CK(toT(Pt, pe(Pd, nb, k), (long)nb * bb, ne));
          else if (j == k + 1) QTX_CK(toT(Pt, pe(Pu, nu, k), nu * bb, ne));
          else if (Pl) QTX_CK(toT(Pt, pe(Pl, nu, j), nu * bb, ne));
          else {
            QTX_CK(toT(Pt, pe(Pu, nu, j), nu * bb, ne));
            opP = OP_C;
            al = -1.0;
          }
          if ((s = mm(Vk, 0, opV, Pt, bb, opP, acc[dj + 2], al, first))) return s;
          first = false;
        }
      }
      return QTX_OK;
    };
    // M_ii = I - (V P^R)_ii, M_{i,i+1} = -(V P^R)_{i,i+1}, M_{i,i-1} = -(V P^R)_{i,i-1}
    if ((s = row(in->PR_diag, in->PR_upper, in->PR_lower, 1))) return s;
    if ((s = emit64(out->M_diag, nb, i, acc[2], -1.0, true))) return s;
    if (i + 1 < nb && (s = emit64(out->M_upper, nu, i, acc[3], -1.0, false))) return s;
    if (i >= 1 && (s = emit64(out->M_lower, nu, i - 1, acc[1], -1.0, false))) return s;
    for (int kind = 0; kind < 2; ++kind) {
      const void* Pd = kind ? in->PG_diag : in->PL_diag;
      const void* Pu = kind ? in->PG_upper : in->PL_upper;
      void* Od = kind ? out->BG_diag : out->BL_diag;
      void* Ou = kind ? out->BG_upper : out->BL_upper;
      if (!Pd) continue;
      if ((s = row(Pd, Pu, nullptr, 2))) return s;
      // B_ii = sum_l (V P)_il (V_il)^H, l = i-1..i+1:  (V_{i,i-1})^H = V_{i-1,i}, V_ii^H, V_{i,i+1}^H
      bool first = true;
      for (int l = i - 1; l <= i + 1; ++l) {
        if (l < 0 || l >= nb) continue;
        const cx<T>* Vl = l == i ? Vt[0] : (l == i + 1 ? Vt[3] : Vt[2]);
        if ((s = mm(acc[l - i + 2], bb, OP_N, Vl, 0, l == i - 1 ? OP_N : OP_C, Bt, 1.0, first))) return s;
        first = false;
      }
      if ((s = emit64(Od, nb, i, Bt, 1.0, false))) return s;
      if (i + 1 < nb) {
        // B_{i,i+1} = sum_l (V P)_il (V_{i+1,l})^H, l = i..i+2:  V_{i,i+1}, V_{i+1,i+1}^H, V_{i+1,i+2}^H
        first = true;
        for (int l = i; l <= i + 2 && l < nb; ++l) {
          const cx<T>* Vl = l == i ? Vt[3] : (l == i + 1 ? Vt[1] : Vt[4]);
          if ((s = mm(acc[l - i + 2], bb, OP_N, Vl, 0, l == i ? OP_N : OP_C, Bt, 1.0, first))) return s;
          first = false;
        }
        if ((s = emit64(Ou, nu, i, Bt, 1.0, false))) return s;
      }
    }
  }
  return QTX_OK;
}

extern "C" {

qtx_status qtx_rgf_plan_create(const qtx_rgf_desc* desc, qtx_rgf_plan* out) {
  if (!out) { g_create_error = "out is NULL"; return QTX_ERR_INVALID_ARG; }
  *out = nullptr;
  std::string err;
  qtx_status s = validate(desc, err);
  if (s) { g_create_error = err; return s; }
  auto* P = new qtx_rgf_plan_s();
  P->d = *desc;
  P->b = desc->block_size;
  P->nb = desc->n_blocks;
  P->Ec = desc->max_energies_in_flight;
  P->bb = (long)P->b * P->b;
  P->esz = desc->precision == QTX_FP32 ? sizeof(cx<float>) : sizeof(cx<double>);
  P->L = make_layout(*desc);
  cudaError_t e = cudaMalloc(&P->ws, P->L.total);
  if (e != cudaSuccess) {
    g_create_error = std::string("workspace cudaMalloc(") + std::to_string(P->L.total) + "): " + cudaGetErrorString(e);
    cudaGetLastError();
    delete P;
    return QTX_ERR_OOM;
  }
  e = cudaMalloc(&P->d_err_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(P->d_err_flag, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&P->h_status, sizeof(int) * P->Ec);
  if (e == cudaSuccess && desc->escalate_tol > 0) e = cudaMallocHost(&P->h_flag, sizeof(int) * P->Ec);
  // identity block for the refinement residual
  if (e == cudaSuccess) {
    std::vector<cx<double>> I((size_t)P->bb, mk<double>(0, 0));
    for (int i = 0; i < P->b; ++i) I[(size_t)i * P->b + i] = mk<double>(1, 0);
    e = cudaMemcpy(P->ws + P->L.ident, I.data(), I.size() * sizeof(cx<double>), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      std::vector<float> Idf((size_t)P->bb * 4, 0.f);  // (re.hi, re.lo, im.hi, im.lo)
      for (int i = 0; i < P->b; ++i) Idf[((size_t)i * P->b + i) * 4] = 1.f;
      e = cudaMemcpy(P->ws + P->L.ident_df, Idf.data(), Idf.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
  }
  if (e != cudaSuccess) {
    g_create_error = std::string("plan setup: ") + cudaGetErrorString(e);
    cudaFree(P->ws);
    if (P->d_err_flag) cudaFree(P->d_err_flag);
    if (P->h_status) cudaFreeHost(P->h_status);
    if (P->h_flag) cudaFreeHost(P->h_flag);
    delete P;
    return QTX_ERR_CUDA;
  }
  *out = P;
  return QTX_OK;
}

qtx_status qtx_rgf_solve(qtx_rgf_plan P, const qtx_rgf_inputs* in, const qtx_rgf_outputs* out, void* stream) {
  if (!P) return QTX_ERR_INVALID_ARG;
  if (!in || !out) { P->err = "inputs/outputs NULL"; return QTX_ERR_INVALID_ARG; }
  if (in->n_energies < 1 || !in->energies) { P->err = "need n_energies >= 1 and an energies array"; return QTX_ERR_INVALID_ARG; }
  const int nbs = in->n_blocks ? in->n_blocks : P->d.n_blocks;
  if (P->d.system_input) {
    if (!in->M_diag || (nbs > 1 && (!in->M_upper || !in->M_lower))) { P->err = "system_input set but M blocks missing"; return QTX_ERR_INVALID_ARG; }
  } else if (!in->H_diag || (nbs > 1 && !in->H_upper)) { P->err = "H_diag / H_upper missing"; return QTX_ERR_INVALID_ARG; }
  if (P->d.has_S && (!in->S_diag || (P->nb > 1 && !in->S_upper))) { P->err = "has_S set but S pointers missing"; return QTX_ERR_INVALID_ARG; }
  if (P->d.has_scattering && (!in->SigL_diag || (!P->d.system_input && !in->SigR_diag))) { P->err = "has_scattering set but Sigma pointers missing"; return QTX_ERR_INVALID_ARG; }
  if (P->d.offdiag_sigma && (in->n_blocks ? in->n_blocks : P->d.n_blocks) > 1 &&
      (!in->SigL_upper || (!P->d.system_input && (!in->SigR_upper || !in->SigR_lower)))) { P->err = "offdiag_sigma set but off-diagonal Sigma pointers missing"; return QTX_ERR_INVALID_ARG; }
  if (P->d.second_rhs && (!in->SigG_diag || (P->d.offdiag_sigma && nbs > 1 && !in->SigG_upper))) { P->err = "second_rhs set but SigG blocks missing"; return QTX_ERR_INVALID_ARG; }
  if (P->d.leads && (!in->lead_H00_L || !in->lead_H01_L || !in->lead_H00_R || !in->lead_H01_R)) { P->err = "leads set but lead blocks missing"; return QTX_ERR_INVALID_ARG; }
  if (P->d.leads && !(in->kT > 0)) { P->err = "leads need kT > 0"; return QTX_ERR_INVALID_ARG; }
  if (in->n_blocks < 0 || in->n_blocks > P->d.n_blocks) { P->err = "inputs->n_blocks exceeds the plan's n_blocks"; return QTX_ERR_INVALID_ARG; }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  P->last = st;
  P->worst = 0;
  // the bounded-wait flag of the tensor-core launches starts clear for every solve
  if (cudaMemsetAsync(P->d_err_flag, 0, sizeof(int), st) != cudaSuccess) {
    P->err = "clearing the wait flag failed";
    cudaGetLastError();
    return QTX_ERR_CUDA;
  }
  // the workspace is laid out for the plan's n_blocks; a shorter device uses its first slices
  P->nb = in->n_blocks ? in->n_blocks : P->d.n_blocks;
  qtx_status s;
  if (P->d.precision == QTX_FP32) s = solve_all<float>(P, in, out, st);
  else if (P->d.precision == QTX_FP64) s = solve_all<double>(P, in, out, st);
  else s = solve_all<df>(P, in, out, st);
  P->nb = P->d.n_blocks;
  if (s == QTX_OK) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { P->err = cudaGetErrorString(e); return QTX_ERR_CUDA; }
  }
  P->out_status = out->status_per_energy;
  P->out_status_n = in->n_energies;
  return s;
}

qtx_status qtx_w_assemble(qtx_rgf_plan P, const qtx_w_inputs* in, const qtx_w_outputs* out, void* stream) {
  if (!P) return QTX_ERR_INVALID_ARG;
  if (!in || !out) { P->err = "inputs/outputs NULL"; return QTX_ERR_INVALID_ARG; }
  const int nb = in->n_blocks ? in->n_blocks : P->d.n_blocks;
  if (in->n_blocks < 0 || nb > P->d.n_blocks || in->n_energies < 1) { P->err = "n_blocks / n_energies out of range"; return QTX_ERR_INVALID_ARG; }
  if (!in->V_diag || !in->PR_diag || !in->PL_diag || !out->M_diag || !out->BL_diag) { P->err = "W assembly: diagonal blocks missing"; return QTX_ERR_INVALID_ARG; }
  if (nb > 1 && (!in->V_upper || !in->PR_upper || !in->PR_lower || !in->PL_upper || !out->M_upper || !out->M_lower || !out->BL_upper)) {
    P->err = "W assembly: off-diagonal blocks missing";
    return QTX_ERR_INVALID_ARG;
  }
  const bool pg = in->PG_diag != nullptr;
  if ((!pg && in->PG_upper) || (pg && ((nb > 1 && !in->PG_upper) || !out->BG_diag || (nb > 1 && !out->BG_upper)))) {
    P->err = "W assembly: P^> (diagonal and upper) and B^> must come together";
    return QTX_ERR_INVALID_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  P->last = st;
  if (cudaMemsetAsync(P->d_err_flag, 0, sizeof(int), st) != cudaSuccess) {
    P->err = "clearing the wait flag failed";
    cudaGetLastError();
    return QTX_ERR_CUDA;
  }
  for (int e0 = 0; e0 < in->n_energies; e0 += P->Ec) {
    const int ne = std::min(P->Ec, in->n_energies - e0);
    qtx_status s;
    if (P->d.precision == QTX_FP32) s = w_assemble_chunk<float>(P, in, out, nb, e0, ne, st);
    else if (P->d.precision == QTX_FP64) s = w_assemble_chunk<double>(P, in, out, nb, e0, ne, st);
    else s = w_assemble_chunk<df>(P, in, out, nb, e0, ne, st);
    if (s) return s;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { P->err = cudaGetErrorString(e); return QTX_ERR_CUDA; }
  return QTX_OK;
}

qtx_status qtx_rgf_status(qtx_rgf_plan P) {
  if (!P) return QTX_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(P->last);
  if (e != cudaSuccess) { P->err = cudaGetErrorString(e); return QTX_ERR_CUDA; }
  int flag = 0;
  e = cudaMemcpy(&flag, P->d_err_flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) { P->err = cudaGetErrorString(e); return QTX_ERR_CUDA; }
  if (flag) { P->err = "tensor-core engine: bounded wait expired"; return QTX_ERR_TIMEOUT; }
  if (P->out_status) {
    P->status_host.assign(P->out_status_n, 0);
    e = cudaMemcpy(P->status_host.data(), P->out_status, sizeof(int) * P->out_status_n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { P->err = cudaGetErrorString(e); return QTX_ERR_CUDA; }
    for (int v : P->status_host) P->worst = std::max(P->worst, v);
  }
  return (qtx_status)P->worst;
}

qtx_status qtx_rgf_set_profiling(qtx_rgf_plan P, int enable) {
  if (!P) return QTX_ERR_INVALID_ARG;
  P->prof = enable != 0;
  P->ev_used = 0;
  P->pipe_flops = P->useful_flops = 0.0;
  return QTX_OK;
}

qtx_status qtx_rgf_gemm_profile(qtx_rgf_plan P, long long* launches, double* ms, double* pipe_flops,
                                double* useful_flops) {
  if (!P) return QTX_ERR_INVALID_ARG;
  double tot = 0.0;
  for (size_t k = 0; k + 1 < P->ev_used; k += 2) {
    cudaError_t e = cudaEventSynchronize(P->ev_pool[k + 1]);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, P->ev_pool[k], P->ev_pool[k + 1]);
    if (e != cudaSuccess) { P->err = cudaGetErrorString(e); return QTX_ERR_CUDA; }
    tot += t;
  }
  if (launches) *launches = (long long)(P->ev_used / 2);
  if (ms) *ms = tot;
  if (pipe_flops) *pipe_flops = P->pipe_flops;
  if (useful_flops) *useful_flops = P->useful_flops;
  P->ev_used = 0;
  P->pipe_flops = P->useful_flops = 0.0;
  return QTX_OK;
}

long long qtx_kernel_launches(void) { return g_launches.load(); }

qtx_status qtx_rgf_destroy(qtx_rgf_plan P) {
  if (!P) return QTX_OK;
  for (cudaEvent_t e : P->ev_pool) cudaEventDestroy(e);
  if (P->ws) cudaFree(P->ws);
  if (P->d_err_flag) cudaFree(P->d_err_flag);
  if (P->h_status) cudaFreeHost(P->h_status);
  if (P->h_flag) cudaFreeHost(P->h_flag);
  delete P;
  return QTX_OK;
}

const char* qtx_rgf_last_error(qtx_rgf_plan P) { return P ? P->err.c_str() : g_create_error.c_str(); }

size_t qtx_rgf_footprint(const qtx_rgf_desc* desc) {
  std::string err;
  if (validate(desc, err) && validate(desc, err) != QTX_ERR_UNSUPPORTED) return 0;
  return make_layout(*desc).total;
}

const char* qtx_rgf_version(void) { return "qtx-rgf 0.1 (sm_103a)"; }

}  // extern "C"

// ============================================================================ component ABI
namespace {

template <typename T>
qtx_status zgemm_via(int precision, int M, int N, int K, int opA, const void* A, long lda, long sA, int opB,
                     const void* B, long ldb, long sB, double alpha, double beta, const void* C0, long ldc0,
                     long sC0, void* C, long ldc, long sC, int batch, cudaStream_t st, std::string& err) {
  const int rA = opA == OP_N ? M : K, cA = opA == OP_N ? K : M;
  const int rB = opB == OP_N ? K : N, cB = opB == OP_N ? N : K;
  const int nA = sA ? batch : 1, nB = sB ? batch : 1, nC0 = (C0 && beta != 0.0) ? (sC0 ? batch : 1) : 0;
  const size_t es = sizeof(cx<T>);
  void *a = nullptr, *b = nullptr, *c0 = nullptr, *c = nullptr, *scr = nullptr;
  int* flag = nullptr;
  const int digits = precision == QTX_EMU64 ? 6 : 2;
  const size_t scr_bytes = std::is_same<T, df>::value ? gemm_tc_scratch_bytes(M, N, K, batch, digits) : 0;
  cudaError_t e = cudaSuccess;
  qtx_status s = QTX_OK;
  auto CK = [&](cudaError_t x) {
    if (x != cudaSuccess && e == cudaSuccess) e = x;
    return x == cudaSuccess;
  };
  CK(cudaMallocAsync(&a, es * (size_t)nA * rA * cA, st));
  CK(cudaMallocAsync(&b, es * (size_t)nB * rB * cB, st));
  if (nC0) CK(cudaMallocAsync(&c0, es * (size_t)nC0 * M * N, st));
  CK(cudaMallocAsync(&c, es * (size_t)batch * M * N, st));
  if (scr_bytes) CK(cudaMallocAsync(&scr, scr_bytes, st));
  CK(cudaMallocAsync((void**)&flag, sizeof(int), st));
  if (e == cudaSuccess) {
    CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
    CK(convert_strided<double, T>((const cx<double>*)A, lda, sA, (cx<T>*)a, cA, (long)rA * cA, rA, cA, nA, st));
    CK(convert_strided<double, T>((const cx<double>*)B, ldb, sB, (cx<T>*)b, cB, (long)rB * cB, rB, cB, nB, st));
    if (nC0) CK(convert_strided<double, T>((const cx<double>*)C0, ldc0, sC0, (cx<T>*)c0, N, (long)M * N, M, N, nC0, st));
  }
  if (e == cudaSuccess) {
    if constexpr (std::is_same<T, df>::value) {
      TcArgs t;
      t.M = M; t.N = N; t.K = K;
      t.A = (const cx<df>*)a; t.lda = cA; t.sA = nA > 1 ? (long)rA * cA : 0; t.opA = opA;
      t.B = (const cx<df>*)b; t.ldb = cB; t.sB = nB > 1 ? (long)rB * cB : 0; t.opB = opB;
      t.C0 = nC0 ? (const cx<df>*)c0 : nullptr; t.ldc0 = N; t.sC0 = nC0 > 1 ? (long)M * N : 0;
      t.C = (cx<df>*)c; t.ldc = N; t.sC = (long)M * N;
      t.alpha = alpha; t.beta = nC0 ? beta : 0.0;
      t.batch = batch; t.active = nullptr;
      CK(gemm_tc(t, digits, scr, scr_bytes, flag, st));
    } else {
      GemmArgs<T> g;
      g.M = M; g.N = N; g.K = K;
      g.A = (const cx<T>*)a; g.lda = cA; g.sA = nA > 1 ? (long)rA * cA : 0; g.opA = opA;
      g.B = (const cx<T>*)b; g.ldb = cB; g.sB = nB > 1 ? (long)rB * cB : 0; g.opB = opB;
      g.C0 = nC0 ? (const cx<T>*)c0 : nullptr; g.ldc0 = N; g.sC0 = nC0 > 1 ? (long)M * N : 0;
      g.C = (cx<T>*)c; g.ldc = N; g.sC = (long)M * N;
      g.alpha = alpha; g.beta = nC0 ? beta : 0.0;
      g.batch = batch; g.active = nullptr;
      CK(gemm_simt<T>(g, st));
    }
    CK(convert_strided<T, double>((const cx<T>*)c, N, (long)M * N, (cx<double>*)C, ldc, sC, M, N, batch, st));
  }
  int hflag = 0;
  if (e == cudaSuccess) CK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  for (void* p : {a, b, c0, c, scr, (void*)flag})
    if (p) cudaFreeAsync(p, st);
  if (e == cudaSuccess) CK(cudaStreamSynchronize(st));
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    cudaGetLastError();
    return QTX_ERR_CUDA;
  }
  if (hflag) { err = "tensor-core engine: bounded wait expired"; s = QTX_ERR_TIMEOUT; }
  return s;
}

template <typename T>
qtx_status zinv_via(qtx_rgf_plan_s* P, int n, void* A, long sA, int batch, int* status, cudaStream_t st) {
  cx<T>* X = reinterpret_cast<cx<T>*>(P->ws + P->L.g);
  const long nn = (long)n * n;
  QTX_CK((convert_strided<double, T>((const cx<double>*)A, n, sA, X, n, nn, n, n, batch, st)));
  qtx_status s = block_inverse<T>(P, X, n, batch, nullptr, status, st);
  if (s) return s;
  QTX_CK((convert_strided<T, double>(X, n, nn, (cx<double>*)A, n, sA, n, n, batch, st)));
  return QTX_OK;
}
template <>
qtx_status zinv_via<double>(qtx_rgf_plan_s* P, int n, void* A, long sA, int batch, int* status, cudaStream_t st) {
  cx<double>* X = reinterpret_cast<cx<double>*>(P->ws + P->L.g);
  const long nn = (long)n * n;
  QTX_CK(cudaMemcpy2DAsync(X, nn * sizeof(cx<double>), A, sA * sizeof(cx<double>), nn * sizeof(cx<double>), batch,
                           cudaMemcpyDeviceToDevice, st));
  qtx_status s = block_inverse<double>(P, X, n, batch, nullptr, status, st);
  if (s) return s;
  QTX_CK(cudaMemcpy2DAsync(A, sA * sizeof(cx<double>), X, nn * sizeof(cx<double>), nn * sizeof(cx<double>), batch,
                           cudaMemcpyDeviceToDevice, st));
  return QTX_OK;
}

thread_local std::string g_kernel_error;

}  // namespace

extern "C" {

qtx_status qtx_zgemm_batched(int precision, int M, int N, int K, int opA, const void* A, long lda, long sA, int opB,
                             const void* B, long ldb, long sB, double alpha, double beta, const void* C0, long ldc0,
                             long sC0, void* C, long ldc, long sC, int batch, void* stream) {
  if (M < 0 || N < 0 || K < 0 || batch < 1 || !A || !B || !C || (beta != 0.0 && !C0) ||
      (opA != OP_N && opA != OP_C) || (opB != OP_N && opB != OP_C)) {
    g_kernel_error = "qtx_zgemm_batched: invalid argument";
    return QTX_ERR_INVALID_ARG;
  }
  if (M == 0 || N == 0) return QTX_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  switch (precision) {
    case QTX_FP64: return zgemm_via<double>(precision, M, N, K, opA, A, lda, sA, opB, B, ldb, sB, alpha, beta, C0, ldc0, sC0, C, ldc, sC, batch, st, g_kernel_error);
    case QTX_FP32: return zgemm_via<float>(precision, M, N, K, opA, A, lda, sA, opB, B, ldb, sB, alpha, beta, C0, ldc0, sC0, C, ldc, sC, batch, st, g_kernel_error);
    case QTX_EMU64:
    case QTX_BF16X3:
      if (!tc_available()) { g_kernel_error = "tensor-core engine needs an sm_103 GPU"; return QTX_ERR_UNSUPPORTED; }
      return zgemm_via<df>(precision, M, N, K, opA, A, lda, sA, opB, B, ldb, sB, alpha, beta, C0, ldc0, sC0, C, ldc, sC, batch, st, g_kernel_error);
    default:
      g_kernel_error = "unknown precision";
      return QTX_ERR_INVALID_ARG;
  }
}

qtx_status qtx_zinv_batched(int precision, int n, void* A, long sA, int batch, int refine_iter, int* status, void* stream) {
  if (n < 1 || n > 4096 || batch < 1 || !A || refine_iter < 0) return QTX_ERR_INVALID_ARG;
  qtx_rgf_desc d{};
  d.n_blocks = 1;
  d.block_size = n;
  d.max_energies_in_flight = batch;
  d.precision = (qtx_precision)precision;
  d.refine_max_iter = refine_iter;
  qtx_rgf_plan P = nullptr;
  qtx_status s = qtx_rgf_plan_create(&d, &P);
  if (s) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* stat = status;
  if (!stat) stat = reinterpret_cast<int*>(P->ws + P->L.flags);
  if (!status) cudaMemsetAsync(stat, 0, sizeof(int) * batch, st);
  if (precision == QTX_FP32) s = zinv_via<float>(P, n, A, sA, batch, stat, st);
  else if (precision == QTX_FP64) s = zinv_via<double>(P, n, A, sA, batch, stat, st);
  else s = zinv_via<df>(P, n, A, sA, batch, stat, st);
  cudaError_t e = cudaStreamSynchronize(st);
  qtx_rgf_destroy(P);
  if (s == QTX_OK && e != cudaSuccess) s = QTX_ERR_CUDA;
  return s;
}

qtx_status qtx_lead_self_energy(int n, const void* H00, const void* H01, const double* energies, int n_energies,
                                double eta, double tol, int max_iter, void* SigR, int* status, void* stream) {
  if (n < 1 || n > 4096 || n_energies < 1 || !H00 || !H01 || !energies || !SigR || max_iter < 1 || !(tol > 0))
    return QTX_ERR_INVALID_ARG;
  qtx_rgf_desc d{};
  d.n_blocks = 1;
  d.block_size = n;
  d.max_energies_in_flight = n_energies;
  d.precision = QTX_FP64;
  d.leads = 1;
  d.decim_tol = tol;
  d.decim_max_iter = max_iter;
  qtx_rgf_plan P = nullptr;
  qtx_status s = qtx_rgf_plan_create(&d, &P);
  if (s) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* stat = status ? status : reinterpret_cast<int*>(P->ws + P->L.flags) + 2 * P->Ec;
  cudaMemsetAsync(stat, 0, sizeof(int) * n_energies, st);
  Ctx<double> c{P, st, n_energies, energies, stat, (long)n * n, n};
  s = contact<double>(c, (const cx<double>*)H00, (const cx<double>*)H01, eta, (cx<double>*)SigR);
  cudaError_t e = cudaStreamSynchronize(st);
  qtx_rgf_destroy(P);
  if (s == QTX_OK && e != cudaSuccess) s = QTX_ERR_CUDA;
  return s;
}

}  // extern "C"

// ----------------------------------------------------------------------------- groups (uneven batches)
// Several plans -- devices of different N_B and b, each with its own energies -- solved together:
// every member's solve runs on its own host thread and stream, so the streams' launches overlap on
// the GPU.  With a pooling threshold of w > 0 waves, a tensor-core product is digitised on the
// member's stream; if it fills at least w waves of the GPU alone it is launched there at once,
// otherwise it is pooled: the member posts it and waits, and the pending products are launched
// together -- one persistent kernel over the union of their tiles, per kernel variant, at most
// kTcMaxGroup products a launch -- on the group's stream once they fill w waves, once every member
// still solving has posted one, or once the poster has waited kPoolWaitUs on the host.  Events order
// each pooled launch after its members' preceding work and before their following work.  The
// grouping only changes which launch computes a tile, never how, so every member's results equal
// its plan's solo solve bit for bit; the launches are plain stream work joined back to the caller's
// stream, so a group solve can be captured in a CUDA graph.  Pooling is off by default: its events
// hold the members in step, which costs more than the merged launches save.
constexpr int kPoolWaves = 0;  // default pooling threshold (qtx_rgf_group_set_pool_waves)
constexpr int kPoolWaitUs = 50;

struct qtx_rgf_group_s {
  std::vector<qtx_rgf_plan_s*> plans;
  std::vector<cudaStream_t> mst;     // member streams
  std::vector<cudaEvent_t> ready;    // per member: its work up to the posted product
  cudaStream_t gst = nullptr;        // launch stream of the pooled products
  std::vector<cudaEvent_t> done;     // ring of launch events
  size_t done_pos = 0;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaEvent_t gjoin = nullptr;
  long pool_tiles = 304;             // pooling threshold in tiles: waves x SMs
  int sms = 152;
  std::mutex mu;
  std::condition_variable cv;
  struct Req {
    TcPrepared p;
    int member = 0;
    bool released = false;
    cudaEvent_t after = nullptr;
    cudaError_t status = cudaSuccess;
  };
  std::vector<Req*> pending;
  long pending_tiles = 0;
  int live = 0;
  long long launches = 0, pooled_products = 0;
  std::string err;

  // with mu held: launch every pending product and release the posting threads
  void launch_pending() {
    cudaError_t e = cudaSuccess;
    for (Req* r : pending)
      if (e == cudaSuccess) e = cudaStreamWaitEvent(gst, ready[r->member], 0);
    std::vector<bool> taken(pending.size(), false);
    for (size_t i = 0; i < pending.size() && e == cudaSuccess; ++i) {
      if (taken[i]) continue;
      const TcPrepared* p[kTcMaxGroup];
      int n = 0;
      for (size_t j = i; j < pending.size() && n < kTcMaxGroup; ++j) {
        if (taken[j] || pending[j]->p.variant != pending[i]->p.variant) continue;
        taken[j] = true;
        p[n++] = &pending[j]->p;
      }
      e = gemm_tc_launch(p, n, gst);
      ++launches;
      pooled_products += n;
    }
    cudaEvent_t ev = done[done_pos++ % done.size()];
    if (e == cudaSuccess) e = cudaEventRecord(ev, gst);
    for (Req* r : pending) {
      r->after = ev;
      r->status = e;
      r->released = true;
    }
    pending.clear();
    pending_tiles = 0;
    cv.notify_all();
  }
};

namespace {

cudaError_t group_gemm(qtx_rgf_plan_s* P, const TcArgs& a, int digits, cudaStream_t st) {
  qtx_rgf_group_s* G = P->group;
  qtx_rgf_group_s::Req r;
  r.member = P->member;
  cudaError_t e = gemm_tc_prepare(a, digits, P->ws + P->L.tc_scratch, P->L.tc_bytes, P->d_err_flag, st, &r.p);
  if (e != cudaSuccess || r.p.tiles == 0) return e;
  if (r.p.tiles >= G->pool_tiles) {  // fills the GPU alone (or pooling is off)
    const TcPrepared* one[1] = {&r.p};
    return gemm_tc_launch(one, 1, st);
  }
  if ((e = cudaEventRecord(G->ready[P->member], st)) != cudaSuccess) return e;
  {
    std::unique_lock<std::mutex> lk(G->mu);
    G->pending.push_back(&r);
    G->pending_tiles += r.p.tiles;
    if (G->pending_tiles >= G->pool_tiles || (int)G->pending.size() == G->live) G->launch_pending();
    while (!r.released)
      if (!G->cv.wait_for(lk, std::chrono::microseconds(kPoolWaitUs), [&] { return r.released; }))
        G->launch_pending();
  }
  if (r.status != cudaSuccess) return r.status;
  return cudaStreamWaitEvent(st, r.after, 0);
}

// a member leaves the group when its solve has returned (successfully or not)
void group_leave(qtx_rgf_group_s* G) {
  std::unique_lock<std::mutex> lk(G->mu);
  --G->live;
  if (G->live > 0 && !G->pending.empty() && (int)G->pending.size() == G->live) G->launch_pending();
}

}  // namespace

extern "C" {

qtx_status qtx_rgf_group_create(int n_plans, const qtx_rgf_plan* plans, qtx_rgf_group* out) {
  if (!out || n_plans < 1 || !plans) return QTX_ERR_INVALID_ARG;
  *out = nullptr;
  for (int m = 0; m < n_plans; ++m)
    if (!plans[m] || plans[m]->group) return QTX_ERR_INVALID_ARG;
  auto* G = new qtx_rgf_group_s();
  G->plans.assign(plans, plans + n_plans);
  int dev = 0, sms = 152;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  G->pool_tiles = (long)kPoolWaves * sms;
  G->sms = sms;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G->gst, cudaStreamNonBlocking);
  G->mst.assign(n_plans, nullptr);
  G->ready.assign(n_plans, nullptr);
  G->join.assign(n_plans, nullptr);
  G->done.assign(4, nullptr);
  for (int m = 0; m < n_plans && e == cudaSuccess; ++m) {
    e = cudaStreamCreateWithFlags(&G->mst[m], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->ready[m], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->join[m], cudaEventDisableTiming);
  }
  for (auto& ev : G->done)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->gjoin, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    g_create_error = std::string("group set-up: ") + cudaGetErrorString(e);
    qtx_rgf_group_destroy(G);
    return QTX_ERR_CUDA;
  }
  *out = G;
  return QTX_OK;
}

qtx_status qtx_rgf_group_solve(qtx_rgf_group G, const qtx_rgf_inputs* const* in, const qtx_rgf_outputs* const* out,
                               void* stream) {
  if (!G || !in || !out) return QTX_ERR_INVALID_ARG;
  const int n = (int)G->plans.size();
  for (int m = 0; m < n; ++m)
    if (!in[m] || !out[m] || !out[m]->status_per_energy) {
      G->err = "group solves need inputs, outputs and a status_per_energy array for every member";
      return QTX_ERR_INVALID_ARG;
    }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  G->err.clear();
  if (cudaEventRecord(G->fork, st) != cudaSuccess) { G->err = "fork event"; return QTX_ERR_CUDA; }
  for (int m = 0; m < n; ++m)
    if (cudaStreamWaitEvent(G->mst[m], G->fork, 0) != cudaSuccess) { G->err = "fork wait"; return QTX_ERR_CUDA; }
  // the group stream starts after the caller's earlier work too
  if (cudaStreamWaitEvent(G->gst, G->fork, 0) != cudaSuccess) { G->err = "fork wait"; return QTX_ERR_CUDA; }
  std::vector<qtx_status> res(n, QTX_OK);
  G->live = n;
  G->pending.clear();
  for (int m = 0; m < n; ++m) {
    G->plans[m]->group = G;
    G->plans[m]->member = m;
  }
  std::vector<std::thread> th;
  th.reserve(n);
  for (int m = 0; m < n; ++m)
    th.emplace_back([&, m] {
      res[m] = qtx_rgf_solve(G->plans[m], in[m], out[m], G->mst[m]);
      group_leave(G);
    });
  for (auto& t : th) t.join();
  for (int m = 0; m < n; ++m) {
    G->plans[m]->group = nullptr;
    G->plans[m]->member = -1;
  }
  qtx_status worst = QTX_OK;
  for (int m = 0; m < n; ++m)
    if (res[m] != QTX_OK && worst == QTX_OK) {
      worst = res[m];
      G->err = std::string("member ") + std::to_string(m) + ": " + G->plans[m]->err;
    }
  // join every member stream and the group stream back into the caller's stream
  for (int m = 0; m < n; ++m) {
    if (cudaEventRecord(G->join[m], G->mst[m]) != cudaSuccess || cudaStreamWaitEvent(st, G->join[m], 0) != cudaSuccess) {
      if (worst == QTX_OK) { worst = QTX_ERR_CUDA; G->err = "join"; }
    }
  }
  if (cudaEventRecord(G->gjoin, G->gst) != cudaSuccess || cudaStreamWaitEvent(st, G->gjoin, 0) != cudaSuccess) {
    if (worst == QTX_OK) { worst = QTX_ERR_CUDA; G->err = "join"; }
  }
  return worst;
}

qtx_status qtx_rgf_group_set_pool_waves(qtx_rgf_group G, int waves) {
  if (!G || waves < 0) return QTX_ERR_INVALID_ARG;
  G->pool_tiles = (long)waves * G->sms;  // 0: every product fills "0 waves", so none is pooled
  return QTX_OK;
}

long long qtx_rgf_group_launches(qtx_rgf_group G) { return G ? G->launches : 0; }

long long qtx_rgf_group_pooled_products(qtx_rgf_group G) { return G ? G->pooled_products : 0; }

const char* qtx_rgf_group_last_error(qtx_rgf_group G) { return G ? G->err.c_str() : g_create_error.c_str(); }

qtx_status qtx_rgf_group_destroy(qtx_rgf_group G) {
  if (!G) return QTX_OK;
  for (auto s : G->mst)
    if (s) cudaStreamDestroy(s);
  if (G->gst) cudaStreamDestroy(G->gst);
  for (auto e : G->ready)
    if (e) cudaEventDestroy(e);
  for (auto e : G->join)
    if (e) cudaEventDestroy(e);
  for (auto e : G->done)
    if (e) cudaEventDestroy(e);
  if (G->fork) cudaEventDestroy(G->fork);
  if (G->gjoin) cudaEventDestroy(G->gjoin);
  delete G;
  return QTX_OK;
}

}  // extern "C"
