/*
 * qtx_rgf.h -- C ABI of the GB300 (sm_103a) RGF selected-inversion library.
 *
 * What it computes (paper: Sec. II-A, Eq. 2 and Table I, G-row): for every energy E of a grid,
 * independently, the diagonal and first off-diagonal blocks of
 *     G^R(E) = M(E)^-1,   M(E) = z S - H - Sigma^R(E),   z = E + i eta,
 *     G^<(E) = G^R Sigma^<(E) G^A,                       G^A = (G^R)^H,
 *     G^>(E) = G^< + G^R - G^A
 * for a block-tridiagonal (BT, Sec. II-A) complex device matrix with N_B slices of block size b,
 * plus the observables of Sec. II-B (current per slice interface, electron density per slice,
 * contact currents, transmission) and their energy integrals.  The solver is the block Gaussian
 * elimination of Sec. IV-A (forward sweep of left-connected Green's functions g_i, g^<_i, then a
 * backward sweep for the selected blocks); contact self-energies come from Sancho-Rubio
 * decimation.  The broadening eta acts as an extra retarded self-energy -i eta S whose lesser part
 * is 0, i.e. G^> above equals G^R (Sigma^> - 2 i eta S) G^A.
 *
 * Memory: every array pointer in qtx_rgf_inputs / qtx_rgf_outputs is a DEVICE pointer owned by
 * the caller; the library never frees or retains it after qtx_rgf_solve returns.  Complex values
 * are interleaved (re, im) double pairs (C99 double complex / cuDoubleComplex), blocks row-major.
 * Block arrays have layout [energy][slice][row][col] (energy index outermost) unless noted.
 * The plan owns its device workspace (allocated in qtx_rgf_plan, freed in qtx_rgf_destroy).
 *
 * Errors: every call returns a qtx_status.  A status other than QTX_OK from qtx_rgf_solve means
 * nothing was enqueued, except QTX_ERR_CUDA for a failure after launch (message in
 * qtx_rgf_last_error).  Numerical failures found on the device (singular pivot, decimation not
 * converged, bounded wait expired) are written per energy to outputs->status_per_energy (if
 * given) and returned by the next qtx_rgf_status() call; they never trap or abort a kernel.
 * Nothing falls back to the CPU.
 */
#ifndef QTX_RGF_H
#define QTX_RGF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QTX_OK = 0,
  QTX_ERR_INVALID_ARG = 1,   /* bad shape, NULL required pointer, unknown enum value */
  QTX_ERR_OOM = 2,           /* workspace allocation failed */
  QTX_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
  QTX_ERR_SINGULAR = 4,      /* a pivot of a block inverse was zero (per energy) */
  QTX_ERR_NOT_CONVERGED = 5, /* lead decimation hit decim_max_iter (per energy) */
  QTX_ERR_TIMEOUT = 6,       /* a bounded device-side wait expired (per energy / per launch) */
  QTX_ERR_UNSUPPORTED = 7    /* valid request the compiled library or the GPU does not provide */
} qtx_status;

/* Arithmetic of the block products and inverses (Sec. IV, V-A of the paper: the solve of Eq. 2 is
 * ZGEMM-dominated; lower precision is traded against accuracy).  Observables are always reduced
 * in FP64 and the lead decimation always runs in FP64. */
typedef enum {
  QTX_FP64 = 0,   /* complex128 throughout (SIMT DFMA) -- the plain FP64 path */
  QTX_FP32 = 1,   /* complex64 storage; products with all dimensions >= 96 (and K <= 1024) on the
                     tcgen05 tensor cores from 4 bf16 digit planes per operand (10 digit products,
                     ~27-bit products, every digit group exact), smaller products and the leaf
                     inverses on the CUDA cores (FFMA) */
  QTX_BF16X3 = 2, /* products from 2 bf16 digit planes per operand (3 digit products, ~13-bit
                     products) on the tcgen05 tensor cores; df32 storage; refined inverses */
  QTX_EMU64 = 3   /* emulated FP64: products from 6 bf16 digit planes per operand (21 digit products
                     on the tcgen05 tensor cores, Ozaki-style slicing, ~41-bit products; 7 planes and
                     28 digit products for blocks larger than 512), df32 storage,
                     inverses in FP32 refined by Newton sweeps with emulated residuals */
} qtx_precision;

/* Output selection bits (qtx_rgf_desc.outputs).  A block is written only if its bit is set AND
 * its pointer in qtx_rgf_outputs is non-NULL. */
enum {
  QTX_OUT_GR_DIAG = 1u << 0,   /* G^R_ii        [N_E][N_B][b][b]   */
  QTX_OUT_GR_UPPER = 1u << 1,  /* G^R_{i,i+1}   [N_E][N_B-1][b][b] */
  QTX_OUT_GR_LOWER = 1u << 2,  /* G^R_{i+1,i}   [N_E][N_B-1][b][b] */
  QTX_OUT_GL_DIAG = 1u << 3,   /* G^<_ii        [N_E][N_B][b][b]   */
  QTX_OUT_GL_UPPER = 1u << 4,  /* G^<_{i,i+1}   [N_E][N_B-1][b][b]; G^<_{i+1,i} = -(G^<_{i,i+1})^H */
  QTX_OUT_GG_DIAG = 1u << 5,   /* G^>_ii        [N_E][N_B][b][b]   */
  QTX_OUT_GG_UPPER = 1u << 6,  /* G^>_{i,i+1}   [N_E][N_B-1][b][b] */
  QTX_OUT_CURRENT = 1u << 7,   /* I_i(E) = 2 Re Tr[(H_{i,i+1} - E S_{i,i+1}) G^<_{i+1,i}]  [N_E][N_B-1] */
  QTX_OUT_DENSITY = 1u << 8,   /* n_i(E) = Im Tr G^<_ii  [N_E][N_B]                                    */
  QTX_OUT_CONTACT = 1u << 9,   /* I_L,R(E) = Re Tr[Sigma^<_c G^>_kk - Sigma^>_c G^<_kk]  [N_E][2]      */
  QTX_OUT_TRANSMISSION = 1u << 10, /* T(E) = Tr[Gam_L A_00] - Tr[Gam_L G_00 Gam_L G_00^H]  [N_E]    */
  QTX_OUT_INTEGRALS = 1u << 11,    /* sum_E w_E I_i(E) [N_B-1],  sum_E w_E n_i(E)/(2 pi) [N_B]     */
  QTX_OUT_CONTINUITY = 1u << 12,   /* current-conservation residual per energy [N_E] (Sec. II-B):
                                      max_i |I_{i-1} + J_i - I_i| / max_i s_i, J_i = Re Tr[Sigma^<_ii G^>_ii -
                                      Sigma^>_ii G^<_ii] (scattering and broadening), I_{-1} = I_L, I_{N_B-1} =
                                      -I_R with contacts, else 0; s_i = the absolute sums of the terms of J_i
                                      and I_i (the size of what each balance cancels, so the residual is
                                      ~kappa * eps of the arithmetic, ~eps for a well-conditioned FP64 solve) */
  QTX_OUT_ALL = (1u << 13) - 1u
};

/* Shapes and numerics, fixed for the life of a plan. */
typedef struct {
  int n_blocks;                /* N_B >= 1 */
  int block_size;              /* b, 1 <= b <= 4096 */
  int max_energies_in_flight;  /* energies solved concurrently; workspace scales with it (>= 1) */
  qtx_precision precision;
  int refine_max_iter;         /* Newton sweeps X += X (I - A X) per block inverse (QTX_EMU64,
                                  QTX_BF16X3; FP32/FP64 apply one step to recursed blocks > 64) */
  int has_S;                   /* 0: S = I (S pointers ignored) */
  int has_scattering;          /* 0: no scattering self-energies (Sigma pointers ignored) */
  int energy_dependent_sigma;  /* 0: one Sigma set [N_B][b][b] for all energies; 1: [N_E][N_B][b][b] */
  int leads;                   /* 0: none; 1: Sancho-Rubio contacts on slices 0 and N_B-1 */
  double decim_tol;            /* stop when max|alpha|,|beta| < decim_tol * max|H01| (e.g. 1e-13) */
  int decim_max_iter;          /* decimation sweeps before QTX_ERR_NOT_CONVERGED (e.g. 100) */
  unsigned outputs;            /* QTX_OUT_* mask */
  int offdiag_sigma;           /* 1: block-tridiagonal scattering self-energies (needs has_scattering):
                                  SigR_upper, SigR_lower, SigL_upper are read as well.  Sigma^R's
                                  off-diagonal blocks enter M_{i,i+1}, M_{i+1,i}; Sigma^<'s add the
                                  cross terms of the lesser recursions (forward: -V g L + (V g L)^H in
                                  the bracket of g^<_i; backward: Q = V g^< + (g L)^H) */
  int storage_bits;            /* 0: the left-connected blocks g_i, g^<_i of the forward sweep are kept
                                  in the sweep's own type until the backward sweep reads them, and so
                                  are the forward sweep's products V_i g_i and V_i g^<_i (one per
                                  right-hand side), which the backward sweep needs again (Sec. II-A:
                                  two block products fewer per slice, N_B - 1 blocks more per kind and
                                  energy in flight); X in {56, 48, 40, 32, 24, 16}: g_i, g^<_i are
                                  kept in the FPX format of X bits (qtx_kernels.h, Sec. V), with two
                                  working blocks per kind in the sweep's type, and the products are
                                  formed again, which shrinks the footprint per energy in flight */
  int sigma_stream;            /* 1 (needs has_scattering and energy_dependent_sigma, not offdiag_sigma):
                                  SigR_diag and SigL_diag are HOST arrays [N_E][N_B][b][b] (pinned, or
                                  the copies are synchronous); each slice's blocks for the energies of
                                  a chunk are copied to a device staging area (2 blocks per energy in
                                  flight) on the solve's stream just before the forward sweep uses
                                  them, so per-energy self-energies of any number of energies need no
                                  device memory of their own */
  int system_input;            /* 1: solve M X M^H = B (Eq. 2) for a caller-given block-tridiagonal M --
                                  e.g. the screened-Coulomb system M = I - V P^R, B = V P^<> V^H of
                                  Table I (see qtx_w_assemble) -- instead of M = z S - H - Sigma^R:
                                  A_i = M_ii, U_i = M_{i,i+1}, V_i = M_{i+1,i} from inputs M_*; B's
                                  blocks come in SigL_diag (and SigL_upper with offdiag_sigma), H, S,
                                  Sigma^R, eta and the energies' values are not used.  Needs has_S = 0,
                                  leads = 0, sigma_stream = 0; GR_* outputs are the BT blocks of M^-1,
                                  GL_* those of X; GG_* (unless second_rhs), current, contact,
                                  transmission and integrals are not produced (their bits must be
                                  clear); density = Im Tr X_ii */
  double refine_tol;           /* QTX_EMU64 / QTX_BF16X3: an energy stops its Newton sweeps once the
                                  Frobenius norm of its residual I - A X is at most refine_tol (the
                                  next iterate's residual is then at most refine_tol^2); 0 = always
                                  refine_max_iter sweeps */
  int second_rhs;              /* 1 (needs system_input, not storage_bits): the solve takes a second
                                  right-hand side B2 in SigG_diag (and SigG_upper with offdiag_sigma)
                                  and writes the BT blocks of M^-1 B2 M^-H to GG_diag / GG_upper,
                                  sharing the retarded sweep (the inverses and the G^R blocks) with
                                  the first right-hand side -- e.g. X^> of the W system from B^>
                                  alongside X^< from B^<.  The plan then keeps one more set of
                                  left-connected blocks (N_B blocks per energy in flight) */
  double escalate_tol;         /* > 0 (QTX_EMU64, QTX_FP32, QTX_BF16X3; block-diagonal Sigma, not
                                  system_input or sigma_stream): after each chunk the continuity residual
                                  (QTX_OUT_CONTINUITY) of every energy is checked, and energies whose
                                  residual is not below escalate_tol are solved again in FP64 on the same
                                  workspace; their outputs and integral contributions are replaced and
                                  outputs->escalated marks them.  Needs one host synchronisation per
                                  chunk (so such solves cannot be captured in a CUDA graph).  FP32 plans
                                  then size their workspace for complex128 blocks.  0 = off */
  int tc_stages;               /* schedule of the tensor-core product kernel: pipeline stages (0 = the
                                  default; 6 digit planes take 2 or 3, 4 planes 2 or 3, 2 planes 4 or 6,
                                  7 planes 2; other values give the default) */
  int tc_ctas;                 /* schedule: persistent CTAs per product launch (0 = one per SM; fewer
                                  leave SMs to products of other plans running concurrently) */
} qtx_rgf_desc;

/* Device inputs (caller-owned, complex128 unless noted). */
typedef struct {
  const void *H_diag;    /* [N_B][b][b] Hermitian H_ii */
  const void *H_upper;   /* [N_B-1][b][b] H_{i,i+1}; H_{i+1,i} = H_{i,i+1}^H (may be NULL if N_B == 1) */
  const void *S_diag;    /* [N_B][b][b] overlap (has_S) */
  const void *S_upper;   /* [N_B-1][b][b] (has_S) */
  const void *SigR_diag; /* scattering Sigma^R_ii, [N_B][b][b] or [N_E][N_B][b][b] (has_scattering) */
  const void *SigL_diag; /* scattering Sigma^<_ii, same layout; Sigma^> = Sigma^< + Sigma^R - Sigma^A */
  const void *lead_H00_L, *lead_H01_L;  /* [b][b] each (leads): principal layer and the coupling */
  const void *lead_H00_R, *lead_H01_R;  /* from a lead cell to the next one away from the device */
  double eta, mu_L, mu_R, kT;           /* broadening, contact chemical potentials, temperature */
  const double *energies;  /* [N_E] device array */
  const double *weights;   /* [N_E] device array of quadrature weights, or NULL for the trapezoid rule */
  int n_energies;          /* N_E >= 1 */
  int n_blocks;            /* slices of this solve: 0 = the plan's n_blocks, else 1..plan's n_blocks (a
                              plan sized for N_B slices serves any shorter device; block arrays are
                              then laid out with this N_B) */
  const void *SigR_upper;  /* offdiag_sigma: Sigma^R_{i,i+1}, [N_B-1][b][b] or [N_E][N_B-1][b][b]
                              (energy_dependent_sigma) */
  const void *SigR_lower;  /* offdiag_sigma: Sigma^R_{i+1,i}, same layout */
  const void *SigL_upper;  /* offdiag_sigma: Sigma^<_{i,i+1}, same layout; Sigma^<_{i+1,i} =
                              -(Sigma^<_{i,i+1})^H (Sigma^< is anti-Hermitian) */
  const void *M_diag;      /* system_input: M_ii [N_E][N_B][b][b] */
  const void *M_upper;     /* system_input: M_{i,i+1} [N_E][N_B-1][b][b] */
  const void *M_lower;     /* system_input: M_{i+1,i} [N_E][N_B-1][b][b] */
  const void *SigG_diag;   /* second_rhs: B2_ii, the layout of SigL_diag */
  const void *SigG_upper;  /* second_rhs with offdiag_sigma: B2_{i,i+1}, the layout of SigL_upper;
                              B2_{i+1,i} = -(B2_{i,i+1})^H */
} qtx_rgf_inputs;

/* Device outputs (caller-owned; NULL = not produced).  Layouts as in QTX_OUT_*. */
typedef struct {
  void *GR_diag, *GR_upper, *GR_lower, *GL_diag, *GL_upper, *GG_diag, *GG_upper; /* complex128 */
  double *current, *density, *contact, *transmission;
  double *current_int, *density_int;
  int *status_per_energy;  /* [N_E] qtx_status per energy */
  double *continuity;      /* [N_E] QTX_OUT_CONTINUITY residual (of the accepted result) */
  int *escalated;          /* [N_E] 1 where escalate_tol made the energy be solved again in FP64, else 0 */
} qtx_rgf_outputs;

typedef struct qtx_rgf_plan_s *qtx_rgf_plan;

/* Validate desc, allocate the device workspace on the current device.  *out receives the plan. */
qtx_status qtx_rgf_plan_create(const qtx_rgf_desc *desc, qtx_rgf_plan *out);

/* Enqueue the solve of all n_energies on `stream` (a cudaStream_t; NULL = legacy default stream).
 * Energies are processed in chunks of max_energies_in_flight.  Returns after enqueueing: the lead
 * decimation tests convergence on the device (lead blocks of at most 32: the whole iteration of an
 * energy in one CTA; larger: decim_max_iter masked sweeps), so with status_per_energy given the
 * solve makes no host synchronisation and can be captured in a CUDA graph.  Without
 * status_per_energy the library synchronises once per chunk to keep the worst status. */
qtx_status qtx_rgf_solve(qtx_rgf_plan plan, const qtx_rgf_inputs *in, const qtx_rgf_outputs *out,
                         void *stream);

/* Synchronise the plan's last stream and return the worst per-energy status of the last solve. */
qtx_status qtx_rgf_status(qtx_rgf_plan plan);

/* Free the workspace.  Safe on NULL. */
qtx_status qtx_rgf_destroy(qtx_rgf_plan plan);

/* Message for the last error on this plan (or the last failed plan creation if plan is NULL).
 * The string is owned by the library and valid until the next call on the same plan. */
const char *qtx_rgf_last_error(qtx_rgf_plan plan);

/* Device workspace bytes a plan with this desc allocates (for admission by HBM footprint). */
size_t qtx_rgf_footprint(const qtx_rgf_desc *desc);

/* Screened-Coulomb system assembly (Table I, W row): per energy, the block-tridiagonal blocks of
 *     M = I - V P^R,     B^< = V P^< V^H,     B^> = V P^> V^H
 * from the exact products of the BT factors (all contributing blocks; blocks beyond the first
 * off-diagonal are not formed), ready for a system_input solve.  V is Hermitian (V_{i+1,i} =
 * V_{i,i+1}^H) and shared by all energies; P^R is general; P^< and P^> are anti-Hermitian (their
 * lower blocks are -(upper)^H).  The block products run in the plan's precision (tcgen05 digit
 * products for QTX_EMU64) batched over the plan's energies in flight; complex128 in and out. */
typedef struct {
  const void *V_diag, *V_upper;              /* [N_B][b][b], [N_B-1][b][b] */
  const void *PR_diag, *PR_upper, *PR_lower; /* [N_E][N_B][b][b], [N_E][N_B-1][b][b], [N_E][N_B-1][b][b] */
  const void *PL_diag, *PL_upper;            /* P^<: [N_E][N_B][b][b], [N_E][N_B-1][b][b] */
  const void *PG_diag, *PG_upper;            /* P^>: same; both NULL = no B^> */
  int n_energies;                            /* N_E >= 1 */
  int n_blocks;                              /* 0 = the plan's n_blocks, else 1..plan's n_blocks */
} qtx_w_inputs;
typedef struct {
  void *M_diag, *M_upper, *M_lower;          /* [N_E][N_B][b][b], [N_E][N_B-1][b][b] x 2 */
  void *BL_diag, *BL_upper;                  /* B^<: [N_E][N_B][b][b], [N_E][N_B-1][b][b] */
  void *BG_diag, *BG_upper;                  /* B^> (NULL when PG_* are NULL) */
} qtx_w_outputs;
/* Uses the plan's workspace (any plan with this b, enough slices, and the wanted precision; a
 * system_input plan can then solve for X^R and X^< from M and B^<, and with second_rhs for X^> from
 * B^> in the same solve).
 * Asynchronous on `stream`.  Errors: QTX_ERR_INVALID_ARG (NULL required pointers, n_blocks beyond
 * the plan's), QTX_ERR_CUDA. */
qtx_status qtx_w_assemble(qtx_rgf_plan plan, const qtx_w_inputs *in, const qtx_w_outputs *out, void *stream);

/* Groups: several plans -- devices of different N_B and b, each with its own energies, inputs and
 * outputs -- solved together (the uneven batches of Sec. II-A's energy-parallel solve: every energy of
 * every device is independent).  qtx_rgf_group_solve runs each member's qtx_rgf_solve on its own
 * stream (forked from and joined back to `stream`) and pools the members' small tensor-core products:
 * a product that fills two waves of the GPU alone is launched at once on its member's stream; smaller
 * ones are posted and launched together -- ONE persistent kernel over the union of their tiles, up to
 * 8 products of one kernel variant per launch -- once they fill two waves, once every member still
 * solving has posted one, or after a short host wait.  Every member's results equal its plan's solo
 * solve bit for bit.  Every member needs status_per_energy (a solo solve without it
 * synchronises the host).  The call returns after enqueueing everything; it makes no host
 * synchronisation, so it can be captured in a CUDA graph.  The plans stay owned by the caller and
 * must outlive the group; a plan belongs to at most one solving group at a time and must not be
 * solved on its own meanwhile.
 * Errors: QTX_ERR_INVALID_ARG (NULL arguments, a member without status_per_energy), the first failing
 * member's status (message in qtx_rgf_group_last_error), QTX_ERR_CUDA. */
typedef struct qtx_rgf_group_s *qtx_rgf_group;
qtx_status qtx_rgf_group_create(int n_plans, const qtx_rgf_plan *plans, qtx_rgf_group *out);
qtx_status qtx_rgf_group_solve(qtx_rgf_group group, const qtx_rgf_inputs *const *inputs,
                               const qtx_rgf_outputs *const *outputs, void *stream);
qtx_status qtx_rgf_group_destroy(qtx_rgf_group group);
const char *qtx_rgf_group_last_error(qtx_rgf_group group);
/* Schedule of the pooling: a product is pooled when it fills fewer than `waves` waves of the GPU
 * (tiles < waves x SMs) and pooled products are launched once they fill that many; 0 = never pool.
 * Default 0: the members' streams then overlap on the GPU without holding one another in step. */
qtx_status qtx_rgf_group_set_pool_waves(qtx_rgf_group group, int waves);
/* Pooled product-kernel launches this group has issued, and the products they covered (monotonic;
 * for tests and profiling). */
long long qtx_rgf_group_launches(qtx_rgf_group group);
long long qtx_rgf_group_pooled_products(qtx_rgf_group group);

/* Library version string. */
const char *qtx_rgf_version(void);

/* Profiling of the block products (the ZGEMM-class kernel that dominates the solve, Sec. IV).
 * When enabled, every later product-kernel launch of this plan is bracketed by a pair of CUDA events
 * recorded on the solve's stream (for the tensor-core modes, around the tcgen05 GEMM kernel itself,
 * not the digit-plane preparation).  qtx_rgf_gemm_profile synchronises on those events and returns,
 * since enabling or the previous query: the number of launches, their summed device time in
 * milliseconds, the tensor-pipe (or FP pipe) flops issued, and the FP64-equivalent useful flops
 * (8 M N K per complex product), then resets the counters.  Any output pointer may be NULL. */
qtx_status qtx_rgf_set_profiling(qtx_rgf_plan plan, int enable);
qtx_status qtx_rgf_gemm_profile(qtx_rgf_plan plan, long long *launches, double *ms,
                                double *pipe_flops, double *useful_flops);

/* Number of kernel launches this library has issued in this process (monotonic). */
long long qtx_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* QTX_RGF_H */
