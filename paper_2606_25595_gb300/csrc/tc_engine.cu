// Tensor-core engine for sm_103a: batched complex GEMM with emulated precision on tcgen05.
//
// C[e] = alpha * op(A[e]) * op(B[e]) + beta * C0[e]   (complex, df32 storage, e = batch index)
//
// Method (Ozaki-style slicing, paper Sec. II-D: operands are split into lower-precision slices whose
// partial products are recombined): every row of op(A) and every column of op(B) is scaled by a
// power of two 2^(P - e) (e: exponent of its largest entry) and rounded to a P-bit integer v, which is
// written as S balanced base-128 digits  v = sum_i d_i 128^(S-i),  |d_1| <= 2^(l1-1), |d_i| <= 64.
// Digit i is stored pre-scaled as d_i * 2^(-7(i-1)) in a bf16 "digit plane" (exact: <= 7 significant
// bits).  The products of digit planes i, j with i + j <= S + 1 run on the tensor cores (kind::f16,
// bf16 inputs, FP32 accumulation in TMEM) into one accumulator per digit group:
//     acc0..acc3: i + j = 2, 3, 4, 5,     acc4: i + j >= 6 (6 and 7 planes; 4 planes stop at i + j = 5,
//     2 planes at i + j = 3, with every group exact).
// acc0..acc3 hold integers times 2^(-7 (i+j-2)) whose magnitudes stay below 2^24 units (the bound l1
// of the leading digit shrinks with K to guarantee it), so their FP32 sums are exact whatever
// rounding the tensor core's accumulator applies; only acc4, at ~2^-24 of the product, is rounded
// (the accumulation truncates, so its error grows with the number of MMA steps: ~2^-38 at K = 256).
// The epilogue adds the five into df32 (the exact groups exactly: their FP32 sum rounded to an integer
// plus the remainder formed term by term, see sum_acc), applies the row/column scales and writes df32.
// With S = 6 digits (21 digit products) the products carry ~41 bits for K <= 256 (the "emulated FP64"
// mode); for K > 512, where l1 = 5, that mode takes S = 7 (28 digit products, ~44 bits) instead.
// With S = 2 (3 digit products) they carry ~13 bits ("BF16x3").
//
// Complex arithmetic uses the real embedding (4M form):
//     [D_re | D_im] = [A_re | A_im] * [[B_re, B_im], [-B_im, B_re]]
// so one MMA chain with N = 2 BNC real columns produces BNC complex columns (BNC = 48 for 6 and 7
// digit planes, 64 for 4 and 2: bnc_of; the last column tile of a product takes only its
// N - BNC (tiles - 1) columns rounded up to 8, with a narrower MMA N).  The right operand's digit
// planes are stored transposed (N x K, K-major) as three BNC-row sub-tiles per block of BNC columns
// and 16 complex k -- Re B, Im B and -Im B -- which the producer pairs into the 2 BNC rows the MMA
// reads: (Re, Im) against A's real parts, (-Im, Re) against its imaginary parts.
//
// Kernel structure (persistent: one CTA per SM walking 128 x BNC complex output tiles, 10 warps):
//   warp 0   producer: one bulk asynchronous copy (cp.async.bulk, mbarrier complete-tx) per plane
//            tile of one K-stage (16 K-elements; the digitiser stores every tile contiguously, already
//            in the 32-byte-swizzled K-major layout the MMA descriptors expect), a ring of 2-6 stages
//            that runs on across tiles;
//   warp 1   allocates 512 TMEM columns once; one thread issues the tcgen05.mma's (2 K16 steps x
//            pairs), tcgen05.commit's each stage back to the producer and each finished tile to the
//            epilogue, and waits for the epilogue to release TMEM before the next tile;
//   warps 2-9 epilogue (two warps per TMEM lane quarter, one per column half): tcgen05.ld of the
//            accumulators and their recombination into df32 in a staging area, release of TMEM, then
//            the row/column scaling, the alpha and beta * C0 terms and coalesced stores --
//            overlapping the next tile's mainloop.
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the kernel sets *err and unwinds.
#include <cuda_bf16.h>

#include <atomic>
#include <cstring>
#include <mutex>


#include "df32.cuh"
#include "kernels.cuh"

namespace qtx {
namespace tc {

constexpr int BM = 128;        // output rows per CTA (TMEM lanes)
constexpr int BKS = 16;        // bf16 K elements per stage (32-byte rows, 32B swizzle) = one MMA K
constexpr int TILE_A = BM * BKS * 2;   // bytes of one A-plane tile (128 rows x 32 B)
constexpr int DW = 7;          // bits per digit below the leading one
// Complex output columns per CTA (BNC; the MMA's N is 2 BNC real columns, one TMEM accumulator is
// 2 BNC columns wide): 48 for 6 and 7 digit planes, whose five accumulators take 480 of the 512 TMEM
// columns; 64 for 4 and 2 planes, whose digit groups all stay exact in at most four accumulators
// (4 x 128 columns), so a tile covers a third more columns at N = 128.
__host__ __device__ constexpr int bnc_of(int S) { return S >= 6 ? 48 : 64; }
// bytes of one B-plane tile in shared memory (2 BNC rows x 32 B) and of one BNC-row sub-tile
__host__ __device__ constexpr int tile_b_of(int S) { return 2 * bnc_of(S) * BKS * 2; }
__host__ __device__ constexpr int sub_b_of(int S) { return bnc_of(S) * BKS * 2; }
// the epilogue's staging area: BM x BNC df32 complex values (16 bytes), the 16-byte column index
// XOR-swizzled by the row's low three bits, so rows written by consecutive lanes and columns read by
// consecutive threads both fall in distinct bank groups
__host__ __device__ constexpr int out_bytes_of(int S) { return BM * bnc_of(S) * 16; }
__host__ __device__ constexpr int out_at(int r, int c, int S) { return r * bnc_of(S) + (c ^ (r & 7)); }

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after limit_ns of %globaltimer (2 s in normal launches), raising *err, or as
// soon as another thread has raised it.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err, uint64_t limit_ns) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(b, parity)) return true;
    if (*((volatile int*)err)) return false;
    if (gtimer() - t0 > limit_ns) {
      atomicExch(err, 1);
      return false;
    }
    __nanosleep(128);
  }
}
// Bounded wait for work this CTA has already issued (bulk copies, MMAs) to complete, used on the way
// out after an error: it does not give up because *err is raised, only after limit_ns.
__device__ __forceinline__ bool mbar_wait_drain(uint64_t* b, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = gtimer();
  while (!mbar_try(b, parity)) {
    if (gtimer() - t0 > limit_ns) return false;
    __nanosleep(64);
  }
  return true;
}
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // bounded waits of normal launches
constexpr uint64_t kWaitTestLimitNs = 100000ull;   // with the wait test switched on
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 32-byte swizzle, 8-row groups 256 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(256u >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1u << 46;            // descriptor version for tcgen05
  d |= (uint64_t)6u << 61;            // 32-byte swizzle
  return d;
}
// Byte offset of element (row rr, k) inside a K-major tile with 32-byte rows and 32-byte swizzle:
// the 16-byte half-row index is XORed with bit 2 of the row (address bit 4 ^= address bit 7).
__host__ __device__ __forceinline__ uint32_t sw32_offset(uint32_t rr, uint32_t kk) {
  const uint32_t o = rr * 32u + kk * 2u;
  return o ^ (((o >> 7) & 1u) << 4);
}
// Instruction descriptor: kind::f16, D = F32, A = B = BF16, both K-major, M = 128, N = n (a multiple
// of 16 up to 96 here).
__host__ __device__ constexpr uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(dtmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// accumulator of digit pair (i, j): exact groups i + j = 2..5, then one rounded group
__host__ __device__ constexpr int acc_of(int i, int j) { return (i + j <= 5) ? (i + j - 2) : 4; }
__host__ __device__ constexpr int n_acc(int S) { return S + 1 >= 6 ? 5 : S; }

// ------------------------------------------------------------------------------ GEMM kernel
// TcParams (per-product kernel parameters) is declared in kernels.cuh.


// A launch covers the tiles of up to kMaxGroup independent products (a grouped launch: the products
// of several devices of different shapes, one persistent kernel over the union of their tiles).
// Problem q owns tiles [tile0[q], tile0[q+1]); within a problem, tiles are ordered column tile
// fastest, then row tile, then batch entry.
constexpr int kMaxGroup = kTcMaxGroup;
struct TcGroup {
  int n;
  int hold;           // test switch: the MMA thread first waits on a barrier nothing arrives at
  uint64_t limit_ns;  // limit of every bounded wait in this launch
  int tile0[kMaxGroup + 1];
  int NBt[kMaxGroup], MBt[kMaxGroup];
  TcParams p[kMaxGroup];
};
// problem of global tile t, and t's index within it
template <bool GROUP>
__device__ __forceinline__ int problem_of(const TcGroup& G, long t, long& lt) {
  if (!GROUP) {
    lt = t;
    return 0;
  }
  int q = 0;
  while (q + 1 < G.n && t >= G.tile0[q + 1]) ++q;
  lt = t - G.tile0[q];
  return q;
}

// Sum of the accumulators of one output value as df32.  The exact groups acc0..acc3 (all of them
// when NACC < 5) hold multiples of 1, 2^-7, 2^-14, 2^-21 with |acc0| <= 2^21 (Keff L^2 for every
// l1 of dims_of) and |acc_g| < 2^(24 - 7 g); acc4 is the rounded tail, below 2^-2.  So:
//   T = acc0 + acc1 + acc2 + acc3 in FP32 has |T| < 2^22 and is within 3 * 2^-3 of their exact sum
//     S4 (three roundings of at most half an ulp of 2^-2);
//   H = T rounded to an integer (adding and subtracting 1.5 * 2^23) is within 7/8 of S4;
//   r = ((acc0 - H) + acc1) + acc2 + acc3 is exact step by step: acc0 - H is an integer below 2^23,
//     and each later partial sum equals S4 - H minus the groups still to come, below 2^11 on the grid
//     of its finest term (at most 18 significant bits);
//   adding acc4 rounds once, by at most 2^-25 (acc4's own accumulation error is far larger);
//   |r| < 1 <= |H| unless H = 0, so (H, r) renormalises with one Fast2Sum.
// 13 FP32 additions for five accumulators, against 31 for a chain of TwoSum steps.
template <int NACC>
__device__ __forceinline__ df sum_acc(const uint32_t (&v)[NACC][8], int c) {
  constexpr int NEX = NACC < 5 ? NACC : 4;  // exact groups
  const float a0 = __uint_as_float(v[0][c]);
  float t = a0;
#pragma unroll
  for (int g = 1; g < NEX; ++g) t = __fadd_rn(t, __uint_as_float(v[g][c]));
  const float H = __fsub_rn(__fadd_rn(t, 12582912.f), 12582912.f);
  float r = __fsub_rn(a0, H);
#pragma unroll
  for (int g = 1; g < NACC; ++g) r = __fadd_rn(r, __uint_as_float(v[g][c]));
  const float hi = __fadd_rn(H, r);
  return mkdf(hi, __fsub_rn(r, __fsub_rn(hi, H)));
}

// Tile of round k for this CTA.  Round k covers tiles [k G, (k + 1) G) (G = gridDim.x; column tile
// fastest, then row tile, then batch entry), dealt to the CTAs rotated by one per round: the
// narrower last column tile then falls to every CTA equally often (whenever G - 1 is coprime to the
// number of column tiles, always for 152 SMs) rather than to a fixed subset of them, while the
// tiles in flight at any time stay those of a few neighbouring batch entries, which share operands
// through L2.
__device__ __forceinline__ long tile_at(int k) {
  const int G = (int)gridDim.x;
  int b = (int)blockIdx.x - k % G;
  if (b < 0) b += G;
  return (long)k * G + b;
}

// The product kernel is persistent: one CTA per SM walks the tiles of successive rounds (tile_at).
// The stage ring and its barriers run on
// across tiles, and TMEM changes hands through two more barriers: accf (the MMA thread's commit:
// a tile's accumulators are complete) and acce (the epilogue's arrival: it has read them into
// registers and the staging area).  So the producer's loads and the MMAs of tile j+1 overlap the
// epilogue's global stores of tile j, and the prologue (TMEM allocation, barrier set-up, first
// loads) is paid once per SM rather than once per tile.  The staging area is separate from the
// stage ring (NST = 3 stages fit beside it for 6 and 4 digit planes, 6 for 2).

// IO: element type of C and C0 -- df (the emulated-FP64 products) or float (the products of the
// FP32 starting inverse, four digit planes: ~27-bit products, all digit groups exact).
template <typename IO> __device__ __forceinline__ cx<IO> c_from_df(cx<df> v);
template <> __device__ __forceinline__ cx<df> c_from_df<df>(cx<df> v) { return v; }
template <> __device__ __forceinline__ cx<float> c_from_df<float>(cx<df> v) {
  return mk<float>(v.re.hi + v.re.lo, v.im.hi + v.im.lo);
}
__device__ __forceinline__ df df_of(df x) { return x; }
__device__ __forceinline__ df df_of(float x) { return mkdf(x, 0.f); }

// GROUP = false: a single product (problem 0; its parameters at fixed offsets); true: a grouped launch.
template <int S, int NST, typename IO, bool GROUP>
__global__ void __launch_bounds__(320, 1) k_tc_gemm(const __grid_constant__ TcGroup G) {
  const int n_tiles = G.tile0[G.n];
  constexpr int BNC = bnc_of(S), TILE_B = tile_b_of(S), SUB_B = sub_b_of(S), ACC_COLS = 2 * BNC;
  constexpr int OUT_BYTES = out_bytes_of(S);
  constexpr int STAGE = S * (TILE_A + TILE_B);
  constexpr int NACC = n_acc(S);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  cx<df>* out = reinterpret_cast<cx<df>*>(base + NST * STAGE);  // [BM][BNC] staging (out_at)
  uint64_t* full = reinterpret_cast<uint64_t*>(base + NST * STAGE + OUT_BYTES);
  uint64_t* empty = full + NST;
  uint64_t* accf = empty + NST;
  uint64_t* acce = accf + 1;
  uint64_t* holdbar = acce + 1;   // never arrived at (the wait test)
  uint64_t* drainbar = acce + 2;  // the MMA thread's final commit
  uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + 3);
  __shared__ int s_got;
  __shared__ int s_eB[BNC];
  __shared__ int s_eA[BM];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 1);
    mbar_init(holdbar, 1);
    mbar_init(drainbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(512) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      long g = 0;  // stage counter across tiles
      bool ok = true;
      for (int k = 0; ok; ++k) {
        const long t = tile_at(k);
        if (t >= n_tiles) break;
        long lt;
        const int q = problem_of<GROUP>(G, t, lt);
        const TcParams& p = G.p[q];
        const int NBt = G.NBt[q], MBt = G.MBt[q];
        const int e = (int)(lt / (NBt * MBt)), mblk = (int)((lt / NBt) % MBt), nblk = (int)(lt % NBt);
        if (p.active && !p.active[e]) continue;
        const long MB = p.M_pad / BM, NB = p.N_pad / BNC, nkb = p.nks / 2;
        const long ea = p.a_batched ? e : 0, eb = p.b_batched ? e : 0;
        // rows taken from each BNC-row sub-tile: all of them, or the last tile's first bn_last (a
        // multiple of 8 rows = whole 256-byte swizzle groups, so the pair stays in the MMA layout)
        const uint32_t sub = (uint32_t)(nblk == NBt - 1 ? p.bn_last : BNC) * BKS * 2;
        for (int ks = 0; ks < p.nks; ++ks, ++g) {
          const int s = (int)(g % NST);
          const uint32_t ph = (uint32_t)(g / NST) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, G.p[0].err, G.limit_ns)) { ok = false; break; }
          mbar_expect_tx(&full[s], S * (TILE_A + 2 * sub));
          unsigned char* st = base + s * STAGE;
          // K-stages [0, nkb) meet A's real parts: B rows (Re, Im); stages [nkb, 2 nkb) meet A's
          // imaginary parts: B rows (-Im, Re)
          const int part = ks >= nkb, kb = (int)(ks - part * nkb);
          const int s0 = part ? 2 : 0, s1 = part ? 0 : 1;
          for (int d = 0; d < S; ++d) {
            bulk_load(st + d * TILE_A, p.pa + (((ea * S + d) * MB + mblk) * p.nks + ks) * (long)TILE_A, TILE_A, &full[s]);
            const unsigned char* sb = p.pb + (((eb * S + d) * NB + nblk) * nkb + kb) * 3L * SUB_B;
            unsigned char* db = st + S * TILE_A + d * TILE_B;
            bulk_load(db, sb + s0 * SUB_B, sub, &full[s]);
            bulk_load(db + sub, sb + s1 * SUB_B, sub, &full[s]);
          }
        }
      }
      // the copies of the last stages issued (at most NST of them, one per slot) land before the
      // CTA goes on to exit, also when a wait gave up and the MMA thread no longer consumes them
      for (long gi = g > NST ? g - NST : 0; gi < g; ++gi)
        mbar_wait_drain(&full[gi % NST], (uint32_t)(gi / NST) & 1u, kWaitLimitNs);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      long g = 0;
      int j = 0;  // tiles processed by this CTA
      bool ok = true;
      // wait test: a barrier nothing arrives at, so the wait gives up before any MMA is issued
      if (G.hold && !mbar_wait(holdbar, 0u, G.p[0].err, G.limit_ns)) ok = false;
      for (int k = 0; ok; ++k) {
        const long t = tile_at(k);
        if (t >= n_tiles) break;
        long lt;
        const int q = problem_of<GROUP>(G, t, lt);
        const TcParams& p = G.p[q];
        const int NBt = G.NBt[q], MBt = G.MBt[q];
        const int e = (int)(lt / (NBt * MBt));
        if (p.active && !p.active[e]) continue;
        const uint32_t idesc = idesc_n(2 * (lt % NBt == NBt - 1 ? p.bn_last : BNC));
        // TMEM is free once the epilogue has read the previous tile's accumulators
        if (!mbar_wait(acce, ((uint32_t)j & 1u) ^ 1u, G.p[0].err, G.limit_ns)) break;
        fence_after();
        uint32_t started = 0;
        for (int ks = 0; ks < p.nks; ++ks, ++g) {
          const int s = (int)(g % NST);
          const uint32_t ph = (uint32_t)(g / NST) & 1u;
          if (!mbar_wait(&full[s], ph, G.p[0].err, G.limit_ns)) { ok = false; break; }
          fence_after();
          const uint32_t sa = su32(base + s * STAGE);
#pragma unroll
          for (int i = 1; i <= S; ++i) {
#pragma unroll
            for (int jj = 1; jj <= S + 1 - i; ++jj) {
              const int gacc = acc_of(i, jj);
              const uint64_t ad = sdesc(sa + (i - 1) * TILE_A);
              const uint64_t bd = sdesc(sa + S * TILE_A + (jj - 1) * TILE_B);
              mma(tmem + gacc * ACC_COLS, ad, bd, idesc, (started >> gacc) & 1u);
              started |= 1u << gacc;
            }
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(accf);
        ++j;
      }
      // every MMA this thread issued has completed before TMEM is freed (a commit tracks all of
      // them; it arrives at once when none is outstanding)
      mma_commit(drainbar);
      mbar_wait_drain(drainbar, 0u, kWaitLimitNs);
    }
    __syncwarp();
  } else {
    // epilogue: warps 2..9; TMEM lane quarter = warp % 4, column half = (warp - 2) / 4
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int r = q * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    int j = 0;
    for (int k = 0;; ++k) {
      const long t = tile_at(k);
      if (t >= n_tiles) break;
      long lt;
      const int q = problem_of<GROUP>(G, t, lt);
      const TcParams& p = G.p[q];
      const int NBt = G.NBt[q], MBt = G.MBt[q];
      const int e = (int)(lt / (NBt * MBt)), mblk = (int)((lt / NBt) % MBt), nblk = (int)(lt % NBt);
      if (p.active && !p.active[e]) continue;
      // complex columns of this tile: Re parts in TMEM columns [0, bn), Im parts in [bn, 2 bn)
      const int bn = nblk == NBt - 1 ? p.bn_last : BNC;
      // every epilogue thread is done with the previous tile's staging area and exponents
      __syncwarp();
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (threadIdx.x >= 64 && threadIdx.x < 64 + BNC)
        s_eB[threadIdx.x - 64] = p.eB[(long)(p.b_batched ? e : 0) * p.N_pad + nblk * BNC + threadIdx.x - 64];
      if (threadIdx.x >= 128 && threadIdx.x < 128 + BM)
        s_eA[threadIdx.x - 128] = p.eA[(long)(p.a_batched ? e : 0) * p.M_pad + mblk * BM + threadIdx.x - 128];
      if (threadIdx.x == 64) s_got = mbar_wait(accf, (uint32_t)j & 1u, G.p[0].err, G.limit_ns) ? 1 : 0;
      __syncwarp();
      asm volatile("bar.sync 2, 256;" ::: "memory");
      if (!s_got) break;
      fence_after();
      // the two warps of a lane quarter take alternate chunks of 8 columns
#pragma unroll 1
      for (int c0 = 8 * h; c0 < bn; c0 += 16) {
        uint32_t vr[NACC][8], vi[NACC][8];
#pragma unroll
        for (int gq = 0; gq < NACC; ++gq) {
          tmem_ld8(trow + gq * ACC_COLS + c0, vr[gq]);
          tmem_ld8(trow + gq * ACC_COLS + bn + c0, vi[gq]);
        }
        tmem_wait_ld();
        // only the recombination runs while the tile holds TMEM; scaling waits for the store phase
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          cx<df> o;
          o.re = sum_acc<NACC>(vr, c);
          o.im = sum_acc<NACC>(vi, c);
          out[out_at(r, c0 + c, S)] = o;
        }
      }
      // accumulators read (tcgen05.wait::ld above): hand TMEM back to the MMA thread
      fence_before();
      __syncwarp();
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (threadIdx.x == 64) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(acce)) : "memory");
      const cx<IO>* C0e = p.C0 ? reinterpret_cast<const cx<IO>*>(p.C0) + (long)e * p.sC0 : nullptr;
      cx<IO>* Ce = reinterpret_cast<cx<IO>*>(p.C) + (long)e * p.sC;
      for (int idx = threadIdx.x - 64; idx < BM * bn; idx += 256) {
        const int rr = idx / bn, cc = idx % bn;
        const int mm = mblk * BM + rr, nn = nblk * BNC + cc;
        if (mm < p.M && nn < p.N) {
          cx<df> v = out[out_at(rr, cc, S)];
          int Es = s_eA[rr] + s_eB[cc] - p.escale;
          Es = Es < -250 ? -250 : (Es > 250 ? 250 : Es);
          const float f1 = __int_as_float((Es / 2 + 127) << 23), f2 = __int_as_float((Es - Es / 2 + 127) << 23);
          // the scales are powers of two: exact (barring over/underflow)
          v.re = mkdf(v.re.hi * f1 * f2, v.re.lo * f1 * f2);
          v.im = mkdf(v.im.hi * f1 * f2, v.im.lo * f1 * f2);
          if (p.akind == 1) {
            v.re = df_neg(v.re);
            v.im = df_neg(v.im);
          } else if (p.akind == 2) {
            v.re = df_mul(v.re, p.alpha);
            v.im = df_mul(v.im, p.alpha);
          }
          if (C0e && p.bkind != 3) {
            const cx<IO> c0v = C0e[(long)mm * p.ldc0 + nn];
            df c0r = df_of(c0v.re), c0i = df_of(c0v.im);
            if (p.bkind == 1) {
              c0r = df_neg(c0r);
              c0i = df_neg(c0i);
            } else if (p.bkind == 2) {
              c0r = df_mul(c0r, p.beta);
              c0i = df_mul(c0i, p.beta);
            }
            v.re = df_add(v.re, c0r);
            v.im = df_add(v.im, c0i);
          }
          Ce[(long)mm * p.ldc + nn] = c_from_df<IO>(v);
        }
      }
      ++j;
    }
  }
  __syncwarp();
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// ------------------------------------------------------------------------------ digitizer
// Digits of one df32 value in floating point (used by the fused pass).  With the row scaled so the
// leading digit's unit is 1 (x' = x 2^(l1 - 1 - e_row), |x'| < 2^(l1-1)), digit i (0-based) is a
// multiple of U_i = 2^(-7 i) -- exactly the pre-scaled plane value d_i 2^(-7 i).  Each digit is the
// residual rounded to a multiple of U_i by adding and subtracting 1.5 * 2^23 * U_i (exact, round to
// nearest), leaving an exact residual of at most U_i / 2 = 64 U_(i+1).  hi gives all S digits; lo
// (|lo'| <= ulp(hi')/2 <= 2^-19) only reaches digits 3.. (0-based), which take the sum of both
// parts; a bottom-up carry brings those back to |d_i| <= 64 U_i (digit 2 may end at 65 U_2).  The
// represented value is within one unit U_(S-1) of x'.
__device__ __forceinline__ float round_sigma(int i) { return 1.5f * __int_as_float((127 + 23 - DW * i) << 23); }
template <int S>
__device__ __forceinline__ void split_digits(df x, float f1, float f2, float (&d)[S]) {
  float r = x.hi * f1 * f2;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const float sg = round_sigma(i);
    const float di = __fsub_rn(__fadd_rn(r, sg), sg);
    d[i] = di;
    r = __fsub_rn(r, di);
  }
  if constexpr (S >= 4) {
    float t = x.lo * f1 * f2;
#pragma unroll
    for (int i = 3; i < S; ++i) {
      const float sg = round_sigma(i);
      const float di = __fsub_rn(__fadd_rn(t, sg), sg);
      d[i] = __fadd_rn(d[i], di);
      t = __fsub_rn(t, di);
    }
#pragma unroll
    for (int i = S - 1; i >= 3; --i) {
      const float sg = round_sigma(i - 1);
      const float c = __fsub_rn(__fadd_rn(d[i], sg), sg);
      d[i] = __fsub_rn(d[i], c);
      d[i - 1] = __fadd_rn(d[i - 1], c);
    }
  }
}
__device__ __forceinline__ uint32_t bf16x2_bits(float lo_half, float hi_half) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo_half, hi_half);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Fused exponent + digit pass over RPC whole logical rows per CTA (used whenever a strip of RPC
// rows fits in shared memory, i.e. K up to ~11000): the strip is read from global memory once into
// shared memory (coalesced along k for direct rows, along r for transposed ones), the row exponents
// are reduced on the way in, and every thread then turns one (row, 8 complex k) item into the S
// digit planes with 16-byte stores -- one swizzled half-row chunk per plane and part.  The strip is
// skewed by one element per 8 so that the threads' 128-byte item reads fall in distinct banks.
// Item layout as k_digitize: A rows [Re | Im]; B re row [Re | -Im], im row [Im | Re] (a bf16 sign
// flip, exact).  Rows r >= R and k >= K are written as zero digits, with exponent -1000.
__host__ __device__ constexpr int strip_skew(int k) { return k + (k >> 3); }

template <int S, int RPC, typename TI>
__global__ void __launch_bounds__(32 * RPC) k_digitize_rows(const cx<TI>* X, long ldx, long sX, int R, int K, int R_pad,
                                                       int K_pad, int transposed, int conj_, int side, int* eout,
                                                       int P, unsigned char* planes, long rows_plane,
                                                       const int* active) {
  const int e = blockIdx.y;
  if (active && !active[e]) return;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int ldS = strip_skew(K_pad) + 1;  // complex elements per strip row
  cx<df>* strip = reinterpret_cast<cx<df>*>(dsm);
  __shared__ int s_ex[RPC];
  constexpr int NT = 32 * RPC;  // threads: one warp per strip row
  const cx<TI>* Xe = X + (long)e * sX;
  // an element as df32 (FP32 inputs: lo = 0)
  auto ld = [&](long off) -> cx<df> {
    const cx<TI> x = Xe[off];
    cx<df> v;
    v.re = df_of(x.re);
    v.im = df_of(x.im);
    return v;
  };
  const int r0 = blockIdx.x * RPC, t = threadIdx.x;
  if (t < RPC) s_ex[t] = -1000;
  __syncthreads();
  const cx<df> zero = {mkdf(0.f, 0.f), mkdf(0.f, 0.f)};
  // ---- load the strip (zero beyond R, K) and reduce the row exponents; loads are batched (all
  // rows of a direct strip, four k of a transposed one) before their first use
  if (!transposed) {
    int mx[RPC];
#pragma unroll
    for (int rr = 0; rr < RPC; ++rr) mx[rr] = -1000;
    for (int k = t; k < K_pad; k += NT) {
      cx<df> v[RPC];
#pragma unroll
      for (int rr = 0; rr < RPC; ++rr) {
        const int r = r0 + rr;
        v[rr] = (r < R && k < K) ? ld((long)r * ldx + k) : zero;
      }
#pragma unroll
      for (int rr = 0; rr < RPC; ++rr) {
        strip[rr * ldS + strip_skew(k)] = v[rr];
        if (r0 + rr < R && k < K) mx[rr] = max(mx[rr], max(df_expo(v[rr].re.hi), df_expo(v[rr].im.hi)));
      }
    }
#pragma unroll
    for (int rr = 0; rr < RPC; ++rr) {
      int m = mx[rr];
      for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
      if ((t & 31) == 0 && m > -1000) atomicMax(&s_ex[rr], m);
    }
  } else {
    constexpr int KS = NT / RPC;  // k stride between a thread's elements
    const int rr = t % RPC, r = r0 + rr;
    int mx = -1000;
    for (int k0 = t / RPC; k0 < K_pad; k0 += 4 * KS) {
      cx<df> v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + u * KS;
        v[u] = (r < R && k < K) ? ld((long)k * ldx + r) : zero;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + u * KS;
        if (k < K_pad) strip[rr * ldS + strip_skew(k)] = v[u];
        if (r < R && k < K) mx = max(mx, max(df_expo(v[u].re.hi), df_expo(v[u].im.hi)));
      }
    }
    if (mx > -1000) atomicMax(&s_ex[rr], mx);
  }
  __syncthreads();
  if (t < RPC && r0 + t < R_pad) eout[(long)e * R_pad + r0 + t] = s_ex[t];
  // ---- digits: item = (row rr, complex k = 8 kc .. 8 kc + 7)
  // left operand: [row_block of 128][k_stage of 16 embedded k][128 x 32 B] tiles, embedded k' = k for
  // Re, K_pad + k for Im.  right operand: [col_block of BNC][k_block of 16 complex k][3][BNC x 32 B]
  // sub-tiles holding Re, Im and -Im (the producer pairs them into the (Re, Im) and (-Im, Re) rows).
  const long nks = 2L * K_pad / BKS, nkb = K_pad / BKS;
  constexpr int BNC = bnc_of(S), SUB_B = sub_b_of(S);
  const long plane_bytes = side == 0 ? (rows_plane / BM) * nks * (long)TILE_A : (long)(R_pad / BNC) * nkb * 3 * SUB_B;
  unsigned char* pe = planes + (long)e * S * plane_bytes;
  const int nkc = K_pad / 8;
  // rows whose planes are written: right-operand columns past N rounded up to 8 are never read (the
  // last column tile's MMA takes only its first bn_last rows), so they stay unwritten
  const int R_wr = side == 1 ? min(R_pad, (R + 7) / 8 * 8) : R_pad;
  // byte offset of the 16-byte chunk holding embedded k' .. k' + 7 (k' a multiple of 8) of row r (left)
  auto chunk_off = [&](long row, int kp) -> long {
    const long blk = row / BM, rr_ = row % BM, ks = kp / BKS, kk = kp % BKS;
    return (blk * nks + ks) * TILE_A + sw32_offset((uint32_t)rr_, (uint32_t)kk);
  };
  // ... of complex k .. k + 7 of column r (right), in sub-tile `sub`
  auto sub_off = [&](long col, int k, int sub) -> long {
    const long cb = col / BNC, rr_ = col % BNC, kb = k / BKS, kk = k % BKS;
    return ((cb * nkb + kb) * 3 + sub) * (long)SUB_B + sw32_offset((uint32_t)rr_, (uint32_t)kk);
  };
#pragma unroll 1
  for (int item = t; item < RPC * nkc; item += NT) {
    const int rr = item / nkc, kc = item % nkc, r = r0 + rr;
    if (r >= R_wr) continue;
    // scale 2^(l1 - 1 - e_row) = 2^(P - 7 (S-1) - e_row), as two factors (e_row may be -1000)
    int Es = P - DW * (S - 1) - s_ex[rr];
    Es = Es < -250 ? -250 : (Es > 250 ? 250 : Es);
    const float f1 = __int_as_float((Es / 2 + 127) << 23), f2 = __int_as_float((Es - Es / 2 + 127) << 23);
    uint32_t wre[S][4], wim[S][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      float d0r[S], d0i[S], d1r[S], d1i[S];
      cx<df> v0 = strip[rr * ldS + strip_skew(8 * kc + j)];
      cx<df> v1 = strip[rr * ldS + strip_skew(8 * kc + j + 1)];
      if (conj_) {
        v0.im = df_neg(v0.im);
        v1.im = df_neg(v1.im);
      }
      split_digits<S>(v0.re, f1, f2, d0r);
      split_digits<S>(v0.im, f1, f2, d0i);
      split_digits<S>(v1.re, f1, f2, d1r);
      split_digits<S>(v1.im, f1, f2, d1i);
#pragma unroll
      for (int i = 0; i < S; ++i) {
        wre[i][j / 2] = bf16x2_bits(d0r[i], d1r[i]);
        wim[i][j / 2] = bf16x2_bits(d0i[i], d1i[i]);
      }
    }
    const int k8 = 8 * kc;
    if (side == 0) {
      const long o_re = chunk_off(r, k8), o_im = chunk_off(r, K_pad + k8);
#pragma unroll
      for (int i = 0; i < S; ++i) {
        unsigned char* pl = pe + (long)i * plane_bytes;
        *reinterpret_cast<uint4*>(pl + o_re) = make_uint4(wre[i][0], wre[i][1], wre[i][2], wre[i][3]);
        *reinterpret_cast<uint4*>(pl + o_im) = make_uint4(wim[i][0], wim[i][1], wim[i][2], wim[i][3]);
      }
    } else {
      const long o0 = sub_off(r, k8, 0), o1 = sub_off(r, k8, 1), o2 = sub_off(r, k8, 2);
      const uint32_t SGN = 0x80008000u;  // bf16 sign bits of both halves
#pragma unroll
      for (int i = 0; i < S; ++i) {
        unsigned char* pl = pe + (long)i * plane_bytes;
        *reinterpret_cast<uint4*>(pl + o0) = make_uint4(wre[i][0], wre[i][1], wre[i][2], wre[i][3]);
        *reinterpret_cast<uint4*>(pl + o1) = make_uint4(wim[i][0], wim[i][1], wim[i][2], wim[i][3]);
        *reinterpret_cast<uint4*>(pl + o2) =
            make_uint4(wim[i][0] ^ SGN, wim[i][1] ^ SGN, wim[i][2] ^ SGN, wim[i][3] ^ SGN);
      }
    }
  }
}

// ------------------------------------------------------------------------------ host side
// Test switch of the bounded waits (qtx_tc_wait_test).
std::atomic<int> g_wait_test{0};

struct Dims {
  int M_pad, N_pad, K_pad, l1, P;
};
inline Dims dims_of(int M, int N, int K, int S) {
  Dims d;
  d.M_pad = (M + BM - 1) / BM * BM;
  d.N_pad = (N + bnc_of(S) - 1) / bnc_of(S) * bnc_of(S);
  d.K_pad = (K + 31) / 32 * 32;
  // Leading digit bound L = 2^(l1-1), others 64: per K term the exact groups are bounded by
  //   i+j=2: L^2,  3: 2 L 64,  4: 2 L 64 + 64^2,  5: 2 L 64 + 2 * 64^2
  // units, so with Keff = 2 K_pad terms they stay below 2^24 for l1 = 7 up to Keff = 512 and
  // l1 = 6 up to Keff = 1024.  Beyond that (b > 512) i+j = 5 is no longer guaranteed exact.
  const int Keff = 2 * d.K_pad;
  d.l1 = Keff <= 512 ? 7 : (Keff <= 1024 ? 6 : 5);
  d.P = DW * (S - 1) + d.l1 - 1;
  return d;
}
struct Scratch {
  unsigned char *pa, *pb;
  int *ea, *eb;
  size_t bytes;
};
inline Scratch carve(void* base, const Dims& d, int batch, int S) {
  auto al = [](size_t x) { return (x + 1023) & ~size_t(1023); };
  Scratch s;
  unsigned char* p = reinterpret_cast<unsigned char*>(base);
  const size_t a = al((size_t)batch * S * d.M_pad * 2 * d.K_pad * sizeof(__nv_bfloat16));
  const size_t b = al((size_t)batch * S * (d.N_pad / bnc_of(S)) * (d.K_pad / BKS) * 3 * sub_b_of(S));  // Re, Im, -Im sub-tiles
  const size_t ea = al((size_t)batch * d.M_pad * sizeof(int));
  const size_t eb = al((size_t)batch * d.N_pad * sizeof(int));
  s.pa = p;
  s.pb = p + a;
  s.ea = reinterpret_cast<int*>(p + a + b);
  s.eb = reinterpret_cast<int*>(p + a + b + ea);
  s.bytes = a + b + ea + eb;
  return s;
}

template <int S, typename TI>
cudaError_t digitize(const cx<TI>* X, long ldx, long sX, int opX, int side, int R, int K, const Dims& d,
                     int* eout, unsigned char* planes, int batch, const int* active, cudaStream_t st) {
  // logical row r of the operand: left A = op(X): row r of op(X); right B = op(X): column r of op(X)
  //   left  N: X[r][k] direct      left  H: conj(X[k][r]) transposed
  //   right N: X[k][r] transposed  right H: conj(X[r][k]) direct
  const int transposed = (side == 0) ? (opX == OP_C) : (opX == OP_N);
  const int cj = opX == OP_C;
  const int R_pad = side == 0 ? d.M_pad : d.N_pad;
  const long rows_plane = side == 0 ? d.M_pad : 2L * d.N_pad;
  // fused pass: RPC rows per CTA with one warp per row -- two rows while the strip stays within
  // 48 KB of shared memory (many small CTAs per SM, so loads, digit arithmetic and stores of
  // different CTAs overlap), else a single row up to the 200 KB the kernel is allowed
  const size_t row_bytes = (size_t)(strip_skew(d.K_pad) + 1) * sizeof(cx<df>);
  const int rpc = 2 * row_bytes <= 48 * 1024 ? 2 : 1;
  if (rpc * row_bytes > 200 * 1024) return cudaErrorInvalidValue;  // K-chunks of <= 1024 always fit
  {
    static bool attr = false;
    if (!attr) {
      cudaError_t ea = cudaFuncSetAttribute(k_digitize_rows<S, 2, TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (ea == cudaSuccess) ea = cudaFuncSetAttribute(k_digitize_rows<S, 1, TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (ea != cudaSuccess) return ea;
      attr = true;
    }
    const size_t smem = rpc * row_bytes;
    dim3 g(R_pad / rpc, batch);
    if (rpc == 2)
      k_digitize_rows<S, 2, TI><<<g, 64, smem, st>>>(X, ldx, sX, R, K, R_pad, d.K_pad, transposed, cj, side, eout, d.P, planes, rows_plane, active);
    else
      k_digitize_rows<S, 1, TI><<<g, 32, smem, st>>>(X, ldx, sX, R, K, R_pad, d.K_pad, transposed, cj, side, eout, d.P, planes, rows_plane, active);
    count_launch();
    return cudaGetLastError();
  }
}

// Digitise one product's operands (into the scratch, or a kept operand) and fill its kernel
// parameters and tile counts.
template <int S, typename IO>
cudaError_t prepare(const TcArgs& a, void* scratch, size_t scratch_bytes, int* err_flag, cudaStream_t st,
                    TcPrepared& out) {
  TcParams& p = out.p;
  // operand and result pointers in the IO type (TcArgs carries the df32 ones; f32 products pass
  // FP32 arrays through the same fields)
  const cx<IO>* A = reinterpret_cast<const cx<IO>*>(a.A);
  const cx<IO>* B = reinterpret_cast<const cx<IO>*>(a.B);
  const Dims d = dims_of(a.M, a.N, a.K, S);
  Scratch sc = carve(scratch, d, a.batch, S);
  if (sc.bytes > scratch_bytes) return cudaErrorInvalidValue;
  cudaError_t e;
  const int ab = a.sA != 0, bb_ = a.sB != 0;
  // digit planes and exponents of each operand: in the scratch, or in a kept operand (digitised
  // there now, or reused as they are)
  unsigned char* pa = a.opndA ? a.opndA->planes : sc.pa;
  unsigned char* pb = a.opndB ? a.opndB->planes : sc.pb;
  int* ea = a.opndA ? a.opndA->expo : sc.ea;
  int* eb = a.opndB ? a.opndB->expo : sc.eb;
  if (!(a.opndA && a.opndA->mode == 2))
    if ((e = digitize<S, IO>(A, a.lda, a.sA, a.opA, 0, a.M, a.K, d, ea, pa, ab ? a.batch : 1, ab ? a.active : nullptr, st))) return e;
  if (!(a.opndB && a.opndB->mode == 2))
    if ((e = digitize<S, IO>(B, a.ldb, a.sB, a.opB, 1, a.N, a.K, d, eb, pb, bb_ ? a.batch : 1, bb_ ? a.active : nullptr, st))) return e;
  p.pa = pa;
  p.pb = pb;
  p.eA = ea;
  p.eB = eb;
  p.M_pad = d.M_pad;
  p.N_pad = d.N_pad;
  p.nks = 2 * d.K_pad / BKS;
  p.M = a.M;
  p.N = a.N;
  p.C = a.C;
  p.ldc = a.ldc;
  p.sC = a.sC;
  p.C0 = a.C0;
  p.ldc0 = a.ldc0;
  p.sC0 = a.sC0;
  // alpha, beta as df32 pairs (an FP64 scalar such as 0.1 keeps ~48 bits) and their kinds
  auto kind_of = [](double x, df& v) {
    v = df_split_fp64(x);
    return x == 1.0 ? 0 : (x == -1.0 ? 1 : 2);
  };
  p.akind = kind_of(a.alpha, p.alpha);
  p.bkind = (a.C0 && a.beta != 0.0) ? kind_of(a.beta, p.beta) : 3;
  if (p.bkind == 3) p.beta = df_split_fp64(0.0);
  p.escale = 2 * d.l1 - 2;
  p.a_batched = ab;
  p.b_batched = bb_;
  p.active = a.active;
  p.err = err_flag;
  out.NBt = d.N_pad / bnc_of(S);
  out.MBt = d.M_pad / BM;
  const int tail = a.N - (out.NBt - 1) * bnc_of(S);  // 1..BNC complex columns in the last column tile
  p.bn_last = (tail + 7) / 8 * 8;
  out.tiles = (long)out.NBt * out.MBt * a.batch;
  return cudaSuccess;
}

// One persistent launch over the tiles of n prepared products (n = 1: a plain product).
template <int S, int NST, typename IO>
cudaError_t launch(const TcPrepared* const* pp, int n, cudaStream_t st, cudaEvent_t* ev) {
  if (n < 1 || n > kMaxGroup) return cudaErrorInvalidValue;
  cudaError_t e;
  const size_t smem = (size_t)NST * S * (TILE_A + tile_b_of(S)) + out_bytes_of(S) + 1024 + 256;
  static bool attr = false;
  static int sms = 0;
  if (!attr) {
    if ((e = cudaFuncSetAttribute(k_tc_gemm<S, NST, IO, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_gemm<S, NST, IO, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
    attr = true;
  }
  TcGroup G;
  G.n = n;
  G.hold = g_wait_test.load(std::memory_order_relaxed);
  G.limit_ns = G.hold ? kWaitTestLimitNs : kWaitLimitNs;
  long total = 0;
  for (int q = 0; q < n; ++q) {
    G.p[q] = pp[q]->p;
    G.NBt[q] = pp[q]->NBt;
    G.MBt[q] = pp[q]->MBt;
    G.tile0[q] = (int)total;
    total += pp[q]->tiles;
    if (total > 0x7fffffffL) return cudaErrorInvalidValue;
  }
  G.tile0[n] = (int)total;
  if (total == 0) return cudaSuccess;
  // one CTA per SM (the kernel holds up to ~230 KB of smem), or the schedule's CTA count
  int ctas = sms;
  for (int q = 0; q < n; ++q)
    if (pp[q]->ctas > 0 && pp[q]->ctas < ctas) ctas = pp[q]->ctas;
  const int grid = (int)(total < ctas ? total : ctas);
  if (ev) cudaEventRecord(ev[0], st);
  if (n == 1) k_tc_gemm<S, NST, IO, false><<<grid, 320, smem, st>>>(G);
  else k_tc_gemm<S, NST, IO, true><<<grid, 320, smem, st>>>(G);
  count_launch();
  if (ev) cudaEventRecord(ev[1], st);
  return cudaGetLastError();
}

}  // namespace tc

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3;
}

// Digits actually used: the emulated-FP64 mode takes a seventh digit when K > 512, where the
// leading digit has shrunk to l1 = 5 bits (dims_of) and six digits would carry only 40 bits.
static int effective_digits(int digits, int K) { return (digits == 6 && K > 512) ? 7 : digits; }

// Contractions longer than kMaxKChunk run as consecutive K-chunks of at most that length, each
// added to the previous partial result in the epilogue (C0 = C, beta = 1, df32 addition): the
// exactness bound of the digit accumulators (the leading digit's l1 bits) only covers K <= 1024.
constexpr int kMaxKChunk = 1024;
static int k_chunks(int K) { return K <= kMaxKChunk ? 1 : (K + kMaxKChunk - 1) / kMaxKChunk; }

size_t gemm_tc_scratch_bytes(int M, int N, int K, int batch, int digits) {
  const int Kc = (K + k_chunks(K) - 1) / k_chunks(K);
  const int S = effective_digits(digits, Kc);
  const tc::Dims d = tc::dims_of(M, N, Kc, S);
  return tc::carve(nullptr, d, batch, S).bytes + 4096;
}

static size_t al1k(size_t x) { return (x + 1023) & ~size_t(1023); }
// digit-plane bytes of one operand (as carve lays them out)
static size_t plane_bytes_of(int side, const tc::Dims& d, int batch, int S) {
  return side == 0 ? (size_t)batch * S * d.M_pad * 2 * d.K_pad * 2
                   : (size_t)batch * S * (d.N_pad / tc::bnc_of(S)) * (d.K_pad / tc::BKS) * 3 * tc::sub_b_of(S);
}

size_t gemm_tc_operand_bytes(int side, int R, int K, int batch, int digits) {
  if (k_chunks(K) > 1) return 0;
  const int S = effective_digits(digits, K);
  const tc::Dims d = side == 0 ? tc::dims_of(R, 1, K, S) : tc::dims_of(1, R, K, S);
  return al1k(plane_bytes_of(side, d, batch, S)) + al1k((size_t)batch * (side == 0 ? d.M_pad : d.N_pad) * sizeof(int));
}

TcOperand tc_operand_at(void* base, int side, int R, int K, int batch, int digits) {
  const int S = effective_digits(digits, K);
  const tc::Dims d = side == 0 ? tc::dims_of(R, 1, K, S) : tc::dims_of(1, R, K, S);
  TcOperand o;
  o.planes = reinterpret_cast<unsigned char*>(base);
  o.expo = reinterpret_cast<int*>(o.planes + al1k(plane_bytes_of(side, d, batch, S)));
  return o;
}

// Pipeline stages of a kernel variant: the requested count if shared memory allows it, else the
// default.  Beside the 96 KB epilogue staging of 48-column tiles, 6 digit planes take 42 KB a stage
// and 7 take 49 KB; beside the 128 KB staging of 64-column tiles, 4 planes take 32 KB and 2 take 16 KB.
static int resolve_stages(int S, bool f32, int want) {
  if (f32 || S == 4) return (want == 2) ? 2 : 3;  // S = 4 (complex64 or df32 in and out): 2 or 3
  if (S == 6) return (want == 2) ? 2 : 3;         // 2 or 3
  if (S == 7) return 2;
  return (want == 4) ? 4 : 6;                   // S = 2: 4 or 6
}

// Kernel variant of a product: digits actually used (effective_digits), the IO type and the stages;
// -1 when the product is split along K (it then runs as consecutive chunks and cannot be prepared on
// its own).
int gemm_tc_variant(const TcArgs& a, int digits) {
  if (k_chunks(a.K) > 1) return -1;
  const int S = effective_digits(digits, a.K);
  return S * 2 + (a.f32 ? 1 : 0) + 100 * resolve_stages(S, a.f32, a.stages);
}

cudaError_t gemm_tc_prepare(const TcArgs& a, int digits, void* scratch, size_t scratch_bytes, int* err_flag,
                            cudaStream_t st, TcPrepared* out) {
  out->variant = gemm_tc_variant(a, digits);
  out->ctas = a.ctas;
  out->tiles = 0;
  if (a.M <= 0 || a.N <= 0 || a.batch <= 0) return cudaSuccess;
  switch (out->variant % 100) {
    case 4 * 2 + 1: return tc::prepare<4, float>(a, scratch, scratch_bytes, err_flag, st, *out);
    case 4 * 2: return tc::prepare<4, df>(a, scratch, scratch_bytes, err_flag, st, *out);
    case 7 * 2: return tc::prepare<7, df>(a, scratch, scratch_bytes, err_flag, st, *out);
    case 6 * 2: return tc::prepare<6, df>(a, scratch, scratch_bytes, err_flag, st, *out);
    case 2 * 2: return tc::prepare<2, df>(a, scratch, scratch_bytes, err_flag, st, *out);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t gemm_tc_launch(const TcPrepared* const* p, int n, cudaStream_t st, cudaEvent_t* ev) {
  if (n < 1 || n > kTcMaxGroup) return cudaErrorInvalidValue;
  for (int q = 1; q < n; ++q)
    if (p[q]->variant != p[0]->variant) return cudaErrorInvalidValue;
  switch (p[0]->variant) {
    case 300 + 4 * 2 + 1: return tc::launch<4, 3, float>(p, n, st, ev);
    case 200 + 4 * 2 + 1: return tc::launch<4, 2, float>(p, n, st, ev);
    case 300 + 4 * 2: return tc::launch<4, 3, df>(p, n, st, ev);
    case 200 + 4 * 2: return tc::launch<4, 2, df>(p, n, st, ev);
    case 200 + 7 * 2: return tc::launch<7, 2, df>(p, n, st, ev);
    case 300 + 6 * 2: return tc::launch<6, 3, df>(p, n, st, ev);
    case 200 + 6 * 2: return tc::launch<6, 2, df>(p, n, st, ev);
    case 600 + 2 * 2: return tc::launch<2, 6, df>(p, n, st, ev);
    case 400 + 2 * 2: return tc::launch<2, 4, df>(p, n, st, ev);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t gemm_tc(const TcArgs& a, int digits, void* scratch, size_t scratch_bytes, int* err_flag,
                    cudaStream_t st, cudaEvent_t* ev) {
  if (a.M <= 0 || a.N <= 0 || a.batch <= 0) return cudaSuccess;
  const int nc = k_chunks(a.K);
  if (nc > 1 && a.f32) return cudaErrorInvalidValue;  // the FP32 products are short contractions
  if (nc > 1) {
    // split K: chunk c covers k in [k0, k1); op N operands advance along their columns (A) or rows
    // (B), op C ones the other way round
    const int Kc = (a.K + nc - 1) / nc;
    if (ev) cudaEventRecord(ev[0], st);
    for (int c = 0; c < nc; ++c) {
      const int k0 = c * Kc, k1 = a.K < k0 + Kc ? a.K : k0 + Kc;
      TcArgs t = a;
      t.opndA = t.opndB = nullptr;  // kept operands cover whole contractions only
      t.K = k1 - k0;
      t.A = a.A + (a.opA == OP_N ? (long)k0 : (long)k0 * a.lda);
      t.B = a.B + (a.opB == OP_N ? (long)k0 * a.ldb : (long)k0);
      if (c > 0) {
        t.C0 = a.C;
        t.ldc0 = a.ldc;
        t.sC0 = a.sC;
        t.beta = 1.0;
      }
      const cudaError_t e = gemm_tc(t, digits, scratch, scratch_bytes, err_flag, st, nullptr);
      if (e != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[1], st);
    return cudaSuccess;
  }
  TcPrepared p;
  cudaError_t e = gemm_tc_prepare(a, digits, scratch, scratch_bytes, err_flag, st, &p);
  if (e != cudaSuccess) return e;
  const TcPrepared* one[1] = {&p};
  return gemm_tc_launch(one, 1, st, ev);
}

}  // namespace qtx

extern "C" qtx_status qtx_tc_wait_test(int enable) {
  qtx::tc::g_wait_test.store(enable ? 1 : 0, std::memory_order_relaxed);
  return QTX_OK;
}
