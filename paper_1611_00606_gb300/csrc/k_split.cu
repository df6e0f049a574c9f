// Split-precision form of the stacked Hermitian contractions (the five large
// BLAS calls of Algorithm 1: S = A^H A + (UB)^H (UB), H = Z^H B + B^H Z +
// Y^H Y + A_f^H X_f), on BF16 tcgen05 tensor cores.
//
// Slicing (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012, restated for a signed-digit
// split):  every real component x of column g of an operand is written as
//     x = 2^E_g * sum_{p=1..s} d_p 2^{-9(p-1)},   d_1 in [-128, 128],
//                                                  d_p in [-256, 256] (p > 1)
// with E_g chosen per column from the column's largest component (so that
// max|x|/2^E_g lies in [64, 128)).  Every d_p * 2^{-9(p-1)} is exact in
// BF16.  Products of two slices are exact; summed over a window of 128 real K
// the slice-pair levels 0 (d_1 e_1), 1 (d_1 e_2 + d_2 e_1) and
// 2 (d_1 e_3 + d_2 e_2 + d_3 e_1) stay within 2^24 units and are therefore
// exact in FP32 tensor-core accumulators, whatever the accumulator's rounding.
// Levels >= 3 (2^-27 and below) share a fourth, inexact accumulator.  Level 0
// stays exact for 1024 K and level 1 for 256 K, so those two are read out only
// every 8th and every 2nd window.  Read-outs go into a double-float
// (hi, lo FP32 pair) accumulator per output element, scaled by 2^{E_i + E_j}:
// levels 0, 1 and 2 into hi with their rounding errors into lo, levels >= 3 into
// lo (the leading digit is typically small, so level 2 is only ~2^-14 below
// level 0 and would cap the pair's precision if it went to lo directly).  Levels
// 0 and 1 take an error-free TwoSum; level 2, far below hi, takes Fast2Sum (half
// the operations), error-free whenever |hi| >= |level-2 value|, and otherwise
// (a running sum within ~2^-14 of zero) off by at most ~2^-24 of that value.
// The pair is summed to FP64 once per tile at the end.
//
// Complex arithmetic on real tensor cores: with the K-major interleaved
// (re, im) storage, Re(L^H R) = L'^T R' and Im(L^H R) = L'^T R'' where R''
// holds (im, -re) pairs.  One MMA with N = 128 computes a 128 x 64 complex
// tile: B rows 0..63 come from R', rows 64..127 from R''.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"

namespace {

constexpr int BM = 128;        // complex rows per tile (MMA M)
constexpr int BNC = 64;        // complex columns per tile
constexpr int BN = 2 * BNC;    // MMA N (Re | Im)
constexpr int KB = 16;         // real K per pipeline stage (= one MMA K step)
constexpr int WIN = 8;         // stages per exact window (128 real K)
constexpr int ROWS_ALIGN = 128;
constexpr int kMaxBatch = 16;                 // requests per grouped per-atom launch
constexpr int kMaxMaps = 2 + 2 * kMaxBatch;   // >= 13 for a contraction
constexpr int kMaxJobs = 7;
constexpr int TILE_BYTES = 64 * KB * 2;  // one 64-row TMA box: 2 KB
constexpr int NUM_DRAIN_WARPS = 16;     // four per TMEM lane quarter
constexpr int NUM_THREADS = 64 + 32 * NUM_DRAIN_WARPS;  // warp 0 TMA, warp 1 MMA, then drain
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded waits: 2 s
// contraction epilogue staging in the (then idle) stage ring: (hi, lo) float2 as
// [2 strips x 64 columns][128 rows], plus 128 row and 128 column exponents
constexpr int STAGING_CONTRACT = 2 * 64 * 128 * 8 + 256 * 4;
// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when 2 s pass or another role raised the abort flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          volatile int* abort_flag) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*abort_flag) return false;
      const uint64_t now = globaltimer();
      if (t0 == 0) t0 = now;
      else if (now - t0 > kWaitNs) return false;
    }
  }
}
// One box of a blocked slice array starting at (k block, 64-row block, plane); the
// tensor map's box holds 16 elements x 64 rows x 1 k block x (1 or 2) row blocks x
// (s or 2 s) planes, laid out in shared memory in that order, 2 KB per (row block,
// plane): one instruction brings in a whole operand of a pipeline stage.
__device__ __forceinline__ void tma_load_tile(uint32_t dst, const CUtensorMap* map, int kb, int rb,
                                              int plane, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"((uint64_t)map), "r"(0), "r"(0), "r"(kb), "r"(rb), "r"(plane), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// UMMA shared-memory descriptor, K-major, 32-byte swizzle: rows of 32 B
// (16 BF16 along K), 8-row core groups 256 B apart.
__device__ __forceinline__ uint64_t sdesc_sw32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for this layout)
  d |= (uint64_t)(256 >> 4) << 32;            // stride byte offset: 8 rows x 32 B
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)6 << 61;                     // swizzle mode: 32 B
  return d;
}
// Instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ float pow2f(int e) {
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return __int_as_float((e + 127) << 23);
}
// Column pairs of the (hi, lo) accumulators live in 64-bit registers and are
// updated with Blackwell's packed FP32 pair arithmetic (round to nearest, as
// TwoSum requires), two columns per instruction.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pack2(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 unpack2(f32x2 r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// Error-free TwoSum of both lanes: hi + v = s + e exactly; hi = s, lo += e.
__device__ __forceinline__ void two_sum_acc2(f32x2& hi, f32x2& lo, f32x2 v) {
  const f32x2 s = add2(hi, v);
  const f32x2 bp = sub2(s, hi);
  const f32x2 ap = sub2(s, bp);
  lo = add2(lo, add2(sub2(hi, ap), sub2(v, bp)));
  hi = s;
}


// Fast2Sum of both lanes (exact when |hi| >= |v|): hi + v = s + e; hi = s, lo += e.
__device__ __forceinline__ void fast_two_sum_acc2(f32x2& hi, f32x2& lo, f32x2 v) {
  const f32x2 s = add2(hi, v);
  lo = add2(lo, sub2(v, sub2(s, hi)));
  hi = s;
}

// Drain 16 TMEM columns of the accumulators in `mask` (level k at column offset
// k*BN) into (hi, lo) pairs kept in units of the current segment's scale
// 2^(E_row + E_col): the window sums of levels 0-2 are exact integers and go into
// hi (TwoSum for levels 0 and 1, Fast2Sum for level 2, read after them); levels
// >= 3 go into lo.
template <int S, uint32_t MASK>
__device__ __forceinline__ void drain16(uint32_t taddr, f32x2 (&hi)[8], f32x2 (&lo)[8]) {
  constexpr bool r0 = MASK & 1u, r1 = MASK & 2u, r2 = S >= 3 && (MASK & 4u),
                 r3 = S >= 4 && (MASK & 8u);
#pragma unroll
  for (int c0 = 0; c0 < 16; c0 += 4) {
    float v0[4], v1[4], v2[4], v3[4];
    if (r0) tmem_ld4(taddr + c0, v0);
    if (r1) tmem_ld4(taddr + BN + c0, v1);
    if (r2) tmem_ld4(taddr + 2 * BN + c0, v2);
    if (r3) tmem_ld4(taddr + 3 * BN + c0, v3);
    tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < 4; c += 2) {
      const int k = (c0 + c) >> 1;
      if (r0) two_sum_acc2(hi[k], lo[k], pack2(v0[c], v0[c + 1]));
      if (r1) two_sum_acc2(hi[k], lo[k], pack2(v1[c], v1[c + 1]));
      if (r2) fast_two_sum_acc2(hi[k], lo[k], pack2(v2[c], v2[c + 1]));
      if (r3) lo[k] = add2(lo[k], pack2(v3[c], v3[c + 1]));
    }
  }
}

// Both 64-column strips of one window read-out; `mask` is one of due_mask()'s values.
template <int S>
__device__ __forceinline__ void drain_window(uint32_t tl, uint32_t mask, f32x2 (&h0)[8],
                                             f32x2 (&l0)[8], f32x2 (&h1)[8], f32x2 (&l1)[8]) {
  if (mask == 0xFu) {
    drain16<S, 0xFu>(tl, h0, l0);
    drain16<S, 0xFu>(tl + (uint32_t)BNC, h1, l1);
  } else if (mask == 0xEu) {
    drain16<S, 0xEu>(tl, h0, l0);
    drain16<S, 0xEu>(tl + (uint32_t)BNC, h1, l1);
  } else {
    drain16<S, 0xCu>(tl, h0, l0);
    drain16<S, 0xCu>(tl + (uint32_t)BNC, h1, l1);
  }
}

// (hi + lo) * 2^k as FP64, the same value as ((double)hi + (double)lo) * 2^k
// but with one FP64 instruction instead of four: GB300 issues FP64 at about two per
// clock per SM, which made the per-atom epilogue (8192 complex results per CTA) longer
// than its MMAs.  The widening conversions and the power-of-two scaling are exact
// bit operations (FP32 subnormals take the library conversion; zero, Inf and NaN are
// left unscaled; |k| stays well inside the exponent range).
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  if (e == 0u && (b & 0x7FFFFFu) != 0u) return (double)f;
  const uint64_t e64 = e == 0u ? 0u : (e == 0xFFu ? 0x7FFu : e + 896u);
  return __longlong_as_double((long long)(((uint64_t)(b >> 31) << 63) | (e64 << 52) |
                                          ((uint64_t)(b & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ double pair_scaled(float hi, float lo, int k) {
  long long b = __double_as_longlong(f32_to_f64(hi) + f32_to_f64(lo));
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex != 0 && ex != 0x7FF) b += (long long)k << 52;
  return __longlong_as_double(b);
}

// ------------------------------------------------------------------ slice-GEMM kernel
//
// One kernel body serves two work decompositions (template MODE):
//  * MODE_CONTRACT: a 128 x 64 complex lower-triangle tile of S or H; K runs
//    over the contraction's segments (L', R', R'' slice arrays).
//  * MODE_ATOMS: the per-atom products of Algorithm 1's loops,
//      Z_a = [T^BA_a | 1/2 T^BB_a] [A_a; B_a],  W2_slot(a) = M2_a A_a,
//    as D[g][n] = sum_k X'[g][k] Op_a[n][k] with X' the coefficient slices of
//    atom a (rows g) and Op_a the sliced real form of the per-atom operator
//    (row n = 2L + c gives Re/Im of output row L).  Tile: 128 g x 128 n.
// Both share the TMA -> smem ring, the tcgen05 issue loop, the exact-window
// TMEM accumulators and the double-float drain; they differ in where each
// K segment's tiles come from, which exponents scale the drain, and the
// epilogue.

// The _R modes are the real-symmetric variant (real A, B, T, U; H, S real symmetric,
// Sec. 1.1): operands hold one real K position per row, contraction tiles are
// 128 x 128 real outputs (B rows = 128 columns of R'), operator rows n = L.
enum { MODE_CONTRACT = 0, MODE_ATOMS = 1, MODE_CONTRACT_R = 2, MODE_ATOMS_R = 3 };
__host__ __device__ constexpr bool is_contract(int mode) { return (mode & 1) == 0; }
__host__ __device__ constexpr bool is_real(int mode) { return mode >= 2; }

struct SplitSeg {
  int mL, mR;       // tensor maps: L' as the left operand, R as the right one
                    // (complex: its plain and rotated slices, interleaved by plane)
  int kblocks;      // stages of KB real K
  const int* eL;    // exponents of the L source columns
  const int* eR;    // exponents of the R source columns
};

// One request of a grouped per-atom launch.
struct AtomsReq {
  int mA, mB;         // coefficient slice maps (plain) of this request
  const int* eA;      // column exponents of its A, B slices
  const int* eB;
  double2* Z;         // outputs, column-major, leading dimension AtomsArgs::ld
  double2* W2;
  int N_G;
  int ngblk;          // 128-row blocks of G
  int tile0;          // first CTA index of this request in the grouped grid
};

struct AtomsArgs {
  AtomsReq rq[kMaxBatch];
  int nreq;
  int mOp[2];             // operator slice maps: [0] Z job, [1] W2 job (shared by requests)
  const int* eOp[2];      // operator row exponents [a][n_pad]
  const int* slot;        // W2 slot of each atom
  int ld;
  int N_A, N_L, P;        // P: operator K per part (an atom's widest K block range)
  int n_pad, ntile;
};

struct SplitParams {
  CUtensorMap maps[kMaxMaps];
  SplitSeg seg[kMaxSeg];
  int nseg;
  int s;          // slices
  int n_stage;    // pipeline depth
  int N_G, ldC, nbj;
  int nbi, band;   // contraction: 128-row blocks, row blocks per band of the tile order
  int bi0;         // contraction: first row block of this launch (tiles of rows [bi0, nbi))
  int ntiles;      // tiles of the launch; a CTA runs tiles blockIdx.x, + gridDim.x, ...
  int rows_pad;   // slice p of a coefficient-side array starts at row p * rows_pad
  double2* C;
  int* err;
  int stall;  // test only: the producer arms no stage and issues no copy, so the MMA
              // thread's and the drain's waits run out (failure-path test)
  AtomsArgs at;
};

// Where one K segment of this CTA's tile lives (blocked slice arrays:
// plane = slice p (+ atom * s for operators), 64-row blocks, 16-wide K blocks).
struct SegInfo {
  const CUtensorMap* mL;
  const CUtensorMap* mR;
  int kbL, rbL, plL;        // L side: first K block, first 64-row block, plane of slice 0
  int kbR, rbR, plR;        // R side: first K block, first 64-row block, plane of slice 0
  int kblocks;
  const int* eRow;          // indexed by the tile's absolute row
  const int* eC0;           // column exponents of TMEM columns [0, 64) (+ column in strip)
  const int* eC1;           // columns [64, 128)
};

struct TileId {
  int i0, j0;      // CONTRACT: row / column origin
  int a, job, n0;  // ATOMS: atom, job (0: Z, 1: W2), operator row origin (i0 = g origin)
  int r;           // ATOMS: request of the grouped launch
  int N_G;         // columns of the (request's) output
  int nseg;
};

template <int MODE>
__device__ __forceinline__ TileId decode_tile(const SplitParams& P, int tile) {
  TileId t{};
  constexpr bool R = is_real(MODE);  // column pairs of 2 x 128 real columns, pair c from row 2c
  if (is_contract(MODE)) {
    // Consecutive tiles 2p, 2p + 1 are column blocks 2c and 2c + 1 of one row block
    // (they read the same L' boxes, which the second finds in L2); row block bi
    // holds column pairs c <= bi (c < npr), so only an odd nbj leaves the last pair
    // a block past the matrix (zero slices, nothing stored).  Pairs are numbered
    // band by band (P.band row blocks per band) and column-major inside a band, so
    // the CTAs resident at one time cover a compact block of rows x columns and
    // share their operand tiles in L2.
    const int npr = (P.nbj + 1) >> 1;
    int p = tile >> 1, bi = 0, c = 0;
    for (int b0 = P.bi0; b0 < P.nbi; b0 += P.band) {
      const int b1 = min(b0 + P.band, P.nbi);
      int n = 0;
      for (int r = b0; r < b1; ++r) n += min((R ? r / 2 : r) + 1, npr);
      if (p < n) {
        for (c = 0; c < npr; ++c) {
          const int lo = max(b0, R ? 2 * c : c), cnt = b1 - lo;
          if (p < cnt) {
            bi = lo + p;
            break;
          }
          p -= cnt;
        }
        break;
      }
      p -= n;
    }
    t.i0 = bi * BM;
    t.j0 = (2 * c + (tile & 1)) * (R ? BN : BNC);
    t.nseg = P.nseg;
    t.N_G = P.N_G;
  } else {
    int r = 0;
    while (r + 1 < P.at.nreq && tile >= P.at.rq[r + 1].tile0) ++r;
    const AtomsReq& R = P.at.rq[r];
    int b = tile - R.tile0;
    t.r = r;
    t.N_G = R.N_G;
    const int gb = b % R.ngblk;
    b /= R.ngblk;
    const int nt = b % P.at.ntile;
    b /= P.at.ntile;
    t.job = b & 1;
    t.a = b >> 1;
    t.i0 = gb * BM;
    t.n0 = nt * BN;
    t.nseg = t.job == 0 ? 2 : 1;
  }
  return t;
}

template <int MODE>
__device__ __forceinline__ SegInfo seg_info(const SplitParams& P, const TileId& t, int sg) {
  SegInfo si;
  if (is_contract(MODE)) {
    // complex: B rows 0..63 from R' and 64..127 from R'' (same 64 columns: the R box
    // is one row block of the interleaved plain / rotated planes); real: B rows = 128
    // consecutive columns of R' (a box of two row blocks)
    const SplitSeg& S = P.seg[sg];
    si.mL = &P.maps[S.mL];
    si.mR = &P.maps[S.mR];
    si.kbL = 0;
    si.rbL = t.i0 >> 6;
    si.plL = 0;
    si.kbR = 0;
    si.rbR = t.j0 >> 6;
    si.plR = 0;
    si.kblocks = S.kblocks;
    si.eRow = S.eL;
    si.eC0 = S.eR + t.j0;
    si.eC1 = S.eR + t.j0 + (is_real(MODE) ? 64 : 0);
  } else {
    const AtomsArgs& A = P.at;
    const AtomsReq& R = A.rq[t.r];
    si.mL = &P.maps[sg == 0 ? R.mA : R.mB];
    si.mR = &P.maps[A.mOp[t.job]];
    const int pr = is_real(MODE) ? 1 : 2;  // real K positions per row
    si.kbL = (pr * t.a * A.N_L) / KB;  // atom a's rows in the packed layout
    si.rbL = t.i0 >> 6;
    si.plL = 0;
    si.kbR = sg * (A.P / KB);  // Z operator: A part in [0, P), B part in [P, 2P)
    si.rbR = t.n0 >> 6;
    si.plR = t.a * P.s;
    si.kblocks = (pr * (t.a + 1) * A.N_L + KB - 1) / KB - si.kbL;
    si.eRow = sg == 0 ? R.eA : R.eB;
    si.eC0 = A.eOp[t.job] + t.a * A.n_pad + t.n0;
    si.eC1 = si.eC0 + 64;
  }
  return si;
}

// Issue one stage's slice-pair MMAs: pairs (p, q) with p + q < S go to the
// accumulator of level min(p + q, 3).  Fully unrolled for a compile-time slice
// count; the descriptors of slice p / q are the stage's base descriptors plus a
// constant (the 14-bit start-address field holds address >> 4 and stays below
// 2^14 for any smem address).  Accumulators in `init_mask` restart: the first
// pair of their level overwrites instead of adding.
// Accumulators read out after window w of a segment (bit k: accumulator k).  Each
// level stays exact for as long as its bound allows: level 0 (<= 2^14 per real K)
// for 1024 K = 8 windows, level 1 (<= 2^16) for 256 K = 2 windows, level 2 for one
// window; levels >= 3 are inexact and read every window.  The last window of a
// segment reads everything (the next segment has another scale).
__device__ __forceinline__ uint32_t due_mask(int w, bool last) {
  if (last) return 0xFu;
  uint32_t m = 0xCu;                 // levels 2 and >= 3
  if ((w & 1) == 1) m |= 0x2u;       // level 1
  if ((w & 7) == 7) m |= 0x1u;       // level 0
  return m;
}

template <int S>
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint64_t ad0, uint64_t bd0,
                                            uint32_t init_mask) {
#pragma unroll
  for (int p = 0; p < S; ++p) {
#pragma unroll
    for (int q = 0; q < S - p; ++q) {
      constexpr int kStep = (2 * TILE_BYTES) >> 4;
      const int lvl = p + q;
      const int acc = lvl < 3 ? lvl : 3;
      const bool lead = (p == 0 && q == acc);  // first pair of its level within a stage
      tc_mma_bf16(tmem + acc * BN, ad0 + (uint64_t)(p * kStep), bd0 + (uint64_t)(q * kStep), kIdesc,
                  (lead && ((init_mask >> acc) & 1u)) ? 0u : 1u);
    }
  }
}

template <int MODE, int S>
__global__ void __launch_bounds__(NUM_THREADS, 1) k_split_gemm(const __grid_constant__ SplitParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int s = S;
  const int NS = P.n_stage;
  const uint32_t a_bytes = (uint32_t)s * 2 * TILE_BYTES;   // s slices x 128 rows
  const uint32_t stage_bytes = 2 * a_bytes;                 // A part + B part
  const uint32_t ring_bytes =
      is_contract(MODE) ? max(NS * stage_bytes, (uint32_t)STAGING_CONTRACT) : NS * stage_bytes;
  uint64_t* full = (uint64_t*)(smem + ring_bytes);
  uint64_t* empty = full + NS;
  uint64_t* acc_full = empty + NS;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* done = acc_empty + 1;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const TileId T0 = decode_tile<MODE>(P, blockIdx.x);  // first tile (tensor-map prefetch)

  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);  // released by the MMA thread's commit
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, NUM_DRAIN_WARPS);
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0 && lane == 0)
    for (int sg = 0; sg < T0.nseg; ++sg) {
      const SegInfo si = seg_info<MODE>(P, T0, sg);
      prefetch_map(si.mL);
      prefetch_map(si.mR);
    }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && P.stall) {
    // ---------------- stall injection (test only): nothing is armed and nothing is in
    // flight, so the MMA thread's and the drain's bounded waits run out
  } else if (warp == 0) {
    // ---------------- TMA producer (lane 0): waits for a free stage, arms it and
    // issues its two boxes, every slice of L' (A operand) and of R (B operand)
    int slot = 0;
    uint32_t phase = 0;
    uint32_t armed = 0;        // bit i: slot i was armed at least once
    uint32_t armed_par = 0;    // bit i: parity of the last armed phase of slot i
    bool ok = true;
    if (lane == 0)
    for (int tile = blockIdx.x; tile < P.ntiles && ok; tile += gridDim.x) {
     const TileId T = decode_tile<MODE>(P, tile);
     for (int sg = 0; sg < T.nseg && ok; ++sg) {
      const SegInfo si = seg_info<MODE>(P, T, sg);
      for (int kb = 0; kb < si.kblocks; ++kb) {
        ok = mbar_wait(&empty[slot], phase ^ 1u, abort_flag);
        if (!ok) break;
        mbar_expect_tx(&full[slot], stage_bytes);
        armed |= 1u << slot;
        armed_par = (armed_par & ~(1u << slot)) | (phase << slot);
        const uint32_t sa = smem_u32(smem + slot * stage_bytes);
        // A: [slice p][row half][64 rows][16] (slice p at p x 4 KB); B: [slice q][R' | R''
        // or the two row halves][64 rows][16] (slice q at q x 4 KB); a_bytes each
        tma_load_tile(sa, si.mL, si.kbL + kb, si.rbL, si.plL, &full[slot]);
        tma_load_tile(sa + a_bytes, si.mR, si.kbR + kb, si.rbR, si.plR, &full[slot]);
        if (++slot == NS) {
          slot = 0;
          phase ^= 1u;
        }
      }
     }
    }
    if (lane == 0) {
      if (!ok) {
        atomicExch(P.err, 1);
        *abort_flag = 1;
      }
      // never leave with bulk copies in flight: wait for every armed phase
      for (int i = 0; i < NS; ++i)
        if (armed & (1u << i)) {
          uint64_t t0 = globaltimer();
          while (!mbar_try(&full[i], (armed_par >> i) & 1u))
            if (globaltimer() - t0 > kWaitNs) break;
        }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (one thread)
    if (lane == 0) {
      int slot = 0;
      uint32_t phase = 0;
      int nwin = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < P.ntiles && ok; tile += gridDim.x) {
       const TileId T = decode_tile<MODE>(P, tile);
       for (int sg = 0; sg < T.nseg && ok; ++sg) {
        const int kbn = seg_info<MODE>(P, T, sg).kblocks;
        uint32_t restart = 0xFu;  // accumulators to restart in the next window
        for (int w0 = 0; w0 < kbn && ok; w0 += WIN) {
          if (nwin > 0 && !mbar_wait(acc_empty, (uint32_t)(nwin - 1) & 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int w1 = min(kbn, w0 + WIN);
          const uint32_t first_mask = restart;
          restart = due_mask(w0 / WIN, w1 == kbn);
          for (int kb = w0; kb < w1; ++kb) {
            if (!mbar_wait(&full[slot], phase, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + slot * stage_bytes);
            issue_stage<S>(tmem, sdesc_sw32(sa), sdesc_sw32(sa + a_bytes),
                           kb == w0 ? first_mask : 0u);
            tc_commit(&empty[slot]);
            if (++slot == NS) {
              slot = 0;
              phase ^= 1u;
            }
          }
          if (ok) tc_commit(acc_full);
          ++nwin;
        }
       }
      }
      if (!ok) {
        atomicExch(P.err, 2);
        *abort_flag = 1;
      }
      // all MMAs retired before the accumulators are freed
      tc_commit(done);
      uint64_t t0 = globaltimer();
      while (!mbar_try(done, 0))
        if (globaltimer() - t0 > kWaitNs) break;
    }
  } else {
    // ---------------- drain warps: TMEM -> double-float accumulators, then the tile's
    // results straight from registers (the next tile's MMAs start as soon as the last
    // read-out has released the accumulators, so these stores overlap them)
    const int q4 = warp & 3;         // TMEM lane quarter this warp may access
    const int cg = (warp - 2) >> 2;  // 16-column group of each 64-column strip
    const uint32_t tl = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(16 * cg);
    int nwin = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < P.ntiles && ok; tile += gridDim.x) {
      const TileId T = decode_tile<MODE>(P, tile);
      const int row = T.i0 + 32 * q4 + lane;
      f32x2 h0[8], l0[8], h1[8], l1[8];  // column pairs of strip 0 (TMEM cols < 64), strip 1
#pragma unroll
      for (int c = 0; c < 8; ++c) h0[c] = l0[c] = h1[c] = l1[c] = 0ull;
      int eRow = 0, eC0 = 0, eC1 = 0;  // current segment's exponents (lane c: column c)
      for (int sg = 0; sg < T.nseg && ok; ++sg) {
        const SegInfo si = seg_info<MODE>(P, T, sg);
        const int nRow = si.eRow[row];
        const int nC0 = si.eC0[16 * cg + (lane & 15)];
        const int nC1 = si.eC1[16 * cg + (lane & 15)];
        if (sg > 0) {  // move the pairs into the new segment's units (exact powers of two)
#pragma unroll
          for (int c = 0; c < 16; c += 2) {
            const int dr = eRow - nRow;
            const f32x2 f0 = pack2(pow2f(dr + __shfl_sync(0xffffffffu, eC0 - nC0, c)),
                                   pow2f(dr + __shfl_sync(0xffffffffu, eC0 - nC0, c + 1)));
            const f32x2 f1 = pack2(pow2f(dr + __shfl_sync(0xffffffffu, eC1 - nC1, c)),
                                   pow2f(dr + __shfl_sync(0xffffffffu, eC1 - nC1, c + 1)));
            h0[c >> 1] = mul2(h0[c >> 1], f0);
            l0[c >> 1] = mul2(l0[c >> 1], f0);
            h1[c >> 1] = mul2(h1[c >> 1], f1);
            l1[c >> 1] = mul2(l1[c >> 1], f1);
          }
        }
        eRow = nRow;
        eC0 = nC0;
        eC1 = nC1;
        for (int w0 = 0; w0 < si.kblocks; w0 += WIN) {
          if (!mbar_wait(acc_full, (uint32_t)nwin & 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          drain_window<S>(tl, due_mask(w0 / WIN, w0 + WIN >= si.kblocks), h0, l0, h1, l1);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acc_empty);
          ++nwin;
        }
      }
      if (!ok || *abort_flag) break;
      // Results: (hi + lo) * 2^(E_row + E_col) in FP64.  Thread = one tile row; pair k
      // of a strip = its TMEM columns 16 cg + 2k and 2k + 1 (lanes 2k, 2k + 1 of eC*).
      if (is_contract(MODE)) {
        // one tile per CTA: stage (hi, lo) in the idle ring (every stage was consumed by
        // an MMA that completed before the last acc_full), then write the tile with
        // consecutive threads on consecutive output addresses
        float2* stg = (float2*)smem;  // [2 strips][64 cols][128 rows]
        int* s_erow = (int*)(smem + 2 * 64 * 128 * sizeof(float2));
        int* s_ecol = s_erow + 128;   // [128]: exponent of each TMEM column
        const int r = 32 * q4 + lane;
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
          const float2 ha = unpack2(h0[c >> 1]), la = unpack2(l0[c >> 1]);
          const float2 hb = unpack2(h1[c >> 1]), lb = unpack2(l1[c >> 1]);
          stg[(0 * 64 + 16 * cg + c) * 128 + r] = make_float2(ha.x, la.x);
          stg[(0 * 64 + 16 * cg + c + 1) * 128 + r] = make_float2(ha.y, la.y);
          stg[(1 * 64 + 16 * cg + c) * 128 + r] = make_float2(hb.x, lb.x);
          stg[(1 * 64 + 16 * cg + c + 1) * 128 + r] = make_float2(hb.y, lb.y);
        }
        if (cg == 0) s_erow[r] = eRow;
        if (q4 == 0 && lane < 16) {
          s_ecol[16 * cg + lane] = eC0;
          s_ecol[64 + 16 * cg + lane] = eC1;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * NUM_DRAIN_WARPS) : "memory");
        const int dt = threadIdx.x - 64;  // 0 .. 32*NUM_DRAIN_WARPS-1
        if (is_real(MODE)) {  // 128 real columns
          double* C = (double*)P.C;
          for (int idx = dt; idx < 128 * 128; idx += 32 * NUM_DRAIN_WARPS) {
            const int jj = idx >> 7, ii = idx & 127;
            const int i = T.i0 + ii, j = T.j0 + jj;
            if (i < P.N_G && j < P.N_G) {
              const float2 v = stg[jj * 128 + ii];
              C[i + (size_t)j * P.ldC] = pair_scaled(v.x, v.y, s_erow[ii] + s_ecol[jj]);
            }
          }
        } else
        for (int idx = dt; idx < 64 * 128; idx += 32 * NUM_DRAIN_WARPS) {
          const int jj = idx >> 7, ii = idx & 127;
          const int i = T.i0 + ii, j = T.j0 + jj;
          if (i < P.N_G && j < P.N_G) {
            const int k = s_erow[ii] + s_ecol[jj];
            const float2 re = stg[jj * 128 + ii], im = stg[(64 + jj) * 128 + ii];
            P.C[i + (size_t)j * P.ldC] = make_double2(pair_scaled(re.x, re.y, k),
                                                      pair_scaled(im.x, im.y, k));
          }
        }
      } else if (is_real(MODE)) {
        // TMEM column c of strip t = output row L = n0 + 64 t + c (real); each thread
        // writes pairs of consecutive rows
        const AtomsArgs& A = P.at;
        const AtomsReq& R = A.rq[T.r];
        double* out = T.job == 0 ? (double*)R.Z + (size_t)T.a * A.N_L
                                 : (double*)R.W2 + (size_t)A.slot[T.a] * A.N_L;
        const int g = row;
        const int Lb = T.n0 + 16 * cg;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int e00 = eRow + __shfl_sync(0xffffffffu, eC0, 2 * k);
          const int e01 = eRow + __shfl_sync(0xffffffffu, eC0, 2 * k + 1);
          const int e10 = eRow + __shfl_sync(0xffffffffu, eC1, 2 * k);
          const int e11 = eRow + __shfl_sync(0xffffffffu, eC1, 2 * k + 1);
          const float2 ha = unpack2(h0[k]), la = unpack2(l0[k]);
          const float2 hb = unpack2(h1[k]), lb = unpack2(l1[k]);
          const int L0 = Lb + 2 * k, L1 = Lb + 64 + 2 * k;
          double* o = out + (size_t)g * A.ld;
          if (g < T.N_G) {
            if (L0 < A.N_L) o[L0] = pair_scaled(ha.x, la.x, e00);
            if (L0 + 1 < A.N_L) o[L0 + 1] = pair_scaled(ha.y, la.y, e01);
            if (L1 < A.N_L) o[L1] = pair_scaled(hb.x, lb.x, e10);
            if (L1 + 1 < A.N_L) o[L1 + 1] = pair_scaled(hb.y, lb.y, e11);
          }
        }
      } else {
        // columns (2k, 2k + 1) of a strip = Re, Im of output row L: strip 0 holds
        // L = 8 cg + k, strip 1 L + 32; each thread writes 8 consecutive complex
        // values (128 contiguous bytes) per strip
        const AtomsArgs& A = P.at;
        const AtomsReq& R = A.rq[T.r];
        double2* out = T.job == 0 ? R.Z + (size_t)T.a * A.N_L
                                  : R.W2 + (size_t)A.slot[T.a] * A.N_L;
        const int g = row;
        const int Lb = (T.n0 >> 1) + 8 * cg;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int e0r = eRow + __shfl_sync(0xffffffffu, eC0, 2 * k);
          const int e0i = eRow + __shfl_sync(0xffffffffu, eC0, 2 * k + 1);
          const int e1r = eRow + __shfl_sync(0xffffffffu, eC1, 2 * k);
          const int e1i = eRow + __shfl_sync(0xffffffffu, eC1, 2 * k + 1);
          const float2 ha = unpack2(h0[k]), la = unpack2(l0[k]);
          const float2 hb = unpack2(h1[k]), lb = unpack2(l1[k]);
          const int L0 = Lb + k, L1 = Lb + 32 + k;
          if (g < T.N_G && L0 < A.N_L)
            out[(size_t)L0 + (size_t)g * A.ld] =
                make_double2(pair_scaled(ha.x, la.x, e0r), pair_scaled(ha.y, la.y, e0i));
          if (g < T.N_G && L1 < A.N_L)
            out[(size_t)L1 + (size_t)g * A.ld] =
                make_double2(pair_scaled(hb.x, lb.x, e1r), pair_scaled(hb.y, lb.y, e1i));
        }
      }
    }
    if (!ok) {
      atomicExch(P.err, 3);
      *abort_flag = 1;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ------------------------------------------------------------------ slicers

// Layout shared by every coefficient-side slice array.  Along K the source's
// complex rows are packed: row k sits at real position 2k (+1 for the imaginary
// part), and the length 2 nblk N_L is padded with zeros to kpad = roundup(., 16).
// A contraction runs over kpad real K; the per-atom products read atom a's rows
// [2 a N_L, 2 (a+1) N_L) as whole 16-wide K blocks, the operator slices of atom a
// being shifted by the same offset (2 a N_L) mod 16 and zero outside the atom.
// In memory each slice plane is blocked as [64-row block][16-wide K block][64 rows]
// [16 elements]: one 2 KB tile per (row block, K block), contiguous, which is
// exactly one TMA box (the TMA applies the 32-byte swizzle on the way to smem).
__device__ __forceinline__ size_t tile_off(int row, int j, int NKB) {
  // element offset of the complex pair j (real elements 2j, 2j+1) of a row
  return ((size_t)((row >> 6) * NKB + (j >> 3)) * 64 + (row & 63)) * 16 + 2 * (j & 7);
}
struct SliceJob {
  const double2* X;  // source: nblk * N_L complex rows x N_G, column-major, ld ldX
  const double* u;   // optional real row weight (the U norms), may be null
  uint16_t* plain;   // [s][rows_pad][kpad] BF16 slices of (re, im) pairs, or with rot
                     // [s][2][rows_pad][kpad]: (re, im) and (im, -re) slices interleaved
  int rot;           // nonzero: also write the (im, -re) slices
  int* expo;         // [rows_pad] column exponents
  int ldX, nblk;
};
struct SliceParams {
  SliceJob job[kMaxJobs];
  int s, N_G, rows_pad, N_L;
  int g0;  // first operand column of this launch (block x slices column g0 + x)
};

// Balanced base-512 digits of round(x * 2^(9(s-1) - E)); d[0] is the leading one.
__device__ __forceinline__ void digits_of(double x, int E, int s, int (&d)[kMaxSlices]) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long Y = 0;
  if (ex != 0) {
    const long long m = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
    const int sh = ex - 1075 - E + 9 * (s - 1);
    if (sh >= 0) {
      Y = m << sh;
    } else if (sh > -63) {
      const int n = -sh;
      Y = (m + (1LL << (n - 1))) >> n;
    }
    if (bits < 0) Y = -Y;
  }
#pragma unroll
  for (int p = kMaxSlices - 1; p >= 1; --p) {
    if (p < s) {
      const long long dp = ((Y + 256) & 511) - 256;
      d[p] = (int)dp;
      Y = (Y - dp) >> 9;
    }
  }
  d[0] = (int)Y;
}

// BF16 bits of d * sc for a digit |d| <= 256 and sc = 2^-9p: the value has at most 8
// significant bits, so it is exact in BF16 and its BF16 bits are the upper half of its
// FP32 bits.  d converts with the 1.5 * 2^23 magic number (FP32 add, exact for
// |d| < 2^22) instead of an int-to-float conversion: the slicer writes 20 BF16 values
// per complex entry and the conversion units (a quarter of the FP32 rate) were its
// limit.
__device__ __forceinline__ uint32_t bf16_digit(int d, float sc) {
  const float f = (__int_as_float(0x4B400000 + d) - 12582912.0f) * sc;
  return __float_as_uint(f) >> 16;
}

// |x| as its bit pattern (non-negative doubles order like their bit patterns), 0 for a
// non-finite x: column maxima are taken with integer instructions, off the FP64 pipe
// (about two instructions per clock per SM on GB300).
__device__ __forceinline__ unsigned long long finite_abs_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  return (b >> 52) == 0x7FFull ? 0ull : b;
}
__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7FF) != 0x7FF;
}

// Exponent E with max / 2^E in [64, 128) (0 for an all-zero or non-finite max).
__device__ __forceinline__ int slice_exponent(double mm) {
  int e = 0;
  if (mm > 0.0 && isfinite(mm)) {
    frexp(mm, &e);
    return e - 7;
  }
  return 0;
}

// Write the s slices of one complex entry (re, im): plain (re, im) at base + p pstride +
// off and, with rot, rotated (im, -re) at base + rot_off + p pstride + off.
__device__ __forceinline__ void put_slices(double2 v, bool zero, int E, int s, uint16_t* base,
                                           bool rot, size_t pstride, size_t rot_off,
                                           size_t off) {
  int dr[kMaxSlices], di[kMaxSlices];
  const bool bad = !zero && !(finite_bits(v.x) && finite_bits(v.y));
  if (!zero) {
    digits_of(v.x, E, s, dr);
    digits_of(v.y, E, s, di);
  } else {
#pragma unroll
    for (int p = 0; p < kMaxSlices; ++p) dr[p] = di[p] = 0;
  }
#pragma unroll
  for (int p = 0; p < kMaxSlices; ++p) {
    if (p < s) {
      const float sc = __int_as_float((127 - 9 * p) << 23);  // 2^{-9p}
      uint32_t pl, rt;
      if (bad) {
        pl = rt = 0x7FC07FC0u;  // NaN pair: propagates through the MMA
      } else {
        const uint32_t br = bf16_digit(dr[p], sc), bi = bf16_digit(di[p], sc);
        pl = br | (bi << 16);
        rt = bi | ((br == 0u ? 0u : br ^ 0x8000u) << 16);  // -dr: sign flip (zero stays +0)
      }
      *(uint32_t*)(base + p * pstride + off) = pl;
      if (rot) *(uint32_t*)(base + rot_off + p * pstride + off) = rt;
    }
  }
}

__global__ void __launch_bounds__(256) k_slice(const __grid_constant__ SliceParams P) {
  const SliceJob J = P.job[blockIdx.y];
  const int g = P.g0 + blockIdx.x;
  const int s = P.s;
  const int K = J.nblk * P.N_L;                  // complex rows of the source
  const int kpad = ((2 * K + KB - 1) / KB) * KB;  // packed real K, whole 16-wide blocks
  const size_t slice_elems = (size_t)P.rows_pad * kpad;
  const size_t pstride = (J.rot ? 2 : 1) * slice_elems;  // plain slice p at p pstride
  __shared__ unsigned long long red[32];
  __shared__ int s_E;
  const int kc = kpad / 2;  // complex positions per padded row
  const int NKB = kpad / KB;
  if (g >= P.N_G) {
    for (int k = threadIdx.x; k < kc; k += blockDim.x)
      for (int p = 0; p < s; ++p) {
        *(uint32_t*)(J.plain + p * pstride + tile_off(g, k, NKB)) = 0u;
        if (J.rot) *(uint32_t*)(J.plain + slice_elems + p * pstride + tile_off(g, k, NKB)) = 0u;
      }
    if (threadIdx.x == 0) J.expo[g] = 0;
    return;
  }
  const double2* col = J.X + (size_t)g * J.ldX;
  unsigned long long m = 0ull;  // bit pattern of the column's largest finite |component| (x |u|)
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double2 v = col[k];
    unsigned long long a = max(finite_abs_bits(v.x), finite_abs_bits(v.y));
    if (J.u) a = finite_abs_bits(__longlong_as_double((long long)a) * fabs(J.u[k]));
    m = max(m, a);
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long mm = 0ull;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = max(mm, red[i]);
    s_E = slice_exponent(__longlong_as_double((long long)mm));
    J.expo[g] = s_E;
  }
  __syncthreads();
  const int E = s_E;
  for (int j = threadIdx.x; j < kc; j += blockDim.x) {
    const bool zero = (j >= K);
    double2 v = make_double2(0.0, 0.0);
    if (!zero) {
      v = col[j];
      if (J.u) {
        v.x *= J.u[j];
        v.y *= J.u[j];
      }
    }
    put_slices(v, zero, E, s, J.plain, J.rot != 0, pstride, slice_elems, tile_off(g, j, NKB));
  }
}

// Slices of the per-atom operators (k-independent, once per factorisation):
// job 0: MZ[a] (N_L x 2N_L), K = [A part | B part] = 2P; job 1: M2[a] (N_L x N_L),
// K = P, P = the widest K block range of an atom in the packed coefficient layout.
// Column l of a part sits at real position (2 a N_L) mod 16 + 2l, the offset of
// atom a's rows inside its first K block, zeros elsewhere.  Real row n = 2L + c of
// output row L: c = 0 gives Re, c = 1 gives Im:
//   row 2L:   (Re M(L,k), -Im M(L,k)) pairs;   row 2L+1: (Im M(L,k), Re M(L,k)).
// Layout [a][p][n_pad][Kop]; one exponent per (a, n), shared by rows 2L, 2L+1.
__global__ void __launch_bounds__(128) k_slice_op(const double2* __restrict__ M, int job, int N_A,
                                                  int N_L, int P, int n_pad, int s,
                                                  uint16_t* __restrict__ out,
                                                  int* __restrict__ expo) {
  const int a = blockIdx.y, n = blockIdx.x;  // n < n_pad
  const int parts = job == 0 ? 2 : 1;
  const int Kop = parts * P;
  const size_t slice_elems = (size_t)n_pad * Kop;
  uint16_t* base = out + (size_t)a * s * slice_elems;
  const int L = n >> 1, c = n & 1;
  const int ldM = N_L;
  const double2* Ma = M + (size_t)a * N_L * (parts * N_L);
  __shared__ double red[4];
  __shared__ int s_E;
  double m = 0.0;
  if (L < N_L)
    for (int k = threadIdx.x; k < parts * N_L; k += blockDim.x) {
      const double2 v = Ma[L + (size_t)k * ldM];
      m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
    }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double mm = fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
    s_E = slice_exponent(mm);
    expo[(size_t)a * n_pad + n] = s_E;
  }
  __syncthreads();
  const int E = s_E;
  const int hp = P / 2;
  const int oc = ((2 * a * N_L) & (KB - 1)) >> 1;  // complex offset of atom a in its K block
  for (int j = threadIdx.x; j < Kop / 2; j += blockDim.x) {
    const int part = j / hp, l = j - part * hp - oc;
    const bool zero = (L >= N_L) || (l < 0) || (l >= N_L);
    double2 v = make_double2(0.0, 0.0);
    if (!zero) {
      const double2 mv = Ma[L + (size_t)(part * N_L + l) * ldM];
      v = c == 0 ? make_double2(mv.x, -mv.y) : make_double2(mv.y, mv.x);
    }
    put_slices(v, zero, E, s, base, false, slice_elems, 0, tile_off(n, j, Kop / KB));
  }
}

// Real sources (real-symmetric variant): nblk * N_L real rows per column, packed one
// K position per row (kpad = roundup(K, 16)); a thread writes the pair of positions
// (2j, 2j + 1) as one 32-bit word per slice, with k_slice's digit and exponent rules
// (no rotated copy: a real contraction needs none).
__global__ void __launch_bounds__(256) k_slice_real(const __grid_constant__ SliceParams P) {
  const SliceJob J = P.job[blockIdx.y];
  const int g = P.g0 + blockIdx.x;
  const int s = P.s;
  const int K = J.nblk * P.N_L;                // real rows of the source
  const int kpad = ((K + KB - 1) / KB) * KB;   // packed K, whole 16-wide blocks
  const size_t slice_elems = (size_t)P.rows_pad * kpad;
  __shared__ unsigned long long red[32];
  __shared__ int s_E;
  const int kc = kpad / 2;  // position pairs per row
  const int NKB = kpad / KB;
  if (g >= P.N_G) {
    for (int k = threadIdx.x; k < kc; k += blockDim.x)
      for (int p = 0; p < s; ++p)
        *(uint32_t*)(J.plain + p * slice_elems + tile_off(g, k, NKB)) = 0u;
    if (threadIdx.x == 0) J.expo[g] = 0;
    return;
  }
  const double* col = (const double*)J.X + (size_t)g * J.ldX;
  unsigned long long m = 0ull;  // bit pattern of the column's largest finite |value| (x |u|)
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double v = col[k];
    m = max(m, finite_abs_bits(J.u ? v * J.u[k] : v));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long mm = 0ull;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = max(mm, red[i]);
    s_E = slice_exponent(__longlong_as_double((long long)mm));
    J.expo[g] = s_E;
  }
  __syncthreads();
  const int E = s_E;
  for (int j = threadIdx.x; j < kc; j += blockDim.x) {
    const int k0 = 2 * j, k1 = k0 + 1;
    double x0 = k0 < K ? col[k0] : 0.0, x1 = k1 < K ? col[k1] : 0.0;
    if (J.u) {
      if (k0 < K) x0 *= J.u[k0];
      if (k1 < K) x1 *= J.u[k1];
    }
    put_slices(make_double2(x0, x1), k0 >= K, E, s, J.plain, false, slice_elems, 0,
               tile_off(g, j, NKB));
  }
}

// Real per-atom operators: the real parts of the (embedded) MZ[a] and M2[a]; operator
// row n = output row L; column l of a part at real position (a N_L) mod 16 + l of the
// part, zeros elsewhere (the packed real layout's offset of atom a).
__global__ void __launch_bounds__(128) k_slice_op_real(const double2* __restrict__ M, int job,
                                                       int N_A, int N_L, int P, int n_pad, int s,
                                                       uint16_t* __restrict__ out,
                                                       int* __restrict__ expo) {
  const int a = blockIdx.y, L = blockIdx.x;  // L < n_pad
  const int parts = job == 0 ? 2 : 1;
  const int Kop = parts * P;
  const size_t slice_elems = (size_t)n_pad * Kop;
  uint16_t* base = out + (size_t)a * s * slice_elems;
  const int ldM = N_L;
  const double2* Ma = M + (size_t)a * N_L * (parts * N_L);
  __shared__ unsigned long long red[4];
  __shared__ int s_E;
  unsigned long long m = 0ull;
  if (L < N_L)
    for (int k = threadIdx.x; k < parts * N_L; k += blockDim.x)
      m = max(m, finite_abs_bits(Ma[L + (size_t)k * ldM].x));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long mm = max(max(red[0], red[1]), max(red[2], red[3]));
    s_E = slice_exponent(__longlong_as_double((long long)mm));
    expo[(size_t)a * n_pad + L] = s_E;
  }
  __syncthreads();
  const int E = s_E;
  const int oa = (a * N_L) & (KB - 1);  // atom a's offset inside its first K block
  for (int j = threadIdx.x; j < Kop / 2; j += blockDim.x) {
    double x[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = 2 * j + h;
      const int part = q / P, l = q - part * P - oa;
      x[h] = (L < N_L && l >= 0 && l < N_L) ? Ma[L + (size_t)(part * N_L + l) * ldM].x : 0.0;
    }
    put_slices(make_double2(x[0], x[1]), L >= N_L, E, s, base, false, slice_elems, 0,
               tile_off(L, j, Kop / KB));
  }
}

// ------------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000)p;
    cudaGetLastError();
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

// Tensor map over a blocked slice array: dims (16 elements, 64 rows, NKB K blocks,
// NRB row blocks, planes `plane_tiles` tiles of 2 KB apart), box (16, 64, 1, box_rb,
// box_planes): every (row block, plane) of a box is one contiguous 2 KB tile, so a box
// lands in shared memory as [plane][row block] 2 KB tiles.
bool encode_tiles(CUtensorMap* m, const uint16_t* base, int NKB, int NRB, int planes,
                  size_t plane_tiles, int box_rb, int box_planes) {
  auto fn = get_encode();
  if (!fn) return false;
  if (box_rb < 1 || box_rb > NRB || box_planes < 1 || box_planes > planes) return false;
  cuuint64_t dims[5] = {(cuuint64_t)KB, 64u, (cuuint64_t)NKB, (cuuint64_t)NRB, (cuuint64_t)planes};
  cuuint64_t strides[4] = {(cuuint64_t)KB * 2, (cuuint64_t)TILE_BYTES,
                           (cuuint64_t)NKB * TILE_BYTES, (cuuint64_t)plane_tiles * TILE_BYTES};
  cuuint32_t box[5] = {(cuuint32_t)KB, 64u, 1u, (cuuint32_t)box_rb, (cuuint32_t)box_planes};
  cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Maps over the slices of one operand source with NKB K blocks and NRB 64-row blocks.
// A source with a rotated copy stores plain and rotated slices interleaved by plane
// (plane 2p: slice p of (re, im) pairs, plane 2p + 1: slice p of (im, -re) pairs).
//  * left role: the s plain slices of two row blocks (128 rows) per box;
//  * right role, complex: the plain and rotated slices of one row block (64 columns)
//    per box (2 s planes); right role, real: as the left role (128 columns).
bool encode_left(CUtensorMap* m, const uint16_t* base, int NKB, int NRB, int s, bool rot) {
  const size_t plane = (size_t)NRB * NKB * (rot ? 2 : 1);
  return encode_tiles(m, base, NKB, NRB, s, plane, 2, s);
}
bool encode_right(CUtensorMap* m, const uint16_t* base, int NKB, int NRB, int s, bool rot) {
  if (!rot) return encode_left(m, base, NKB, NRB, s, false);
  return encode_tiles(m, base, NKB, NRB, 2 * s, (size_t)NRB * NKB, 1, 2 * s);
}

}  // namespace

// Rows (operand columns g) of a slice array: whole 128-row blocks; 256 for real plans,
// whose contraction column pairs span 256 columns.
static inline int rows_pad_of(int N_G, bool real = false) {
  const int al = real ? 2 * ROWS_ALIGN : ROWS_ALIGN;
  return ((N_G + al - 1) / al) * al;
}
// Packed real K of a source of nblk blocks of N_L rows (whole 16-wide blocks): two
// positions per complex row, one per real row.
static inline int kpad_of(int nblk, int N_L, bool real = false) {
  return (((real ? 1 : 2) * nblk * N_L + KB - 1) / KB) * KB;
}
// Real K of one part of a per-atom operator: the most 16-wide K blocks any atom's
// rows [pr a N_L, pr (a+1) N_L) of the packed layout touch (pr positions per row).
static int op_part_k(int N_A, int N_L, bool real = false) {
  const int pr = real ? 1 : 2;
  int nkb = 0;
  for (int a = 0; a < N_A; ++a)
    nkb = std::max(nkb, (pr * (a + 1) * N_L + KB - 1) / KB - (pr * a * N_L) / KB);
  return nkb * KB;
}
// Operator rows (2 N_L real rows; N_L for real plans) padded to whole 128-row tiles.
static inline int op_rows_pad(int N_L, bool real = false) {
  return (((real ? 1 : 2) * N_L + BN - 1) / BN) * BN;
}

// Blocks (of N_L complex rows) of each source and whether it needs the rotated copy.
static void source_shape(int src, int N_A, int n_fail, bool real, int& nblk, bool& rot) {
  rot = !real && (src != SRC_AF);
  nblk = (src == SRC_AF || src == SRC_X) ? n_fail : N_A;
}

size_t hs_plan_s::split_ws_bytes(int N_G, int n_fail) const {
  if (precision != HS_SPLIT_BF16) return 0;
  const int nf = n_fail > 0 ? n_fail : 1;
  const int rp = rows_pad_of(N_G, real);
  size_t b = 0;
  for (int src = 0; src < NSRC; ++src) {
    int nblk;
    bool rot;
    source_shape(src, N_A, nf, real, nblk, rot);
    const size_t one = (size_t)slices * rp * kpad_of(nblk, N_L, real) * 2;
    b += (rot ? 2 : 1) * one + sizeof(int) * rp;
  }
  return b;
}

int hs_plan_s::split_ws_alloc(Workspace& w, int N_G, int n_fail, cudaStream_t st, bool async) {
  if (precision != HS_SPLIT_BF16) return HS_OK;
  if (!get_encode()) return HS_ECUDA;
  const int rp = rows_pad_of(N_G, real);
  auto al = [&](void** ptr, size_t bytes) -> bool {
    return (async ? hs_malloc_async(ptr, bytes, st, hs_serve_pool(this)) : cudaMalloc(ptr, bytes)) ==
           cudaSuccess;
  };
  for (int src = 0; src < NSRC; ++src) {
    int nblk;
    bool rot;
    source_shape(src, N_A, n_fail, real, nblk, rot);
    const size_t one = (size_t)slices * rp * kpad_of(nblk, N_L, real) * 2;
    if (!al((void**)&w.sb[src].plain, (rot ? 2 : 1) * one)) return HS_ENOMEM;
    w.sb[src].rot = rot;
    if (!al((void**)&w.sb[src].expo, sizeof(int) * rp)) return HS_ENOMEM;
  }
  return HS_OK;
}

size_t hs_plan_s::split_fixed_bytes() const {
  if (precision != HS_SPLIT_BF16) return 0;
  const size_t P = (size_t)op_part_k(N_A, N_L, real), np = (size_t)op_rows_pad(N_L, real);
  return (size_t)N_A * slices * np * (3 * P) * 2 + 2 * sizeof(int) * N_A * np;
}

int hs_plan_s::split_plan_alloc() {
  if (precision != HS_SPLIT_BF16) return HS_OK;
  if (!get_encode()) return HS_ECUDA;
  const size_t P = (size_t)op_part_k(N_A, N_L, real), np = (size_t)op_rows_pad(N_L, real);
  const size_t zb = (size_t)N_A * slices * np * 2 * P * 2, wb = zb / 2;
  if (cudaMalloc((void**)&op_slices[0], zb) != cudaSuccess ||
      cudaMalloc((void**)&op_slices[1], wb) != cudaSuccess ||
      cudaMalloc((void**)&op_expo[0], sizeof(int) * N_A * np) != cudaSuccess ||
      cudaMalloc((void**)&op_expo[1], sizeof(int) * N_A * np) != cudaSuccess) {
    cudaGetLastError();
    return HS_ENOMEM;
  }
  return HS_OK;
}

void hs_plan_s::split_plan_release() {
  for (int j = 0; j < 2; ++j) {
    if (op_slices[j]) cudaFree(op_slices[j]);
    if (op_expo[j]) cudaFree(op_expo[j]);
    op_slices[j] = nullptr;
    op_expo[j] = nullptr;
  }
}

// Slice MZ and M2 (k-independent) after every factorisation.
int hs_plan_s::split_factor(cudaStream_t st) {
  if (precision != HS_SPLIT_BF16) return HS_OK;
  const int P = op_part_k(N_A, N_L, real), np = op_rows_pad(N_L, real);
  for (int job = 0; job < 2; ++job) {
    const double2* M = job == 0 ? MZ : M2;
    if (real)
      k_slice_op_real<<<dim3(np, N_A), 128, 0, st>>>(M, job, N_A, N_L, P, np, slices,
                                                      op_slices[job], op_expo[job]);
    else
      k_slice_op<<<dim3(np, N_A), 128, 0, st>>>(M, job, N_A, N_L, P, np, slices, op_slices[job],
                                                 op_expo[job]);
    HS_CUDA_TRY(cudaGetLastError());
  }
  return HS_OK;
}

static int set_smem(const void* fn, size_t smem) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                 cudaSuccess
             ? HS_OK
             : HS_ECUDA;
}

template <int MODE, int S>
static int launch_one(int grid, size_t smem, cudaStream_t st, const SplitParams& P) {
  int rc = set_smem((const void*)k_split_gemm<MODE, S>, smem);
  if (rc) return rc;
  k_split_gemm<MODE, S><<<grid, NUM_THREADS, smem, st>>>(P);
  return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ECUDA;
}

template <int MODE>
static int launch_mode(int s, int grid, size_t smem, cudaStream_t st, const SplitParams& P) {
  switch (s) {
    case 2: return launch_one<MODE, 2>(grid, smem, st, P);
    case 3: return launch_one<MODE, 3>(grid, smem, st, P);
    case 4: return launch_one<MODE, 4>(grid, smem, st, P);
    case 5: return launch_one<MODE, 5>(grid, smem, st, P);
    case 6: return launch_one<MODE, 6>(grid, smem, st, P);
    case 7: return launch_one<MODE, 7>(grid, smem, st, P);
    default: return HS_EINVAL;
  }
}

// Test-only stall injection (HS_TEST_STALL=1): every slice-GEMM launch arms no stage and
// issues no copy, so its bounded waits give up (2 s) and the kernel sets the device error
// word and returns (the host sees HS_EDEVICE).  Read at every launch.
static bool stall_injection() {
  const char* e = std::getenv("HS_TEST_STALL");
  return e && e[0] == '1';
}

// The launch parameters as they go to the device: the stall flag.
static void set_waits(SplitParams& P) { P.stall = stall_injection() ? 1 : 0; }

static int launch_gemm(int mode, int s, int grid, size_t smem, cudaStream_t st,
                       const SplitParams& P0) {
  SplitParams P = P0;
  set_waits(P);
  switch (mode) {
    case MODE_CONTRACT: return launch_mode<MODE_CONTRACT>(s, grid, smem, st, P);
    case MODE_ATOMS: return launch_mode<MODE_ATOMS>(s, grid, smem, st, P);
    case MODE_CONTRACT_R: return launch_mode<MODE_CONTRACT_R>(s, grid, smem, st, P);
    case MODE_ATOMS_R: return launch_mode<MODE_ATOMS_R>(s, grid, smem, st, P);
    default: return HS_EINVAL;
  }
}

template <int MODE>
static const void* atoms_fn_m(int s) {
  switch (s) {
    case 2: return (const void*)k_split_gemm<MODE, 2>;
    case 3: return (const void*)k_split_gemm<MODE, 3>;
    case 4: return (const void*)k_split_gemm<MODE, 4>;
    case 5: return (const void*)k_split_gemm<MODE, 5>;
    case 6: return (const void*)k_split_gemm<MODE, 6>;
    case 7: return (const void*)k_split_gemm<MODE, 7>;
    default: return nullptr;
  }
}
static const void* atoms_fn(int s) { return atoms_fn_m<MODE_ATOMS>(s); }

// The grouped per-atom launch as the single kernel node of a CUDA graph:
// captured once per plan, then re-parameterised (cudaGraphExecKernelNodeSetParams:
// grid and arguments of this batch) and replayed for every batch.  Updates only
// affect later launches, so a replay still running is undisturbed.
struct AtomsGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t node = nullptr;
};

AtomsGraph* hs_atoms_graph_new() { return new (std::nothrow) AtomsGraph(); }
void hs_atoms_graph_free(AtomsGraph* a) {
  if (!a) return;
  if (a->exec) cudaGraphExecDestroy(a->exec);
  if (a->g) cudaGraphDestroy(a->g);
  delete a;
}

static int graph_launch_atoms(AtomsGraph& G, int s, int grid, size_t smem, cudaStream_t st,
                              const SplitParams& P0) {
  SplitParams P = P0;
  set_waits(P);
  const void* fn = atoms_fn(s);
  if (!fn) return HS_EINVAL;
  int rc = set_smem(fn, smem);
  if (rc) return rc;
  void* args[1] = {(void*)&P};
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.func = (void*)fn;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(NUM_THREADS);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = args;
  if (!G.exec) {
    HS_CUDA_TRY(cudaGraphCreate(&G.g, 0));
    HS_CUDA_TRY(cudaGraphAddKernelNode(&G.node, G.g, nullptr, 0, &kp));
    HS_CUDA_TRY(cudaGraphInstantiate(&G.exec, G.g, 0));
  } else {
    HS_CUDA_TRY(cudaGraphExecKernelNodeSetParams(G.exec, G.node, &kp));
  }
  HS_CUDA_TRY(cudaGraphLaunch(G.exec, st));
  return HS_OK;
}

// ---------------------------------------------------------------- autotuner
// Launch knobs tuned on the real work: the first synchronous assembly with an untuned
// key times every candidate value (the trial launches compute the same result as the
// final one) and keeps the fastest; a candidate other than the first must win by 2 %.
//  * ring depth (TMA pipeline stages) of each kernel mode, key "mode:s:N_L:bucket";
//  * the contraction's band width (row blocks per band of its tile order, which sets
//    how compact the block of tiles resident at one time is and so the L2 reuse of
//    the slice boxes), key "band:mode:s:N_L:bucket", candidates 8, 4, 16, 32;
//  * the slicer's block size (threads per operand column), key
//    "slice:real:s:N_L:bucket", candidates 256, 128.
// bucket = N_G / 1024 rounded up.  Serving requests use tuned values when there are
// some and the defaults otherwise.  HS_AUTOTUNE=0 disables tuning; HS_TUNE_CACHE=<file>
// loads (whenever the name changes) and appends "key value" lines.  The per-atom kernel's grid is not a knob: its
// ring fills an SM's shared memory, so it runs one CTA per SM by construction.
namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
std::string g_tune_path;  // the HS_TUNE_CACHE file read last ("" = none yet)

std::string tune_key(int mode, int s, int N_L, int N_G) {
  return std::to_string(mode) + ":" + std::to_string(s) + ":" + std::to_string(N_L) + ":" +
         std::to_string((N_G + 1023) / 1024);
}

// Reads the cache file named by HS_TUNE_CACHE whenever that name changes (its values
// override the ones in memory).
void tune_load_locked() {
  const char* path = std::getenv("HS_TUNE_CACHE");
  if (!path || g_tune_path == path) return;
  g_tune_path = path;
  std::FILE* f = std::fopen(path, "r");
  if (!f) return;
  char key[128];
  int v;
  while (std::fscanf(f, "%127s %d", key, &v) == 2) g_tune[key] = v;
  std::fclose(f);
}

void tune_store_locked(const std::string& key, int v) {
  g_tune[key] = v;
  const char* path = std::getenv("HS_TUNE_CACHE");
  if (!path) return;
  std::FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d\n", key.c_str(), v);
  std::fclose(f);
}

size_t smem_for(int mode, int n_stage, int stage_bytes) {
  const size_t ring = (size_t)n_stage * stage_bytes;
  return (is_contract(mode) ? std::max(ring, (size_t)STAGING_CONTRACT) : ring) + 1024 + 256;
}

// The cached value of `key` if any; else, when tuning is allowed, the fastest of
// `cand` (cand[0] is the default) timed with `trial(value)`, which enqueues the real
// work; else cand[0].  `found` tells whether the value came from the cache.
int tuned_choice(const std::string& key, const std::vector<int>& cand, bool allow,
                 cudaStream_t st, const std::function<int(int)>& trial, bool* found = nullptr) {
  if (found) *found = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      if (found) *found = true;
      return it->second;
    }
  }
  const char* env = std::getenv("HS_AUTOTUNE");
  if (!allow || cand.size() < 2 || (env && env[0] == '0') || stall_injection()) return cand[0];
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cand[0];
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cand[0];
  }
  int best = cand[0];
  float best_ms = 1e30f;
  for (int v : cand) {
    float ms = 0.f;
    if (cudaEventRecord(e0, st) != cudaSuccess || trial(v) != HS_OK ||
        cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    if (ms < 0.98f * best_ms) {  // a later candidate must win clearly
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_store_locked(key, best);
  return best;
}

// Depth for this launch; `trial(depth)` enqueues the real work with that depth.
int tuned_depth(int mode, int s, int N_L, int N_G, int max_depth, bool allow, cudaStream_t st,
                const std::function<int(int)>& trial) {
  std::vector<int> cand;
  for (int d = max_depth; d >= 2; --d) cand.push_back(d);
  const int v = tuned_choice(tune_key(mode, s, N_L, N_G), cand, allow, st, trial);
  return std::min(std::max(v, 2), max_depth);
}
}  // namespace

// Row blocks per band of the contraction's tile order: tuned per key (8 by default:
// 152 resident CTAs then span about 8 row blocks x 19 column blocks); HS_BAND > 0 fixes it.
static int band_override() {
  static const int band = []() {
    const char* e = std::getenv("HS_BAND");
    const int v = e ? std::atoi(e) : 0;
    return v >= 1 ? v : 0;
  }();
  return band;
}
static int contract_band(int mode = 0, int s = 0, int N_L = 0, int N_G = 0) {
  if (band_override()) return band_override();
  if (s == 0) return 8;
  bool found = false;
  const int v = tuned_choice("band:" + tune_key(mode, s, N_L, N_G), {8}, false, nullptr,
                             [](int) { return HS_OK; }, &found);
  return found && v >= 1 ? v : 8;
}
static int tuned_band(int mode, int s, int N_L, int N_G, bool allow, cudaStream_t st,
                      const std::function<int(int)>& trial) {
  if (band_override()) return band_override();
  const int v = tuned_choice("band:" + tune_key(mode, s, N_L, N_G), {8, 4, 16, 32}, allow, st,
                             trial);
  return v >= 1 ? v : 8;
}

// Threads per slicer block (one block per operand column).
static int slice_threads(bool real, int s, int N_L, int N_G, bool allow, cudaStream_t st,
                         const std::function<int(int)>& trial) {
  const int v = tuned_choice("slice:" + std::to_string(real ? 1 : 0) + ":" + std::to_string(s) +
                                 ":" + std::to_string(N_L) + ":" +
                                 std::to_string((N_G + 1023) / 1024),
                             {256, 128}, allow, st, trial);
  return v == 128 ? v : 256;
}

int hs_plan_s::split_geometry(int& n_stage, size_t& smem) const {
  const int stage_bytes = 4 * slices * TILE_BYTES;
  const int budget = 227 * 1024 - 1024 - 256;
  n_stage = budget / stage_bytes;
  if (n_stage > 8) n_stage = 8;
  if (n_stage < 2) return HS_EINVAL;
  smem = smem_for(MODE_CONTRACT, n_stage, stage_bytes);
  return HS_OK;
}

static void slice_job(SliceParams& sp, int& nj, Workspace& w, int src, const double2* X, int ldX,
                      int nblk, const double* u) {
  SliceBuf& b = w.sb[src];
  sp.job[nj++] = SliceJob{X, u, b.plain, b.rot, b.expo, ldX, nblk};
}

static int slice_launch(SliceParams& sp, int nj, int s, int N_G, int rp, int N_L, bool real,
                        cudaStream_t st, int g0 = 0, int ng = -1, int threads = 256) {
  if (ng < 0) ng = rp - g0;
  if (g0 < 0 || ng < 0 || g0 + ng > rp) return HS_EINVAL;
  if (ng == 0) return HS_OK;  // nothing left to slice
  if (threads != 128 && threads != 256) return HS_EINVAL;
  sp.g0 = g0;
  sp.s = s;
  sp.N_G = N_G;
  sp.rows_pad = rp;
  sp.N_L = N_L;
  if (real) k_slice_real<<<dim3(ng, nj), threads, 0, st>>>(sp);
  else k_slice<<<dim3(ng, nj), threads, 0, st>>>(sp);
  return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ECUDA;
}

// 1. slice the inputs A, U.B, B of one k-point (tune: time the slicer's block sizes on
//    this work if its key is untuned)
int hs_plan_s::split_inputs(const double2* A, const double2* B, int ldAB, const double* U,
                            int N_G, Workspace& w, cudaStream_t st, int g0, int ng, bool tune) {
  const int rp = rows_pad_of(N_G, real);
  if (rows_pad_of(w.N_G, real) < rp || w.n_fail < N_f || !w.sb[SRC_A].plain) return HS_EINVAL;
  SliceParams sp{};
  int nj = 0;
  slice_job(sp, nj, w, SRC_A, A, ldAB, N_A, nullptr);
  slice_job(sp, nj, w, SRC_UB, B, ldAB, N_A, U);
  slice_job(sp, nj, w, SRC_B, B, ldAB, N_A, nullptr);
  const int threads = slice_threads(real, slices, N_L, N_G, tune && g0 == 0 && ng < 0, st,
                                    [&](int t) {
                                      return slice_launch(sp, nj, slices, N_G, rp, N_L, real, st,
                                                          g0, ng, t);
                                    });
  return slice_launch(sp, nj, slices, N_G, rp, N_L, real, st, g0, ng, threads);
}

// 2. per-atom products of up to kMaxBatch k-points in one grouped launch: Z and
//    W2 = [Y; X] in FP64.  With `graph`, the launch is the (re-parameterised) kernel
//    node of the plan's captured graph.
int hs_plan_s::split_atoms(const AtomsJob* jobs, int n, cudaStream_t st, AtomsGraph* graph) {
  if (n < 1 || n > kMaxBatch) return HS_EINVAL;
  const int s = slices, Pp = op_part_k(N_A, N_L, real), np = op_rows_pad(N_L, real);
  const int mode = real ? MODE_ATOMS_R : MODE_ATOMS;
  int n_stage;
  size_t smem;
  int rc = split_geometry(n_stage, smem);
  if (rc) return rc;
  SplitParams* PA = new (std::nothrow) SplitParams;
  if (!PA) return HS_ENOMEM;
  std::memset(PA, 0, sizeof(*PA));
  AtomsArgs& at = PA->at;
  // operator slices [a][p][n_pad][Kop]: the right operand, two row blocks x s planes
  bool ok = encode_tiles(&PA->maps[0], op_slices[0], 2 * Pp / KB, np / 64, N_A * s,
                         (size_t)(np / 64) * (2 * Pp / KB), 2, s) &&
            encode_tiles(&PA->maps[1], op_slices[1], Pp / KB, np / 64, N_A * s,
                         (size_t)(np / 64) * (Pp / KB), 2, s);
  at.mOp[0] = 0;
  at.mOp[1] = 1;
  int grid = 0;
  for (int r = 0; r < n && ok; ++r) {
    Workspace& w = *jobs[r].w;
    const int rp = rows_pad_of(jobs[r].N_G, real);
    AtomsReq& R = at.rq[r];
    R.mA = 2 + 2 * r;
    R.mB = 3 + 2 * r;
    const int nkb = kpad_of(N_A, N_L, real) / KB;
    ok = encode_left(&PA->maps[R.mA], w.sb[SRC_A].plain, nkb, rp / 64, s, w.sb[SRC_A].rot) &&
         encode_left(&PA->maps[R.mB], w.sb[SRC_B].plain, nkb, rp / 64, s, w.sb[SRC_B].rot);
    R.eA = w.sb[SRC_A].expo;
    R.eB = w.sb[SRC_B].expo;
    R.Z = w.Z;
    R.W2 = w.W2;
    R.N_G = jobs[r].N_G;
    R.ngblk = rp / BM;
    R.tile0 = grid;
    grid += R.ngblk * (np / BN) * 2 * N_A;
  }
  if (!ok) {
    delete PA;
    return HS_ECUDA;
  }
  at.nreq = n;
  // persistent: one CTA per SM, each running every gridDim.x-th tile
  PA->ntiles = grid;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
      delete PA;
      return HS_ECUDA;
    }
    grid = std::min(grid, nsm);
  }
  at.eOp[0] = op_expo[0];
  at.eOp[1] = op_expo[1];
  at.slot = slot_d;
  at.ld = N_A * N_L;
  at.N_A = N_A;
  at.N_L = N_L;
  at.P = Pp;
  at.n_pad = np;
  at.ntile = np / BN;
  PA->s = s;
  PA->err = err_d;
  const int stage_bytes = 4 * s * TILE_BYTES;
  const int depth = tuned_depth(mode, s, N_L, jobs[0].N_G, n_stage, graph == nullptr, st,
                                [&](int d) {
                                  PA->n_stage = d;
                                  return launch_gemm(mode, s, grid, smem_for(mode, d, stage_bytes),
                                                     st, *PA);
                                });
  PA->n_stage = depth;
  smem = smem_for(mode, depth, stage_bytes);
  rc = graph ? graph_launch_atoms(*graph, s, grid, smem, st, *PA)
             : launch_gemm(mode, s, grid, smem, st, *PA);
  delete PA;
  return rc;
}

// 3. gather A_f, slice the per-atom outputs, and the two stacked contractions
int hs_plan_s::split_outputs(const double2* A, int ldAB, int N_G, double2* H, double2* S,
                             Workspace& w, cudaStream_t st, bool timed, cudaEvent_t s_done,
                             bool skip_S, bool mirror) {
  const int K = N_A * N_L;
  const int N_h = N_A - N_f;
  const int s = slices;
  const int rp = rows_pad_of(N_G, real);
  const int mode = real ? MODE_CONTRACT_R : MODE_CONTRACT;
  int n_stage;
  size_t smem;
  int rc = split_geometry(n_stage, smem);
  if (rc) return rc;
  if (real)
    HS_CUDA_TRY(hs_launch_gather_af_real((const double*)A, ldAB, fail_list_d, N_f, N_L, N_G,
                                         (double*)w.AF, st));
  else
    HS_CUDA_TRY(hs_launch_gather_af(A, ldAB, fail_list_d, N_f, N_L, N_G, w.AF, st));
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[4], st));
  {
    SliceParams sp{};
    int nj = 0;
    slice_job(sp, nj, w, SRC_Z, w.Z, K, N_A, nullptr);
    if (N_h > 0) slice_job(sp, nj, w, SRC_Y, w.W2, K, N_h, nullptr);
    if (N_f > 0) {
      slice_job(sp, nj, w, SRC_AF, w.AF, N_f * N_L, N_f, nullptr);
      const double2* X = real ? (const double2*)((const double*)w.W2 + (size_t)N_h * N_L)
                              : w.W2 + (size_t)N_h * N_L;
      slice_job(sp, nj, w, SRC_X, X, K, N_f, nullptr);
    }
    const int threads = slice_threads(real, s, N_L, N_G, false, st, [](int) { return HS_OK; });
    rc = slice_launch(sp, nj, s, N_G, rp, N_L, real, st, 0, -1, threads);
    if (rc) return rc;
  }
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[5], st));

  SplitParams* PP = new (std::nothrow) SplitParams;
  if (!PP) return HS_ENOMEM;
  SplitParams& P = *PP;
  std::memset(&P, 0, sizeof(P));
  int map_of[NSRC][2];
  int nm = 0;
  auto add_map = [&](int src, int nblk) -> bool {  // [0]: left role, [1]: right role
    SliceBuf& b = w.sb[src];
    const int nkb = kpad_of(nblk, N_L, real) / KB;
    map_of[src][0] = nm;
    if (!encode_left(&P.maps[nm++], b.plain, nkb, rp / 64, s, b.rot)) return false;
    map_of[src][1] = nm;
    return encode_right(&P.maps[nm++], b.plain, nkb, rp / 64, s, b.rot);
  };
  bool ok = add_map(SRC_A, N_A) && add_map(SRC_UB, N_A) && add_map(SRC_Z, N_A) &&
            add_map(SRC_B, N_A);
  if (N_h > 0) ok = ok && add_map(SRC_Y, N_h);
  if (N_f > 0) ok = ok && add_map(SRC_AF, N_f) && add_map(SRC_X, N_f);
  if (!ok) {
    delete PP;
    return HS_ECUDA;
  }
  P.s = s;
  P.n_stage = n_stage;
  P.N_G = N_G;
  P.ldC = N_G;
  P.nbj = (N_G + (real ? BN : BNC) - 1) / (real ? BN : BNC);  // output column tiles
  P.rows_pad = rp;
  P.err = err_d;
  const int nbi = (N_G + BM - 1) / BM;
  int tiles = 0;
  for (int b = 0; b < nbi; ++b)  // CTA pairs: column pair c from row block c (2c if real)
    tiles += 2 * std::min((real ? b / 2 : b) + 1, (P.nbj + 1) / 2);
  P.nbi = nbi;
  P.band = contract_band(mode, s, N_L, N_G);
  P.ntiles = tiles;  // one tile per CTA
  auto seg = [&](int srcL, int srcR, int nblk) {
    SplitSeg g;
    g.mL = map_of[srcL][0];
    g.mR = map_of[srcR][1];
    g.kblocks = kpad_of(nblk, N_L, real) / KB;
    g.eL = w.sb[srcL].expo;
    g.eR = w.sb[srcR].expo;
    return g;
  };
  // S = A^H A + (UB)^H (UB)
  P.nseg = 2;
  P.seg[0] = seg(SRC_A, SRC_A, N_A);
  P.seg[1] = seg(SRC_UB, SRC_UB, N_A);
  P.C = S;
  {
    const int stage_bytes = 4 * s * TILE_BYTES;
    // trials re-run the S contraction: not when the caller already made S (its mirror
    // may be running on another stream)
    const bool tune = timed && !skip_S;
    const int depth = tuned_depth(mode, s, N_L, N_G, n_stage, tune, st, [&](int d) {
      P.n_stage = d;
      return launch_gemm(mode, s, tiles, smem_for(mode, d, stage_bytes), st, P);
    });
    P.n_stage = depth;
    smem = smem_for(mode, depth, stage_bytes);
    P.band = tuned_band(mode, s, N_L, N_G, tune, st, [&](int b) {
      P.band = b;
      return launch_gemm(mode, s, tiles, smem, st, P);
    });
  }
  if (!skip_S) rc = launch_gemm(mode, s, tiles, smem, st, P);
  if (rc == HS_OK && !skip_S && mirror) {  // S is final once mirrored: it can leave while H runs
    const cudaError_t e = real ? hs_launch_mirror_real((double*)S, N_G, N_G, st)
                               : hs_launch_mirror(S, N_G, N_G, st);
    if (e != cudaSuccess || (s_done && cudaEventRecord(s_done, st) != cudaSuccess)) rc = HS_ECUDA;
  }
  if (rc == HS_OK && timed && cudaEventRecord(ev[6], st) != cudaSuccess) rc = HS_ECUDA;
  if (rc == HS_OK) {
    // H = Z^H B + B^H Z + Y^H Y + A_f^H X_f
    int n = 0;
    P.seg[n++] = seg(SRC_Z, SRC_B, N_A);
    P.seg[n++] = seg(SRC_B, SRC_Z, N_A);
    if (N_h > 0) P.seg[n++] = seg(SRC_Y, SRC_Y, N_h);
    if (N_f > 0) P.seg[n++] = seg(SRC_AF, SRC_X, N_f);
    P.nseg = n;
    P.C = H;
    rc = launch_gemm(mode, s, tiles, smem, st, P);
    if (rc == HS_OK && timed && cudaEventRecord(ev[7], st) != cudaSuccess) rc = HS_ECUDA;
  }
  delete PP;
  return rc;
}

// The S contraction restricted to the lower-triangle tiles of row blocks [bi0, bi1):
// they read only A and U.B slice rows below 128 * bi1, so a caller that slices column
// chunks as they arrive can run them before the later chunks exist.
int hs_plan_s::split_contract_S_rows(int N_G, double2* S, Workspace& w, cudaStream_t st, int bi0,
                                     int bi1) {
  const int s = slices;
  const int rp = rows_pad_of(N_G, real);
  const int mode = real ? MODE_CONTRACT_R : MODE_CONTRACT;
  const int nbi = (N_G + BM - 1) / BM;
  bi0 = std::max(bi0, 0);
  bi1 = std::min(bi1, nbi);
  if (bi1 <= bi0) return HS_OK;
  int n_stage;
  size_t smem;
  int rc = split_geometry(n_stage, smem);
  if (rc) return rc;
  SplitParams* PP = new (std::nothrow) SplitParams;
  if (!PP) return HS_ENOMEM;
  SplitParams& P = *PP;
  std::memset(&P, 0, sizeof(P));
  int map_of[2][2];
  int nm = 0;
  bool ok = true;
  for (int i = 0; i < 2 && ok; ++i) {
    SliceBuf& b = w.sb[i == 0 ? SRC_A : SRC_UB];
    const int nkb = kpad_of(N_A, N_L, real) / KB;
    map_of[i][0] = nm;
    ok = encode_left(&P.maps[nm++], b.plain, nkb, rp / 64, s, b.rot);
    map_of[i][1] = nm;
    ok = ok && encode_right(&P.maps[nm++], b.plain, nkb, rp / 64, s, b.rot);
  }
  if (!ok) {
    delete PP;
    return HS_ECUDA;
  }
  P.s = s;
  P.N_G = N_G;
  P.ldC = N_G;
  P.nbj = (N_G + (real ? BN : BNC) - 1) / (real ? BN : BNC);
  P.rows_pad = rp;
  P.err = err_d;
  int tiles = 0;
  for (int b = bi0; b < bi1; ++b) tiles += 2 * std::min((real ? b / 2 : b) + 1, (P.nbj + 1) / 2);
  P.bi0 = bi0;
  P.nbi = bi1;
  P.band = contract_band(mode, s, N_L, N_G);
  P.ntiles = tiles;
  for (int i = 0; i < 2; ++i) {
    SplitSeg& g = P.seg[i];
    g.mL = map_of[i][0];
    g.mR = map_of[i][1];
    g.kblocks = kpad_of(N_A, N_L, real) / KB;
    g.eL = g.eR = w.sb[i == 0 ? SRC_A : SRC_UB].expo;
  }
  P.nseg = 2;
  P.C = S;
  const int stage_bytes = 4 * s * TILE_BYTES;
  P.n_stage = tuned_depth(mode, s, N_L, N_G, n_stage, false, st, [](int) { return HS_OK; });
  rc = launch_gemm(mode, s, tiles, smem_for(mode, P.n_stage, stage_bytes), st, P);
  delete PP;
  return rc;
}

int hs_plan_s::split_enqueue(const double2* A, const double2* B, int ldAB, const double* U,
                             int N_G, double2* H, double2* S, Workspace& w, cudaStream_t st,
                             bool timed, cudaEvent_t s_done, bool presliced, bool mirror) {
  int rc = presliced ? HS_OK : split_inputs(A, B, ldAB, U, N_G, w, st, 0, -1, timed);
  if (rc) return rc;
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[9], st));
  AtomsJob job{&w, N_G};
  rc = split_atoms(&job, 1, st, nullptr);
  if (rc) return rc;
  return split_outputs(A, ldAB, N_G, H, S, w, st, timed, s_done, presliced, mirror);
}

// ---------------------------------------------------------------------------
// hs_reduce on split plans: the two-sided transform C = L^{-1} H L^{-H} (Sec. 1.1) as
// two BF16 slice contractions.  With B = L^{-H} (upper triangular) and Z = H B / 2,
// C = Z^H B + B^H Z.  The full product H B comes from the lower triangle of M^H M for
// the stacked operand M = [B | 0 | H] (n complex rows; B at columns [0, n), zeros up
// to n_pad = rows_pad_of(n), H at [n_pad, n_pad + n)): below the split, its row blocks
// hold H^H B = H B, K-major as the next contraction reads it.  Only those row blocks
// are launched (bi0 = n_pad / BM), written through a base shifted back by n_pad rows.
// The second contraction reads B's slices as M's first n rows.

void hs_plan_s::split_reduce_release() {
  for (SliceBuf* b : {&red_M, &red_Zs, &red_M2}) {
    if (b->plain) cudaFree(b->plain);
    if (b->expo) cudaFree(b->expo);
    *b = SliceBuf{};
  }
  if (red_Z) cudaFree(red_Z);
  if (red_half) cudaFree(red_half);
  if (red_P2) cudaFree(red_P2);
  if (red_Z2) cudaFree(red_Z2);
  red_Z = red_Z2 = red_P2 = nullptr;
  red_half = nullptr;
  for (cudaEvent_t& e : red_pev)
    if (e) cudaEventDestroy(e);
  red_pev.clear();
  red_split_cap = 0;
}

int hs_plan_s::split_reduce_alloc(int n) {
  if (red_split_cap >= n) return HS_OK;
  split_reduce_release();
  if (!get_encode()) return HS_ECUDA;
  const int n_pad = rows_pad_of(n), NM = n_pad + n;
  const int rpM = rows_pad_of(NM), rp = rows_pad_of(n);
  const size_t kpad = (size_t)kpad_of(n, 1);
  const size_t oneM = (size_t)slices * rpM * kpad * 2, oneZ = (size_t)slices * rp * kpad * 2;
  const bool ok =
      cudaMalloc((void**)&red_M.plain, 2 * oneM) == cudaSuccess &&
      cudaMalloc((void**)&red_M.expo, sizeof(int) * rpM) == cudaSuccess &&
      cudaMalloc((void**)&red_Zs.plain, 2 * oneZ) == cudaSuccess &&
      cudaMalloc((void**)&red_Zs.expo, sizeof(int) * rp) == cudaSuccess &&
      cudaMalloc((void**)&red_Z, sizeof(double2) * (size_t)n * NM) == cudaSuccess &&
      cudaMalloc((void**)&red_half, sizeof(double) * (size_t)n) == cudaSuccess &&
      // the inverse's scratch: slices of K <= kRedPanel over up to n_pad + n columns,
      // a kRedPanel x n transposed block, an n x (n_pad + n) product
      cudaMalloc((void**)&red_M2.plain, (size_t)2 * slices * rpM * kpad_of(kRedPanel, 1) * 2) ==
          cudaSuccess &&
      cudaMalloc((void**)&red_M2.expo, sizeof(int) * rpM) == cudaSuccess &&
      cudaMalloc((void**)&red_P2, sizeof(double2) * (size_t)kRedPanel * n) == cudaSuccess &&
      cudaMalloc((void**)&red_Z2, sizeof(double2) * (size_t)n * NM) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    split_reduce_release();
    return HS_ENOMEM;
  }
  std::vector<double> half((size_t)n, 0.5);
  if (cudaMemcpy(red_half, half.data(), sizeof(double) * n, cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    split_reduce_release();
    return HS_ECUDA;
  }
  red_pev.assign((size_t)(n + kRedPanel - 1) / kRedPanel, nullptr);
  for (cudaEvent_t& e : red_pev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      split_reduce_release();
      return HS_ECUDA;
    }
  red_M.rot = red_Zs.rot = red_M2.rot = true;  // plain and rotated slices interleaved
  red_split_cap = n;
  return HS_OK;
}

static int contract_tiles(const SplitParams& P) {
  int tiles = 0;
  for (int b = P.bi0; b < P.nbi; ++b) tiles += 2 * std::min(b + 1, (P.nbj + 1) / 2);
  return tiles;
}

int hs_plan_s::split_reduce_transform(const double2* B, double2* H, int n, cudaStream_t st,
                                      cudaEvent_t mid) {
  if (precision != HS_SPLIT_BF16 || real || n < 1) return HS_EINVAL;
  int rc = split_reduce_alloc(n);
  if (rc) return rc;
  const int s = slices;
  const int n_pad = rows_pad_of(n), NM = n_pad + n;
  const int rpM = rows_pad_of(NM), rp = rows_pad_of(n);
  const int NKB = kpad_of(n, 1) / KB;
  int n_stage;
  size_t smem;
  rc = split_geometry(n_stage, smem);
  if (rc) return rc;
  // 1. slices of M: B (zeros past column n up to n_pad), then H from column n_pad on (the
  //    source pointer is shifted back so that column g reads H's column g - n_pad)
  {
    SliceParams sp{};
    sp.job[0] = SliceJob{B, nullptr, red_M.plain, red_M.rot, red_M.expo, n, n};
    rc = slice_launch(sp, 1, s, n, rpM, 1, false, st, 0, n_pad);
    if (rc) return rc;
    SliceParams sq{};
    const double2* Hs =
        (const double2*)((uintptr_t)H - (uintptr_t)n_pad * (uintptr_t)n * sizeof(double2));
    sq.job[0] = SliceJob{Hs, nullptr, red_M.plain, red_M.rot, red_M.expo, n, n};
    rc = slice_launch(sq, 1, s, NM, rpM, 1, false, st, n_pad, -1);
    if (rc) return rc;
  }
  SplitParams* PP = new (std::nothrow) SplitParams;
  if (!PP) return HS_ENOMEM;
  std::unique_ptr<SplitParams> own(PP);
  SplitParams& P = *PP;
  // 2. H B: row blocks of M's H part against every column block up to the diagonal
  std::memset(&P, 0, sizeof(P));
  if (!encode_left(&P.maps[0], red_M.plain, NKB, rpM / 64, s, true) ||
      !encode_right(&P.maps[1], red_M.plain, NKB, rpM / 64, s, true))
    return HS_ECUDA;
  P.seg[0] = SplitSeg{0, 1, NKB, red_M.expo, red_M.expo};
  P.nseg = 1;
  P.s = s;
  P.N_G = NM;
  P.ldC = n;
  P.nbj = (NM + BNC - 1) / BNC;
  P.rows_pad = rpM;
  P.err = err_d;
  P.bi0 = n_pad / BM;
  P.nbi = (NM + BM - 1) / BM;
  P.band = contract_band();
  P.ntiles = contract_tiles(P);
  P.C = (double2*)((uintptr_t)red_Z - (uintptr_t)n_pad * sizeof(double2));  // row n_pad -> 0
  P.n_stage = n_stage;
  rc = launch_gemm(MODE_CONTRACT, s, P.ntiles, smem, st, P);
  if (rc) return rc;
  if (mid && cudaEventRecord(mid, st) != cudaSuccess) return HS_ECUDA;
  // 3. slices of Z = (H B) / 2: the first n columns of red_Z, halved by the row weight
  {
    SliceParams sz{};
    sz.job[0] = SliceJob{red_Z, red_half, red_Zs.plain, red_Zs.rot, red_Zs.expo, n, n};
    rc = slice_launch(sz, 1, s, n, rp, 1, false, st);
    if (rc) return rc;
  }
  // 4. C = Z^H B + B^H Z, lower tiles, into H; then the mirror
  std::memset(&P, 0, sizeof(P));
  if (!encode_left(&P.maps[0], red_Zs.plain, NKB, rp / 64, s, true) ||
      !encode_right(&P.maps[1], red_Zs.plain, NKB, rp / 64, s, true) ||
      !encode_left(&P.maps[2], red_M.plain, NKB, rpM / 64, s, true) ||
      !encode_right(&P.maps[3], red_M.plain, NKB, rpM / 64, s, true))
    return HS_ECUDA;
  P.seg[0] = SplitSeg{0, 3, NKB, red_Zs.expo, red_M.expo};  // Z^H B
  P.seg[1] = SplitSeg{2, 1, NKB, red_M.expo, red_Zs.expo};  // B^H Z
  P.nseg = 2;
  P.s = s;
  P.N_G = n;
  P.ldC = n;
  P.nbj = (n + BNC - 1) / BNC;
  P.rows_pad = rp;
  P.err = err_d;
  P.bi0 = 0;
  P.nbi = (n + BM - 1) / BM;
  P.band = contract_band();
  P.ntiles = contract_tiles(P);
  P.C = H;
  P.n_stage = n_stage;
  rc = launch_gemm(MODE_CONTRACT, s, P.ntiles, smem, st, P);
  if (rc) return rc;
  return hs_launch_mirror(H, n, n, st) == cudaSuccess ? HS_OK : HS_ECUDA;
}

// ---------------------------------------------------------------------------
// General products on the slice path for the blocked Cholesky and inverse of hs_reduce.
// Operands are K-major (K complex rows x columns, column-major); red_M holds their
// slices (its capacity, sized for the two-sided transform, covers K <= kRedPanel and
// up to n_pad + n columns).

// out = lower(X^H X) (nc x nc, leading dimension nc; whole lower tiles written).
int hs_plan_s::split_herk_lower(const double2* X, int ldX, int K, int nc, double2* out,
                                SliceBuf& sb, cudaStream_t st) {
  const int s = slices, rp = rows_pad_of(nc), NKB = kpad_of(K, 1) / KB;
  int n_stage;
  size_t smem;
  int rc = split_geometry(n_stage, smem);
  if (rc) return rc;
  SliceParams sp{};
  sp.job[0] = SliceJob{X, nullptr, sb.plain, sb.rot, sb.expo, ldX, K};
  rc = slice_launch(sp, 1, s, nc, rp, 1, false, st);
  if (rc) return rc;
  SplitParams* PP = new (std::nothrow) SplitParams;
  if (!PP) return HS_ENOMEM;
  std::unique_ptr<SplitParams> own(PP);
  SplitParams& P = *PP;
  std::memset(&P, 0, sizeof(P));
  if (!encode_left(&P.maps[0], sb.plain, NKB, rp / 64, s, sb.rot) ||
      !encode_right(&P.maps[1], sb.plain, NKB, rp / 64, s, sb.rot))
    return HS_ECUDA;
  P.seg[0] = SplitSeg{0, 1, NKB, sb.expo, sb.expo};
  P.nseg = 1;
  P.s = s;
  P.N_G = nc;
  P.ldC = nc;
  P.nbj = (nc + BNC - 1) / BNC;
  P.rows_pad = rp;
  P.err = err_d;
  P.bi0 = 0;
  P.nbi = (nc + BM - 1) / BM;
  P.band = contract_band();
  P.ntiles = contract_tiles(P);
  P.C = out;
  P.n_stage = n_stage;
  return launch_gemm(MODE_CONTRACT, s, P.ntiles, smem, st, P);
}

// out = A^H B (m x nc) for A (K x m) and B (K x nc): the block below the split of
// lower(M^H M) for M = [B | 0 | A] (zeros from column nc up to nc_pad); out is
// m x (nc_pad + m) with leading dimension m, the product in its first nc columns.
int hs_plan_s::split_gemm_ahb(const double2* A, int ldA, int m, const double2* B, int ldB, int nc,
                              int K, double2* out, SliceBuf& sb, cudaStream_t st) {
  const int s = slices, nc_pad = rows_pad_of(nc), NM = nc_pad + m, rpM = rows_pad_of(NM);
  const int NKB = kpad_of(K, 1) / KB;
  int n_stage;
  size_t smem;
  int rc = split_geometry(n_stage, smem);
  if (rc) return rc;
  SliceParams sp{};
  sp.job[0] = SliceJob{B, nullptr, sb.plain, sb.rot, sb.expo, ldB, K};
  rc = slice_launch(sp, 1, s, nc, rpM, 1, false, st, 0, nc_pad);
  if (rc) return rc;
  SliceParams sq{};
  const double2* As =
      (const double2*)((uintptr_t)A - (uintptr_t)nc_pad * (uintptr_t)ldA * sizeof(double2));
  sq.job[0] = SliceJob{As, nullptr, sb.plain, sb.rot, sb.expo, ldA, K};
  rc = slice_launch(sq, 1, s, NM, rpM, 1, false, st, nc_pad, -1);
  if (rc) return rc;
  SplitParams* PP = new (std::nothrow) SplitParams;
  if (!PP) return HS_ENOMEM;
  std::unique_ptr<SplitParams> own(PP);
  SplitParams& P = *PP;
  std::memset(&P, 0, sizeof(P));
  if (!encode_left(&P.maps[0], sb.plain, NKB, rpM / 64, s, sb.rot) ||
      !encode_right(&P.maps[1], sb.plain, NKB, rpM / 64, s, sb.rot))
    return HS_ECUDA;
  P.seg[0] = SplitSeg{0, 1, NKB, sb.expo, sb.expo};
  P.nseg = 1;
  P.s = s;
  P.N_G = NM;
  P.ldC = m;
  P.nbj = (NM + BNC - 1) / BNC;
  P.rows_pad = rpM;
  P.err = err_d;
  P.bi0 = nc_pad / BM;
  P.nbi = (NM + BM - 1) / BM;
  P.band = contract_band();
  P.ntiles = contract_tiles(P);
  P.C = (double2*)((uintptr_t)out - (uintptr_t)nc_pad * sizeof(double2));  // row nc_pad -> 0
  P.n_stage = n_stage;
  return launch_gemm(MODE_CONTRACT, s, P.ntiles, smem, st, P);
}

// Right-looking Cholesky in panels of kRedPanel columns: each panel in FP64, then
// S22 -= L21 L21^H = lower(X^H X) with X = L21^H on the slice path.
int hs_plan_s::split_cholesky(double2* S, int n, int* fail, cudaStream_t st) {
  int rc = split_reduce_alloc(n);
  if (rc) return rc;
  for (int j0 = 0; j0 < n; j0 += kRedPanel) {
    const int pw = std::min(kRedPanel, n - j0);
    if (hs_launch_cholesky_panel(S, n, j0, pw, fail, st) != cudaSuccess) return HS_ECUDA;
    // panel j0 / kRedPanel of L is final: later updates touch columns right of it only
    if (cudaEventRecord(red_pev[j0 / kRedPanel], st) != cudaSuccess) return HS_ECUDA;
    const int r0 = j0 + pw, n2 = n - r0;
    if (n2 <= 0) break;
    double2* X = red_P;  // pw x n2, leading dimension pw
    if (hs_launch_ctrans(S + (size_t)r0 + (size_t)j0 * n, n, n2, pw, X, pw, st) != cudaSuccess)
      return HS_ECUDA;
    rc = split_herk_lower(X, pw, pw, n2, red_Z, red_M, st);
    if (rc) return rc;
    if (hs_launch_sub(S + (size_t)r0 + (size_t)r0 * n, n, red_Z, n2, n2, n2, 1, fail, st) !=
        cudaSuccess)
      return HS_ECUDA;
  }
  return hs_launch_zero_upper(S, n, fail, st) == cudaSuccess ? HS_OK : HS_ECUDA;
}

// Forward substitution L W = I in block rows of kRedPanel: each block row in FP64,
// then W[r0 :, 0 : ncols] -= L[r0 :, i0 : i0 + pw] W[i0 : i0 + pw, 0 : ncols] on the
// slice path (A = that block of L, conjugate-transposed to K-major).  Block row i reads
// L's panel i only: it starts once split_cholesky has recorded that panel's event.
int hs_plan_s::split_inverse(const double2* L, double2* W, int n, const int* fail,
                             cudaStream_t st) {
  int rc = split_reduce_alloc(n);
  if (rc) return rc;
  if (hs_launch_eye(W, n, fail, st) != cudaSuccess) return HS_ECUDA;
  for (int i0 = 0; i0 < n; i0 += kRedPanel) {
    const int pw = std::min(kRedPanel, n - i0);
    if (cudaStreamWaitEvent(st, red_pev[i0 / kRedPanel], 0) != cudaSuccess) return HS_ECUDA;
    if (hs_launch_inverse_blockrow(L, W, n, i0, pw, fail, st) != cudaSuccess) return HS_ECUDA;
    const int r0 = i0 + pw, m = n - r0, ncols = i0 + pw;
    if (m <= 0) break;
    double2* A = red_P2;  // pw x m, leading dimension pw
    if (hs_launch_ctrans(L + (size_t)r0 + (size_t)i0 * n, n, m, pw, A, pw, st) != cudaSuccess)
      return HS_ECUDA;
    rc = split_gemm_ahb(A, pw, m, W + i0, n, ncols, pw, red_Z2, red_M2, st);
    if (rc) return rc;
    if (hs_launch_sub(W + r0, n, red_Z2, m, m, ncols, 0, fail, st) != cudaSuccess)
      return HS_ECUDA;
  }
  return HS_OK;
}
