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
#include <new>

#include "split_common.h"

using namespace hs_split;

namespace {

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
// W = 8 or 16 consecutive TMEM columns of this warp's 32 lanes, one register each.
template <int W>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[W]) {
  static_assert(W == 8 || W == 16, "8 or 16 columns");
  uint32_t r[W];
  if constexpr (W == 8) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  }
#pragma unroll
  for (int i = 0; i < W; ++i) v[i] = __uint_as_float(r[i]);
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
//
// drain_cols reads W columns of every accumulator in MASK with one load-and-wait
// round trip and folds them into pairs k0 .. k0 + W/2 - 1.  Every round trip waits
// out the TMEM load latency, so drain16 takes the widest reads the 96-register budget
// holds: the common window (levels 2 and >= 3 due) in one round trip of 16 columns,
// three accumulators in two of 8, and all four in four of 8 (levels 0 and 1, then 2
// and >= 3, so that every element still sees levels 0, 1, 2, 3 in that order and the
// result is unchanged).
template <int S, uint32_t MASK, int W>
__device__ __forceinline__ void drain_cols(uint32_t taddr, int k0, f32x2 (&hi)[8],
                                           f32x2 (&lo)[8]) {
  constexpr bool r0 = MASK & 1u, r1 = MASK & 2u, r2 = S >= 3 && (MASK & 4u),
                 r3 = S >= 4 && (MASK & 8u);
  float v0[W], v1[W], v2[W], v3[W];
  if (r0) tmem_ld<W>(taddr, v0);
  if (r1) tmem_ld<W>(taddr + BN, v1);
  if (r2) tmem_ld<W>(taddr + 2 * BN, v2);
  if (r3) tmem_ld<W>(taddr + 3 * BN, v3);
  tmem_wait_ld();
#pragma unroll
  for (int c = 0; c < W; c += 2) {
    const int k = k0 + (c >> 1);
    if (r0) two_sum_acc2(hi[k], lo[k], pack2(v0[c], v0[c + 1]));
    if (r1) two_sum_acc2(hi[k], lo[k], pack2(v1[c], v1[c + 1]));
    if (r2) fast_two_sum_acc2(hi[k], lo[k], pack2(v2[c], v2[c + 1]));
    if (r3) lo[k] = add2(lo[k], pack2(v3[c], v3[c + 1]));
  }
}
template <int S, uint32_t MASK>
__device__ __forceinline__ void drain16(uint32_t taddr, f32x2 (&hi)[8], f32x2 (&lo)[8]) {
  if constexpr (MASK == 0xCu) {
    drain_cols<S, MASK, 16>(taddr, 0, hi, lo);
  } else if constexpr (S >= 4 && MASK == 0xFu) {
#pragma unroll
    for (int c0 = 0; c0 < 16; c0 += 8) {
      drain_cols<S, 0x3u, 8>(taddr + c0, c0 >> 1, hi, lo);
      drain_cols<S, 0xCu, 8>(taddr + c0, c0 >> 1, hi, lo);
    }
  } else {
#pragma unroll
    for (int c0 = 0; c0 < 16; c0 += 8) drain_cols<S, MASK, 8>(taddr + c0, c0 >> 1, hi, lo);
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
      if (!is_contract(MODE) && (!ok || *abort_flag)) break;
      // Results: (hi + lo) * 2^(E_row + E_col) in FP64.  Thread = one tile row; pair k
      // of a strip = its TMEM columns 16 cg + 2k and 2k + 1 (lanes 2k, 2k + 1 of eC*).
      if (is_contract(MODE)) {
        // one tile per CTA: stage (hi, lo) in the idle ring (every stage was consumed by
        // an MMA that completed before the last acc_full), then write the tile with
        // consecutive threads on consecutive output addresses.  Every drain warp reaches
        // the staging barrier exactly once, also after a failed wait (the launch then
        // reports an error and stores nothing): warps that leave here on their own view
        // of the abort flag would otherwise leave the others at the barrier.
        float2* stg = (float2*)smem;  // [2 strips][64 cols][128 rows]
        int* s_erow = (int*)(smem + 2 * 64 * 128 * sizeof(float2));
        int* s_ecol = s_erow + 128;   // [128]: exponent of each TMEM column
        const int r = 32 * q4 + lane;
        const bool good = ok && !*abort_flag;
        if (good)
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
        if (!good) {
        } else if (is_real(MODE)) {  // 128 real columns
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

}  // namespace

// ------------------------------------------------------------------ launches

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

namespace hs_split {

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

// The launch parameters as they go to the device: the stall flag.
static void set_waits(SplitParams& P) { P.stall = stall_injection() ? 1 : 0; }

int launch_gemm(int mode, int s, int grid, size_t smem, cudaStream_t st,
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

int graph_launch_atoms(AtomsGraph& G, int s, int grid, size_t smem, cudaStream_t st,
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


}  // namespace hs_split
