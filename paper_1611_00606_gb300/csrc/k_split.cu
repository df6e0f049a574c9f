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
// BF16.  Products of two slices are exact; summed over a window of 256 real K
// of 128 real K the slice-pair levels 0 (d_1 e_1), 1 (d_1 e_2 + d_2 e_1) and
// 2 (d_1 e_3 + d_2 e_2 + d_3 e_1) stay within 2^24 units and are therefore
// exact in FP32 tensor-core accumulators, whatever the accumulator's rounding.
// Levels >= 3 (2^-27 and below) share a fourth, inexact accumulator.  After
// every window the four TMEM accumulators are drained into a double-float
// (hi, lo FP32 pair) accumulator per output element, scaled by 2^{E_i + E_j}:
// levels 0, 1 and 2 through an error-free TwoSum into hi, levels >= 3 into lo
// (the leading digit is typically small, so level 2 is only ~2^-14 below
// level 0 and would cap the pair's precision if it went to lo directly).
// The pair is summed to FP64 once per tile at the end.
//
// Complex arithmetic on real tensor cores: with the K-major interleaved
// (re, im) storage, Re(L^H R) = L'^T R' and Im(L^H R) = L'^T R'' where R''
// holds (im, -re) pairs.  One MMA with N = 128 computes a 128 x 64 complex
// tile: B rows 0..63 come from R', rows 64..127 from R''.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <vector>

#include "plan.h"

namespace {

constexpr int BM = 128;        // complex rows per tile (MMA M)
constexpr int BNC = 64;        // complex columns per tile
constexpr int BN = 2 * BNC;    // MMA N (Re | Im)
constexpr int KB = 16;         // real K per pipeline stage (= one MMA K step)
constexpr int WIN = 8;         // stages per exact window (128 real K)
constexpr int ROWS_ALIGN = 128;
constexpr int kMaxMaps = 13;
constexpr int kMaxJobs = 7;
constexpr int TILE_BYTES = 64 * KB * 2;  // one 64-row TMA box: 2 KB
constexpr int NUM_THREADS = 320;         // warp 0 TMA, warp 1 MMA, warps 2..9 drain
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded waits: 2 s

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
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
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
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  const float ap = s - bp;
  lo += (hi - ap) + (v - bp);
  hi = s;
}


// Drain one 32-column strip of the four window accumulators (level k at
// column offset k*BN) into (hi, lo) pairs.  rsc = 2^eL (this thread's row);
// lane c of csc holds 2^eR of column c.
__device__ __forceinline__ void drain_cols(uint32_t taddr, int s, float rsc, float csc,
                                           float (&hi)[32], float (&lo)[32]) {
#pragma unroll
  for (int c0 = 0; c0 < 32; c0 += 4) {
    float v0[4], v1[4], v2[4], v3[4];
    tmem_ld4(taddr + c0, v0);
    tmem_ld4(taddr + BN + c0, v1);
    if (s >= 3) tmem_ld4(taddr + 2 * BN + c0, v2);
    if (s >= 4) tmem_ld4(taddr + 3 * BN + c0, v3);
    tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float sc = rsc * __shfl_sync(0xffffffffu, csc, c0 + c);
      two_sum_acc(hi[c0 + c], lo[c0 + c], v0[c] * sc);
      two_sum_acc(hi[c0 + c], lo[c0 + c], v1[c] * sc);
      if (s >= 3) two_sum_acc(hi[c0 + c], lo[c0 + c], v2[c] * sc);
      if (s >= 4) lo[c0 + c] = fmaf(v3[c], sc, lo[c0 + c]);
    }
  }
}

// ------------------------------------------------------------------ contraction

struct SplitSeg {
  int mL, mR, mRr;  // tensor maps of L', R', R''
  int kblocks;      // stages of KB real K
  const int* eL;    // exponents of the L source columns
  const int* eR;    // exponents of the R source columns
};

struct __align__(64) SplitParams {
  CUtensorMap maps[kMaxMaps];
  SplitSeg seg[kMaxSeg];
  int nseg;
  int s;          // slices
  int n_stage;    // pipeline depth
  int N_G, ldC, nbj;
  int rows_pad;   // slice p of an operand starts at row p * rows_pad
  double2* C;
  int* err;
};

__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_contract_split(const __grid_constant__ SplitParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = P.s;
  const int NS = P.n_stage;
  const uint32_t a_bytes = (uint32_t)s * 2 * TILE_BYTES;   // s slices x 128 rows
  const uint32_t stage_bytes = 2 * a_bytes;                 // A part + B part
  uint64_t* full = (uint64_t*)(smem + NS * stage_bytes);
  uint64_t* empty = full + NS;
  uint64_t* acc_full = empty + NS;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* done = acc_empty + 1;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  // lower-triangle tile of 128 x 64: row block bi, column block bj <= 2 bi + 1
  int t = blockIdx.x, bi = 0;
  for (;;) {
    const int n = min(2 * bi + 2, P.nbj);
    if (t < n) break;
    t -= n;
    ++bi;
  }
  const int bj = t;
  const int i0 = bi * BM, j0 = bj * BNC;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 8);
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0 && lane == 0)
    for (int sg = 0; sg < P.nseg; ++sg) {
      prefetch_map(&P.maps[P.seg[sg].mL]);
      prefetch_map(&P.maps[P.seg[sg].mR]);
      prefetch_map(&P.maps[P.seg[sg].mRr]);
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

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int slot = 0;
      uint32_t phase = 0;
      uint32_t armed = 0;        // bit i: slot i was armed at least once
      uint32_t armed_par = 0;    // bit i: parity of the last armed phase of slot i
      bool ok = true;
      for (int sg = 0; sg < P.nseg && ok; ++sg) {
        const SplitSeg S = P.seg[sg];
        const CUtensorMap* mL = &P.maps[S.mL];
        const CUtensorMap* mR = &P.maps[S.mR];
        const CUtensorMap* mRr = &P.maps[S.mRr];
        for (int kb = 0; kb < S.kblocks; ++kb) {
          if (!mbar_wait(&empty[slot], phase ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[slot], stage_bytes);
          armed |= 1u << slot;
          armed_par = (armed_par & ~(1u << slot)) | (phase << slot);
          const uint32_t sa = smem_u32(smem + slot * stage_bytes);
          const uint32_t sb = sa + a_bytes;
          const int x = kb * KB;
          for (int p = 0; p < s; ++p) {
            const int yr = p * P.rows_pad;
            tma_load_2d(sa + p * 2 * TILE_BYTES, mL, x, yr + i0, &full[slot]);
            tma_load_2d(sa + p * 2 * TILE_BYTES + TILE_BYTES, mL, x, yr + i0 + 64, &full[slot]);
            tma_load_2d(sb + p * 2 * TILE_BYTES, mR, x, yr + j0, &full[slot]);
            tma_load_2d(sb + p * 2 * TILE_BYTES + TILE_BYTES, mRr, x, yr + j0, &full[slot]);
          }
          if (++slot == NS) {
            slot = 0;
            phase ^= 1u;
          }
        }
      }
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
      for (int sg = 0; sg < P.nseg && ok; ++sg) {
        const int kbn = P.seg[sg].kblocks;
        for (int w0 = 0; w0 < kbn && ok; w0 += WIN) {
          if (nwin > 0 && !mbar_wait(acc_empty, (uint32_t)(nwin - 1) & 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int w1 = min(kbn, w0 + WIN);
          for (int kb = w0; kb < w1; ++kb) {
            if (!mbar_wait(&full[slot], phase, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + slot * stage_bytes);
            const uint32_t sb = sa + a_bytes;
            const bool first = (kb == w0);
            for (int p = 0; p < s; ++p) {
              const uint64_t ad = sdesc_sw32(sa + p * 2 * TILE_BYTES);
              for (int q = 0; p + q < s; ++q) {
                const int lvl = p + q;
                const int acc = lvl < 3 ? lvl : 3;
                const bool init = first && p == 0 && q == acc;  // first pair of this level
                tc_mma_bf16(tmem + acc * BN, ad, sdesc_sw32(sb + q * 2 * TILE_BYTES), kIdesc,
                            init ? 0u : 1u);
              }
            }
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
    // ---------------- drain warps 2..9: TMEM -> double-float accumulators
    const int q4 = warp & 3;        // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;  // column half
    const int row = i0 + 32 * q4 + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * q4) << 16);
    float hr[32], lr[32], hi_[32], li[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) hr[c] = lr[c] = hi_[c] = li[c] = 0.f;
    int nwin = 0;
    bool ok = true;
    for (int sg = 0; sg < P.nseg && ok; ++sg) {
      const SplitSeg S = P.seg[sg];
      const float rsc = pow2f(S.eL[row]);
      const float csc = pow2f(S.eR[j0 + 32 * h + lane]);  // lane c: column c's scale
      for (int w0 = 0; w0 < S.kblocks; w0 += WIN) {
        if (!mbar_wait(acc_full, (uint32_t)nwin & 1u, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        drain_cols(tl + (uint32_t)(32 * h), s, rsc, csc, hr, lr);            // Re
        drain_cols(tl + (uint32_t)(BNC + 32 * h), s, rsc, csc, hi_, li);     // Im
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);
        ++nwin;
      }
    }
    if (!ok) {
      atomicExch(P.err, 3);
      *abort_flag = 1;
    } else if (row < P.N_G) {
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int j = j0 + 32 * h + c;
        if (j < P.N_G)
          P.C[row + (size_t)j * P.ldC] =
              make_double2((double)hr[c] + (double)lr[c], (double)hi_[c] + (double)li[c]);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ------------------------------------------------------------------ slicer

struct SliceJob {
  const double2* X;  // source: K x N_G complex, column-major, ld ldX
  const double* u;   // optional real row weight (the U norms), may be null
  uint16_t* plain;   // [s][rows_pad][kpad] BF16 slices of (re, im) pairs
  uint16_t* rot;     // same for (im, -re) pairs, may be null
  int* expo;         // [rows_pad] column exponents
  int ldX, K, kpad;
};
struct SliceParams {
  SliceJob job[kMaxJobs];
  int s, N_G, rows_pad;
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

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

__global__ void __launch_bounds__(256) k_slice(const __grid_constant__ SliceParams P) {
  const SliceJob J = P.job[blockIdx.y];
  const int g = blockIdx.x;
  const int s = P.s;
  const size_t slice_elems = (size_t)P.rows_pad * J.kpad;
  __shared__ double red[32];
  __shared__ int s_E;
  const int kc = J.kpad / 2;  // complex entries per padded row
  if (g >= P.N_G) {
    for (int k = threadIdx.x; k < kc; k += blockDim.x)
      for (int p = 0; p < s; ++p) {
        ((uint32_t*)(J.plain + p * slice_elems + (size_t)g * J.kpad))[k] = 0u;
        if (J.rot) ((uint32_t*)(J.rot + p * slice_elems + (size_t)g * J.kpad))[k] = 0u;
      }
    if (threadIdx.x == 0) J.expo[g] = 0;
    return;
  }
  const double2* col = J.X + (size_t)g * J.ldX;
  double m = 0.0;
  for (int k = threadIdx.x; k < J.K; k += blockDim.x) {
    double2 v = col[k];
    const double w = J.u ? fabs(J.u[k]) : 1.0;
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)) * w);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = fmax(mm, red[i]);
    int e = 0;
    if (mm > 0.0 && isfinite(mm)) frexp(mm, &e);
    s_E = (mm > 0.0 && isfinite(mm)) ? e - 7 : 0;
    J.expo[g] = s_E;
  }
  __syncthreads();
  const int E = s_E;
  for (int k = threadIdx.x; k < kc; k += blockDim.x) {
    int dr[kMaxSlices], di[kMaxSlices];
    bool bad = false;
    if (k < J.K) {
      double2 v = col[k];
      if (J.u) {
        v.x *= J.u[k];
        v.y *= J.u[k];
      }
      bad = !(isfinite(v.x) && isfinite(v.y));
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
          pl = (uint32_t)bf16_bits((float)dr[p] * sc) |
               ((uint32_t)bf16_bits((float)di[p] * sc) << 16);
          rt = (uint32_t)bf16_bits((float)di[p] * sc) |
               ((uint32_t)bf16_bits((float)(-dr[p]) * sc) << 16);
        }
        ((uint32_t*)(J.plain + p * slice_elems + (size_t)g * J.kpad))[k] = pl;
        if (J.rot) ((uint32_t*)(J.rot + p * slice_elems + (size_t)g * J.kpad))[k] = rt;
      }
    }
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

bool encode_map(CUtensorMap* m, const uint16_t* base, int kpad, int rows_total) {
  auto fn = get_encode();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows_total};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)KB, 64u};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

static inline int kpad_of(int K) { return ((2 * K + KB - 1) / KB) * KB; }
static inline int rows_pad_of(int N_G) { return ((N_G + ROWS_ALIGN - 1) / ROWS_ALIGN) * ROWS_ALIGN; }

// Complex rows (K) of each source and whether it needs the rotated copy.
static void source_shape(int src, int K, int N_L, int n_fail, int& rows, bool& rot) {
  rot = (src != SRC_AF);
  rows = (src == SRC_AF || src == SRC_X) ? n_fail * N_L : K;
}

static size_t slicebuf_bytes(int s, int rows_pad, int Kc, bool rot) {
  const size_t one = (size_t)s * rows_pad * kpad_of(Kc) * 2;
  return (rot ? 2 : 1) * one + sizeof(int) * rows_pad;
}

size_t hs_plan_s::split_ws_bytes(int N_G, int n_fail) const {
  if (precision != HS_SPLIT_BF16) return 0;
  const int K = N_A * N_L;
  const int nf = n_fail > 0 ? n_fail : 1;
  const int rp = rows_pad_of(N_G);
  size_t b = 0;
  for (int src = 0; src < NSRC; ++src) {
    int rows;
    bool rot;
    source_shape(src, K, N_L, nf, rows, rot);
    b += slicebuf_bytes(slices, rp, rows, rot);
  }
  return b;
}

int hs_plan_s::split_ws_alloc(Workspace& w, int N_G, int n_fail, cudaStream_t st, bool async) {
  if (precision != HS_SPLIT_BF16) return HS_OK;
  if (!get_encode()) return HS_ECUDA;
  const int K = N_A * N_L;
  const int rp = rows_pad_of(N_G);
  auto al = [&](void** ptr, size_t bytes) -> bool {
    return (async ? hs_malloc_async(ptr, bytes, st, hs_serve_pool(this)) : cudaMalloc(ptr, bytes)) ==
           cudaSuccess;
  };
  for (int src = 0; src < NSRC; ++src) {
    int rows;
    bool rot;
    source_shape(src, K, N_L, n_fail, rows, rot);
    const size_t one = (size_t)slices * rp * kpad_of(rows) * 2;
    if (!al((void**)&w.sb[src].plain, one)) return HS_ENOMEM;
    if (rot && !al((void**)&w.sb[src].rot, one)) return HS_ENOMEM;
    if (!al((void**)&w.sb[src].expo, sizeof(int) * rp)) return HS_ENOMEM;
  }
  return HS_OK;
}

int hs_plan_s::split_enqueue(const SegList& sS, const SegList& sH, int N_G, double2* H,
                             double2* S, Workspace& w, cudaStream_t st, bool timed) {
  const int K = N_A * N_L;
  const int N_h = N_A - N_f;
  const int s = slices;
  const int rp = rows_pad_of(N_G);
  if (rows_pad_of(w.N_G) < rp || w.n_fail < N_f || !w.sb[SRC_A].plain) return HS_EINVAL;
  // sources: sS.s[0] = (A, A), sS.s[1] = (B, B, U), sH.s[0] = (Z, B), then (Y, Y), (A_f, X_f)
  const Seg& sA = sS.s[0];
  const Seg& sUB = sS.s[1];
  const Seg& sZ = sH.s[0];
  const double2* Yp = nullptr;
  const double2* AFp = nullptr;
  const double2* Xp = nullptr;
  int ldW = K, ldAF = 1;
  for (int i = 2; i < sH.n; ++i) {
    if (sH.s[i].L == sH.s[i].R) {
      Yp = sH.s[i].L;
      ldW = sH.s[i].ldL;
    } else {
      AFp = sH.s[i].L;
      ldAF = sH.s[i].ldL;
      Xp = sH.s[i].R;
    }
  }
  SliceParams sp{};
  sp.s = s;
  sp.N_G = N_G;
  sp.rows_pad = rp;
  int nj = 0;
  auto job = [&](int src, const double2* X, int ldX, int Kr, const double* u) {
    SliceBuf& b = w.sb[src];
    sp.job[nj++] = SliceJob{X, u, b.plain, b.rot, b.expo, ldX, Kr, kpad_of(Kr)};
  };
  job(SRC_A, sA.L, sA.ldL, K, nullptr);
  job(SRC_UB, sUB.L, sUB.ldL, K, sUB.u);
  job(SRC_Z, sZ.L, sZ.ldL, K, nullptr);
  job(SRC_B, sZ.R, sZ.ldR, K, nullptr);
  if (N_h > 0) job(SRC_Y, Yp, ldW, N_h * N_L, nullptr);
  if (N_f > 0) {
    job(SRC_AF, AFp, ldAF, N_f * N_L, nullptr);
    job(SRC_X, Xp, ldW, N_f * N_L, nullptr);
  }
  k_slice<<<dim3(rp, nj), 256, 0, st>>>(sp);
  HS_CUDA_TRY(cudaGetLastError());
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[5], st));

  // tensor maps: index = 2*src + {0 plain, 1 rot} except A_f (plain only)
  SplitParams P;
  std::memset(&P, 0, sizeof(P));
  int map_of[NSRC][2];
  int nm = 0;
  // a slice array's rows: rp per slice (this call's padding, within capacity)
  auto add_map = [&](int src, int Kr) -> int {
    SliceBuf& b = w.sb[src];
    map_of[src][0] = nm;
    if (!encode_map(&P.maps[nm++], b.plain, kpad_of(Kr), s * rp)) return HS_ECUDA;
    if (b.rot) {
      map_of[src][1] = nm;
      if (!encode_map(&P.maps[nm++], b.rot, kpad_of(Kr), s * rp)) return HS_ECUDA;
    }
    return HS_OK;
  };
  int rc = HS_OK;
  rc |= add_map(SRC_A, K);
  rc |= add_map(SRC_UB, K);
  rc |= add_map(SRC_Z, K);
  rc |= add_map(SRC_B, K);
  if (N_h > 0) rc |= add_map(SRC_Y, N_h * N_L);
  if (N_f > 0) {
    rc |= add_map(SRC_AF, N_f * N_L);
    rc |= add_map(SRC_X, N_f * N_L);
  }
  if (rc != HS_OK) return HS_ECUDA;

  P.s = s;
  P.N_G = N_G;
  P.ldC = N_G;
  P.nbj = (N_G + BNC - 1) / BNC;
  P.rows_pad = rp;
  P.err = err_d;
  const int stage_bytes = 4 * s * TILE_BYTES;
  const int budget = 227 * 1024 - 1024 - 256;
  P.n_stage = budget / stage_bytes;
  if (P.n_stage > 8) P.n_stage = 8;
  if (P.n_stage < 2) return HS_EINVAL;
  const size_t smem = (size_t)P.n_stage * stage_bytes + 1024 + 256;
  HS_CUDA_TRY(cudaFuncSetAttribute(k_contract_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  const int nbi = (N_G + BM - 1) / BM;
  int tiles = 0;
  for (int b = 0; b < nbi; ++b) tiles += std::min(2 * b + 2, P.nbj);
  auto seg = [&](int srcL, int srcR, int Kr) {
    SplitSeg g;
    g.mL = map_of[srcL][0];
    g.mR = map_of[srcR][0];
    g.mRr = map_of[srcR][1];
    g.kblocks = kpad_of(Kr) / KB;
    g.eL = w.sb[srcL].expo;
    g.eR = w.sb[srcR].expo;
    return g;
  };
  // S = A^H A + (UB)^H (UB)
  P.nseg = 2;
  P.seg[0] = seg(SRC_A, SRC_A, K);
  P.seg[1] = seg(SRC_UB, SRC_UB, K);
  P.C = S;
  k_contract_split<<<tiles, NUM_THREADS, smem, st>>>(P);
  HS_CUDA_TRY(cudaGetLastError());
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[6], st));
  // H = Z^H B + B^H Z + Y^H Y + A_f^H X_f
  int n = 0;
  P.seg[n++] = seg(SRC_Z, SRC_B, K);
  P.seg[n++] = seg(SRC_B, SRC_Z, K);
  if (N_h > 0) P.seg[n++] = seg(SRC_Y, SRC_Y, N_h * N_L);
  if (N_f > 0) P.seg[n++] = seg(SRC_AF, SRC_X, N_f * N_L);
  P.nseg = n;
  P.C = H;
  k_contract_split<<<tiles, NUM_THREADS, smem, st>>>(P);
  HS_CUDA_TRY(cudaGetLastError());
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[7], st));
  return HS_OK;
}
