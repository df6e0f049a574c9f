// Slicers of the split-precision form: FP64 operands and per-atom operators to BF16
// slices (the signed-digit split described in k_split.cu), written in the blocked
// layout the slice-GEMM kernel's tensor maps read.
#include <cuda_runtime.h>

#include <cstdint>

#include "split_common.h"

using namespace hs_split;

namespace {

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

}  // namespace

namespace hs_split {

int slice_launch(SliceParams& sp, int nj, int s, int N_G, int rp, int N_L, bool real,
                 cudaStream_t st, int g0, int ng, int threads) {
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

int slice_op_launch(const double2* M, int job, int N_A, int N_L, int Pk, int n_pad, int s,
                    uint16_t* out, int* expo, bool real, cudaStream_t st) {
  if (real)
    k_slice_op_real<<<dim3(n_pad, N_A), 128, 0, st>>>(M, job, N_A, N_L, Pk, n_pad, s, out, expo);
  else
    k_slice_op<<<dim3(n_pad, N_A), 128, 0, st>>>(M, job, N_A, N_L, Pk, n_pad, s, out, expo);
  return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ECUDA;
}

}  // namespace hs_split
