// Reduction of the generalized eigenproblem H c = lambda S c of one k-point
// (Sec. 1.1) to standard form, FP64:
//
//   S = L L^H            blocked right-looking Cholesky (64-column panels)
//   W = L^{-1}           blocked forward substitution on the identity
//   P = W tril_h(H)      tril_h(H): lower triangle of H, diagonal Re(H_jj) / 2, so
//                        that H = tril_h(H) + tril_h(H)^H for Hermitian H
//   G = P W^H            then C = L^{-1} H L^{-H} = G + G^H
//
// All N^3 work runs in one tiled complex GEMM (k_zgemm) that skips the zero
// triangles of its operands tile by tile: 4/3 (Cholesky) + 4/3 (inverse) +
// 4/3 (P) + 8/3 (G) = 20/3 N^3 real flops.  FP64 on GB300 issues about two DFMA
// per clock per SM, so these kernels are bound by the FP64 pipe, not by memory.
//
// Every kernel first reads the failure word: once a Cholesky pivot is not
// strictly positive (zero, negative or NaN) the rest of the chain does nothing.
#include <cuda_runtime.h>

#include "hs_internal.h"

namespace {

constexpr int NB = 64;   // diagonal block of the Cholesky and of the inverse
constexpr int kNumSMs = 152;  // GB300
constexpr int RK = 16;   // K step of k_zgemm
constexpr int kThreads = 256;

__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
// acc -= a conj(b)
__device__ __forceinline__ void zfms_conj(double2& acc, double2 a, double2 b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(-a.y, b.x, acc.y);
  acc.y = fma(a.x, b.y, acc.y);
}
// acc -= a b
__device__ __forceinline__ void zfms(double2& acc, double2 a, double2 b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc += a b
__device__ __forceinline__ void zfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// ---------------------------------------------------------------------------
// Cholesky of the jb x jb diagonal block at (j0, j0), in shared memory.  Reads the
// lower triangle (the trailing updates of the earlier panels have been applied);
// writes L's lower triangle back.  A pivot that is not strictly positive sets
// *fail = j0 + k + 1 (1-based column) and ends the block.
__global__ void __launch_bounds__(kThreads) k_potrf_diag(double2* __restrict__ S, int ld, int j0,
                                                         int jb, int* __restrict__ fail) {
  extern __shared__ double2 a[];  // NB x NB column-major: a[c * NB + r]
  if (*fail) return;
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += kThreads) {
    const int r = e % NB, c = e / NB;
    a[e] = (r < jb && c < jb && r >= c) ? S[(size_t)(j0 + r) + (size_t)(j0 + c) * ld]
                                        : make_double2(0.0, 0.0);
  }
  __shared__ double s_rl;  // 1 / L_kk of the current column
  for (int k = 0; k < jb; ++k) {
    __syncthreads();
    const double d = a[k * NB + k].x;
    if (!(d > 0.0)) {  // the same value in every thread: the whole block leaves
      if (tid == 0) atomicCAS(fail, 0, j0 + k + 1);
      return;
    }
    // one thread takes 1/sqrt (FP64 issues slowly on this GPU: every warp repeating it
    // cost as much as the column's update); L_kk = d / sqrt(d)
    double l = 0.0;
    if (tid == 0) {
      const double rl = rsqrt(d);
      l = d * rl;
      s_rl = rl;
    }
    __syncthreads();  // every thread has read d: the diagonal may now hold L_kk
    if (tid == 0) a[k * NB + k] = make_double2(l, 0.0);
    const double rl = s_rl;
    for (int r = k + 1 + tid; r < jb; r += kThreads) {
      a[k * NB + r].x *= rl;
      a[k * NB + r].y *= rl;
    }
    __syncthreads();
    // trailing lower triangle, m columns: column k + 1 + p (m - p entries) is paired with
    // column jb - 1 - p (p + 1 entries), so every pair holds m + 1 entries and the
    // ceil(m / 2) x (m + 1) pairs spread evenly over the threads (consecutive threads on
    // consecutive rows of one column)
    const int m = jb - k - 1;
    const int np = (m + 1) / 2;
    for (int e = tid; e < np * (m + 1); e += kThreads) {
      const int p = e / (m + 1), q = e - p * (m + 1);
      int c, r;
      if (q < m - p) {
        c = k + 1 + p;
        r = c + q;
      } else {
        c = jb - 1 - p;
        r = c + (q - (m - p));
        if (c == k + 1 + p) continue;  // odd m: the middle column pairs with itself
      }
      zfms_conj(a[c * NB + r], a[k * NB + r], a[k * NB + c]);
    }
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += kThreads) {
    const int r = e % NB, c = e / NB;
    if (r < jb && c < jb && r >= c) S[(size_t)(j0 + r) + (size_t)(j0 + c) * ld] = a[e];
  }
}

// Panel below a factored diagonal block: X <- X L_jj^{-H} for rows [r0, r0 + nrows)
// of columns [j0, j0 + jb), RPR rows per CTA (small CTAs: the panels are narrow, and
// FP64 issues slowly, so the rows are spread over as many SMs as possible).  Column
// c of X L_jj^H = B reads sum_{k <= c} X[r, k] conj(L[c, k]) = B[r, c]: solved left
// to right.
constexpr int RPR = 16;
constexpr int kSmallThreads = 128;
__global__ void __launch_bounds__(kSmallThreads) k_trsm_rpanel(double2* __restrict__ S, int ld,
                                                               int j0, int jb, int r0, int nrows,
                                                               const int* __restrict__ fail) {
  extern __shared__ double2 sm[];
  double2* Lb = sm;            // NB x NB column-major: L[r][c] at c * NB + r
  double2* x = sm + NB * NB;   // RPR rows x NB columns, column-major: x[c * RPR + r]
  if (*fail) return;
  const int tid = threadIdx.x;
  const int rb = r0 + blockIdx.x * RPR;
  const int nr = min(RPR, r0 + nrows - rb);
  for (int e = tid; e < NB * NB; e += kSmallThreads) {
    const int r = e % NB, c = e / NB;
    Lb[e] = (r < jb && c < jb && r >= c) ? S[(size_t)(j0 + r) + (size_t)(j0 + c) * ld]
                                         : make_double2(0.0, 0.0);
  }
  for (int e = tid; e < RPR * NB; e += kSmallThreads) {
    const int r = e % RPR, c = e / RPR;
    x[e] = (r < nr && c < jb) ? S[(size_t)(rb + r) + (size_t)(j0 + c) * ld]
                              : make_double2(0.0, 0.0);
  }
  // the diagonal's reciprocals up front, in parallel, off the column chain
  __shared__ double rdiag[NB];
  for (int c = tid; c < jb; c += kSmallThreads)
    rdiag[c] = 1.0 / S[(size_t)(j0 + c) + (size_t)(j0 + c) * ld].x;
  for (int c = 0; c < jb; ++c) {
    __syncthreads();
    if (tid < RPR) {
      const double rl = rdiag[c];
      x[c * RPR + tid].x *= rl;
      x[c * RPR + tid].y *= rl;
    }
    __syncthreads();
    const int m = jb - c - 1;
    for (int e = tid; e < RPR * m; e += kSmallThreads) {
      const int r = e % RPR, cc = c + 1 + e / RPR;
      zfms_conj(x[cc * RPR + r], x[c * RPR + r], Lb[c * NB + cc]);
    }
  }
  __syncthreads();
  for (int e = tid; e < RPR * NB; e += kSmallThreads) {
    const int r = e % RPR, c = e / RPR;
    if (r < nr && c < jb) S[(size_t)(rb + r) + (size_t)(j0 + c) * ld] = x[e];
  }
}

// Block row of a forward substitution: X <- L_ii^{-1} X for rows [i0, i0 + ib) and
// columns [0, ncols) of X, RPR columns per CTA; L_ii = L[i0 : i0 + ib, i0 : i0 + ib]
// (lower triangle read).
__global__ void __launch_bounds__(kSmallThreads) k_trsm_ldiag(const double2* __restrict__ L,
                                                              int ldl, int i0, int ib,
                                                              double2* __restrict__ X, int ldx,
                                                              int ncols,
                                                              const int* __restrict__ fail) {
  extern __shared__ double2 sm[];
  double2* Lb = sm;            // NB x NB column-major
  double2* x = sm + NB * NB;   // NB rows x RPR columns, row stride RPR + 1
  constexpr int XS = RPR + 1;
  if (*fail) return;
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * RPR;
  const int nc = min(RPR, ncols - c0);
  for (int e = tid; e < NB * NB; e += kSmallThreads) {
    const int r = e % NB, c = e / NB;
    Lb[e] = (r < ib && c < ib && r >= c) ? L[(size_t)(i0 + r) + (size_t)(i0 + c) * ldl]
                                         : make_double2(0.0, 0.0);
  }
  for (int e = tid; e < NB * RPR; e += kSmallThreads) {
    const int r = e % NB, col = e / NB;
    x[r * XS + col] = (r < ib && col < nc) ? X[(size_t)(i0 + r) + (size_t)(c0 + col) * ldx]
                                           : make_double2(0.0, 0.0);
  }
  // the diagonal's reciprocals up front, in parallel, off the row chain
  __shared__ double rdiag[NB];
  for (int k = tid; k < ib; k += kSmallThreads)
    rdiag[k] = 1.0 / L[(size_t)(i0 + k) + (size_t)(i0 + k) * ldl].x;
  for (int k = 0; k < ib; ++k) {
    __syncthreads();
    if (tid < RPR) {
      const double rl = rdiag[k];
      x[k * XS + tid].x *= rl;
      x[k * XS + tid].y *= rl;
    }
    __syncthreads();
    const int m = ib - k - 1;
    for (int e = tid; e < RPR * m; e += kSmallThreads) {
      const int col = e % RPR, r = k + 1 + e / RPR;
      zfms(x[r * XS + col], Lb[k * NB + r], x[k * XS + col]);
    }
  }
  __syncthreads();
  for (int e = tid; e < NB * RPR; e += kSmallThreads) {
    const int r = e % NB, col = e / NB;
    if (r < ib && col < nc) X[(size_t)(i0 + r) + (size_t)(c0 + col) * ldx] = x[r * XS + col];
  }
}

// ---------------------------------------------------------------------------
// C = alpha op(A) op(B) (+ C when beta): A column-major m x k; op(B) = B (k x n,
// column-major) or B^H (B stored n x k).  64 x 64 output tiles, 256 threads with
// 4 x 4 complex results each.  Structure flags bound the K range of every tile:
//   lower  skip tiles strictly above the diagonal (tile column > tile row);
//   triA   A lower triangular: k < end of the tile's rows;
//   triB   op(B) upper triangular: k < end of the tile's columns;
//   halfB  op(B) = tril_h(B): k >= the tile's first column, B[j][j] -> Re(B[j][j]) / 2,
//          entries above the diagonal read as zero.
// Tiles are issued heaviest first (reverse order) to shorten the last wave.
struct ZgemmArgs {
  const double2* A;
  const double2* B;
  double2* C;
  int lda, ldb, ldc;
  int m, n, k;
  double alpha;
  int beta, conjB, lower, triA, triB, halfB;
  const int* fail;
};

// TS x TS output tiles (TS = 64 or 32), 256 threads with (TS/16) x (TS/16) complex
// results each.  GB300 runs FP64 at 2 operations per clock per SM, so a tile's time is
// its FP64 work on one SM: skinny products (the updates inside a Cholesky panel, a
// few dozen 64-wide tiles) take the 32-wide tiles, which spread the same work over
// four times as many SMs.
template <int TS>
__global__ void __launch_bounds__(kThreads, 2) k_zgemm(const ZgemmArgs g) {
  constexpr int RP = TS / 16;  // results per thread along rows and along columns
  __shared__ double2 As[RK][TS];
  __shared__ double2 Bs[RK][TS + 1];
  if (*g.fail) return;
  const int ti = gridDim.y - 1 - blockIdx.y, tj = gridDim.x - 1 - blockIdx.x;
  if (g.lower && tj > ti) return;
  const int r0 = ti * TS, c0 = tj * TS;
  int kb = 0, ke = g.k;
  if (g.triA) ke = min(ke, r0 + TS);
  if (g.triB) ke = min(ke, c0 + TS);
  if (g.halfB) kb = c0;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double2 acc[RP][RP];
#pragma unroll
  for (int i = 0; i < RP; ++i)
#pragma unroll
    for (int j = 0; j < RP; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = kb; k0 < ke; k0 += RK) {
#pragma unroll
    for (int q = 0; q < RP; ++q) {  // RK x TS = 256 RP elements per operand
      const int e = tid + kThreads * q;
      {  // A: TS rows x 16 k, consecutive threads on consecutive rows
        const int rr = e % TS, kk = e / TS;
        const int r = r0 + rr, kx = k0 + kk;
        As[kk][rr] = (r < g.m && kx < ke) ? g.A[(size_t)r + (size_t)kx * g.lda]
                                          : make_double2(0.0, 0.0);
      }
      if (g.conjB) {  // op(B)[k][c] = conj(B[c + k ldb]): consecutive threads on c
        const int cc = e % TS, kk = e / TS;
        const int c = c0 + cc, kx = k0 + kk;
        Bs[kk][cc] = (c < g.n && kx < ke) ? zconj(g.B[(size_t)c + (size_t)kx * g.ldb])
                                          : make_double2(0.0, 0.0);
      } else {  // op(B)[k][c] = B[k + c ldb]: consecutive threads on k
        const int kk = e & 15, cc = e >> 4;
        const int c = c0 + cc, kx = k0 + kk;
        double2 v = (c < g.n && kx < ke) ? g.B[(size_t)kx + (size_t)c * g.ldb]
                                         : make_double2(0.0, 0.0);
        if (g.halfB) {
          if (kx < c) v = make_double2(0.0, 0.0);
          else if (kx == c) v = make_double2(0.5 * v.x, 0.0);
        }
        Bs[kk][cc] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < RK; ++kk) {
      double2 a[RP], b[RP];
#pragma unroll
      for (int i = 0; i < RP; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < RP; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RP; ++i)
#pragma unroll
        for (int j = 0; j < RP; ++j) zfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RP; ++i)
#pragma unroll
    for (int j = 0; j < RP; ++j) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
      if (r < g.m && c < g.n) {
        double2* p = g.C + (size_t)r + (size_t)c * g.ldc;
        double2 v = make_double2(g.alpha * acc[i][j].x, g.alpha * acc[i][j].y);
        if (g.beta) {
          const double2 o = *p;
          v.x += o.x;
          v.y += o.y;
        }
        *p = v;
      }
    }
}

// ---------------------------------------------------------------------------
// W = I (n x n, leading dimension n).
__global__ void k_eye(double2* __restrict__ W, int n, const int* __restrict__ fail) {
  if (*fail) return;
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e % n, c = e / n;
    W[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
}

// Zero the strict upper triangle of the factor (S's storage after the Cholesky).
__global__ void k_zero_upper(double2* __restrict__ S, int n, int ld, const int* __restrict__ fail) {
  if (*fail) return;
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e % n, c = e / n;
    if (r < c) S[r + c * (size_t)ld] = make_double2(0.0, 0.0);
  }
}

// In place: C = G + G^H over the full matrix, diagonal exactly real.  One CTA per
// 32 x 32 block pair (bi >= bj): both blocks are read before either is written.
__global__ void k_hermsum(double2* __restrict__ C, int n, int ld, const int* __restrict__ fail) {
  __shared__ double2 lo[32][33], up[32][33];
  if (*fail) return;
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bi < bj) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int i = bi * 32 + tx, j = bj * 32 + k;  // lo[k][tx] = G(i, j)
    lo[k][tx] = (i < n && j < n) ? C[i + (size_t)j * ld] : make_double2(0.0, 0.0);
    const int i2 = bj * 32 + tx, j2 = bi * 32 + k;  // up[k][tx] = G(i2, j2), i2 in bj, j2 in bi
    up[k][tx] = (i2 < n && j2 < n) ? C[i2 + (size_t)j2 * ld] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  // lower block: C(i, j) = G(i, j) + conj(G(j, i)), i in bi, j in bj
  for (int k = ty; k < 32; k += 8) {
    const int i = bi * 32 + tx, j = bj * 32 + k;
    if (i < n && j < n) {
      const double2 g = lo[k][tx], h = up[tx][k];  // h = G(j, i)
      C[i + (size_t)j * ld] =
          (i == j) ? make_double2(g.x + h.x, 0.0) : make_double2(g.x + h.x, g.y - h.y);
    }
  }
  if (bi == bj) return;  // the diagonal block was written whole above
  // upper block: C(j, i) = conj(C(i, j)), j in bj (rows), i in bi (columns)
  for (int k = ty; k < 32; k += 8) {
    const int jr = bj * 32 + tx, ic = bi * 32 + k;  // element (jr, ic): G(jr, ic) + conj(G(ic, jr))
    if (jr < n && ic < n) {
      const double2 g = up[k][tx], h = lo[tx][k];  // g = G(jr, ic), h = G(ic, jr)
      C[jr + (size_t)ic * ld] = make_double2(g.x + h.x, g.y - h.y);
    }
  }
}

// B = A^H: A is rows x cols (leading dimension lda), B cols x rows (ldb); 32 x 32
// blocks through shared memory.
__global__ void k_ctrans(const double2* __restrict__ A, int lda, int rows, int cols,
                         double2* __restrict__ B, int ldb) {
  __shared__ double2 t[32][33];
  const int bx = blockIdx.x, by = blockIdx.y;    // source block: rows by, columns bx
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int i = by * 32 + tx, j = bx * 32 + k;  // t[k][tx] = A(i, j)
    t[k][tx] = (i < rows && j < cols) ? A[i + (size_t)j * lda] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int i = bx * 32 + tx, j = by * 32 + k;  // B(i, j) = conj(A(j, i)) = conj(t[tx][k])
    if (i < cols && j < rows) B[i + (size_t)j * ldb] = zconj(t[tx][k]);
  }
}

// C -= T over m x nc (lower: only r >= c), both column-major.
__global__ void k_sub(double2* __restrict__ C, int ldc, const double2* __restrict__ T, int ldt,
                      int m, int nc, int lower, const int* __restrict__ fail) {
  if (*fail) return;
  const size_t total = (size_t)m * nc;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    if (lower && r < c) continue;
    double2* p = C + r + (size_t)c * ldc;
    const double2 t = T[r + (size_t)c * ldt];
    *p = make_double2(p->x - t.x, p->y - t.y);
  }
}

// 64-wide tiles unless that leaves most SMs idle: fewer than two 64-wide tiles per SM
// take 32-wide tiles.  The choice depends on m and n only, never on the structure
// flags: P = W tril_h(H) writes only tiles on or below the diagonal and
// G = P W^H (triA) reads P up to the end of each tile's rows, so both products of one
// n must tile alike.
cudaError_t zgemm(const ZgemmArgs& g, cudaStream_t st) {
  if (g.m <= 0 || g.n <= 0) return cudaSuccess;
  const long long t64 = (long long)((g.n + 63) / 64) * ((g.m + 63) / 64);
  if (t64 < 2 * kNumSMs) {
    const dim3 grid((g.n + 31) / 32, (g.m + 31) / 32);
    k_zgemm<32><<<grid, kThreads, 0, st>>>(g);
  } else {
    const dim3 grid((g.n + 63) / 64, (g.m + 63) / 64);
    k_zgemm<64><<<grid, kThreads, 0, st>>>(g);
  }
  return cudaGetLastError();
}

ZgemmArgs zargs(const double2* A, int lda, const double2* B, int ldb, double2* C, int ldc, int m,
                int n, int k, double alpha, int beta, const int* fail) {
  ZgemmArgs g{};
  g.A = A;
  g.B = B;
  g.C = C;
  g.lda = lda;
  g.ldb = ldb;
  g.ldc = ldc;
  g.m = m;
  g.n = n;
  g.k = k;
  g.alpha = alpha;
  g.beta = beta;
  g.fail = fail;
  return g;
}

constexpr size_t kDiagSmem = (size_t)NB * NB * sizeof(double2);                 // 64 KB
constexpr size_t kPanelSmem = kDiagSmem + (size_t)RPR * NB * sizeof(double2);        // 80 KB
constexpr size_t kLdiagSmem = kDiagSmem + (size_t)NB * (RPR + 1) * sizeof(double2);  // 81 KB

cudaError_t set_smem() {
  static cudaError_t once = []() {
    cudaError_t e = cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDiagSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_trsm_rpanel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kPanelSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_trsm_ldiag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kLdiagSmem);
    return e;
  }();
  return once;
}

}  // namespace

static int grid_for(size_t total) {
  const size_t b = (total + kThreads - 1) / kThreads;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// FP64 factorisation of the panel S[j0 :, j0 : j0 + pw) in 64-column blocks; each
// block's trailing update stays inside the panel (the caller updates the rest).
cudaError_t hs_launch_cholesky_panel(double2* S, int n, int j0, int pw, int* fail,
                                     cudaStream_t st) {
  cudaError_t e = set_smem();
  if (e != cudaSuccess) return e;
  for (int jj = j0; jj < j0 + pw; jj += NB) {
    const int jb = j0 + pw - jj < NB ? j0 + pw - jj : NB;
    k_potrf_diag<<<1, kThreads, kDiagSmem, st>>>(S, n, jj, jb, fail);
    const int r0 = jj + jb, rest = n - r0;
    if (rest > 0) {
      k_trsm_rpanel<<<(rest + RPR - 1) / RPR, kSmallThreads, kPanelSmem, st>>>(S, n, jj, jb, r0,
                                                                               rest, fail);
      const int ncol = j0 + pw - r0;  // panel columns right of this block
      if (ncol > 0) {
        // S[r0 :, r0 : j0 + pw) lower tiles -= L21 L21^H (rows r0.. x the first ncol of them)
        const double2* L21 = S + (size_t)r0 + (size_t)jj * n;
        ZgemmArgs g = zargs(L21, n, L21, n, S + (size_t)r0 + (size_t)r0 * n, n, rest, ncol, jb,
                            -1.0, 1, fail);
        g.conjB = 1;
        g.lower = 1;
        e = zgemm(g, st);
        if (e != cudaSuccess) return e;
      }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t hs_launch_zero_upper(double2* S, int n, const int* fail, cudaStream_t st) {
  k_zero_upper<<<grid_for((size_t)n * n), kThreads, 0, st>>>(S, n, n, fail);
  return cudaGetLastError();
}

// S <- L (lower; strict upper zeroed), blocked right-looking: one panel of width n.
cudaError_t hs_launch_cholesky(double2* S, int n, int* fail, cudaStream_t st) {
  cudaError_t e = hs_launch_cholesky_panel(S, n, 0, n, fail, st);
  if (e != cudaSuccess) return e;
  return hs_launch_zero_upper(S, n, fail, st);
}

cudaError_t hs_launch_eye(double2* W, int n, const int* fail, cudaStream_t st) {
  k_eye<<<grid_for((size_t)n * n), kThreads, 0, st>>>(W, n, fail);
  return cudaGetLastError();
}

// FP64 block row [i0, i0 + pw) of the forward substitution L W = I, in 64-row blocks:
// block ii's solution has nonzero columns [0, ii + ib); its update of the rows below
// stays inside the block row (the caller updates the rest).
cudaError_t hs_launch_inverse_blockrow(const double2* L, double2* W, int n, int i0, int pw,
                                       const int* fail, cudaStream_t st) {
  cudaError_t e = set_smem();
  if (e != cudaSuccess) return e;
  for (int ii = i0; ii < i0 + pw; ii += NB) {
    const int ib = i0 + pw - ii < NB ? i0 + pw - ii : NB;
    const int ncols = ii + ib;
    k_trsm_ldiag<<<(ncols + RPR - 1) / RPR, kSmallThreads, kLdiagSmem, st>>>(L, n, ii, ib, W, n,
                                                                             ncols, fail);
    const int r0 = ii + ib, rest = i0 + pw - r0;
    if (rest > 0) {
      // W[r0 : i0 + pw, 0 : ncols] -= L[r0 :, ii : ii + ib] W[ii : ii + ib, 0 : ncols]
      ZgemmArgs g = zargs(L + (size_t)r0 + (size_t)ii * n, n, W + (size_t)ii, n, W + (size_t)r0,
                          n, rest, ncols, ib, -1.0, 1, fail);
      e = zgemm(g, st);
      if (e != cudaSuccess) return e;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// W <- L^{-1} (lower triangular; L = the factor in S): one block row of height n.
cudaError_t hs_launch_tri_inverse(const double2* L, double2* W, int n, const int* fail,
                                  cudaStream_t st) {
  cudaError_t e = hs_launch_eye(W, n, fail, st);
  if (e != cudaSuccess) return e;
  return hs_launch_inverse_blockrow(L, W, n, 0, n, fail, st);
}

// P <- W tril_h(H) (lower triangular; only tiles on or below the diagonal are written).
cudaError_t hs_launch_reduce_p(const double2* W, const double2* H, double2* P, int n,
                               const int* fail, cudaStream_t st) {
  ZgemmArgs g = zargs(W, n, H, n, P, n, n, n, n, 1.0, 0, fail);
  g.lower = 1;
  g.triA = 1;
  g.halfB = 1;
  return zgemm(g, st);
}

// G <- P W^H (full), written over H; then H <- G + G^H.
cudaError_t hs_launch_reduce_g(const double2* P, const double2* W, double2* H, int n,
                               const int* fail, cudaStream_t st) {
  ZgemmArgs g = zargs(P, n, W, n, H, n, n, n, n, 1.0, 0, fail);
  g.conjB = 1;
  g.triA = 1;
  g.triB = 1;
  return zgemm(g, st);
}

cudaError_t hs_launch_ctrans(const double2* A, int lda, int rows, int cols, double2* B, int ldb,
                            cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  k_ctrans<<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, st>>>(A, lda, rows, cols,
                                                                              B, ldb);
  return cudaGetLastError();
}

cudaError_t hs_launch_sub(double2* C, int ldc, const double2* T, int ldt, int m, int nc, int lower,
                          const int* fail, cudaStream_t st) {
  if (m <= 0 || nc <= 0) return cudaSuccess;
  k_sub<<<grid_for((size_t)m * nc), kThreads, 0, st>>>(C, ldc, T, ldt, m, nc, lower, fail);
  return cudaGetLastError();
}

cudaError_t hs_launch_hermsum(double2* H, int n, const int* fail, cudaStream_t st) {
  const int nb = (n + 31) / 32;
  k_hermsum<<<dim3(nb, nb), dim3(32, 8), 0, st>>>(H, n, n, fail);
  return cudaGetLastError();
}
