// Split-precision form of the generalized-eigenproblem reduction (hs_reduce on split
// plans): the slice-path products of the blocked Cholesky, the inverse and the
// two-sided transform.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "split_common.h"

using namespace hs_split;

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
  if (precision != HS_SPLIT_BF16 || n < 1) return HS_EINVAL;  // real plans: complex embedding
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
