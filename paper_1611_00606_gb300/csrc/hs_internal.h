// Internal declarations shared by the libhs translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hs.h"

#define HS_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) { hs_last_cuda_error(e_); return HS_ECUDA; } \
  } while (0)

void hs_last_cuda_error(cudaError_t e);

// One K-segment of a stacked Hermitian contraction:  C += L^H diag(u^2) R,
// L and R column-major complex with K rows; u (optional, real, length K)
// scales both sides (the U_a norms of Eq. (s)).
struct Seg {
  const double2* L;
  const double2* R;
  const double* u;
  int ldL, ldR, K;
};
constexpr int kMaxSeg = 4;
struct SegList {
  Seg s[kMaxSeg];
  int n;
};

// ---- factor step (k_factor.cu) ---------------------------------------------
// Batched FP64 Cholesky of the lower triangle of T_AA[a] (one CTA per atom).
// fail[a] = 1 when a pivot is not > 0; M2[a] = L_a^H (upper) or the full
// Hermitian T_AA[a] on failure.  MZ[a] = [T_AB[a]^H | 1/2 T_BB[a]] (N_L x 2N_L).
cudaError_t hs_launch_factor(const double2* T_AA, const double2* T_AB, const double2* T_BB,
                             int N_A, int N_L, double2* M2, double2* MZ, int* fail,
                             cudaStream_t st);

// ---- FP64 kernels (k_fp64.cu) ------------------------------------------------
// Per-atom products of one k-point (both FP64 and split plans):
//   Z[a rows]         = MZ[a] [A_a; B_a]
//   W2[slot[a] rows]  = M2[a] A_a        (M2 upper triangular when fail[a] == 0)
// A, B, Z, W2 have leading dimension ld (= K).
cudaError_t hs_launch_atoms_fp64(const double2* MZ, const double2* M2, const int* fail,
                                 const int* slot, const double2* A, const double2* B,
                                 int ldAB, double2* Z, double2* W2, int ldW, int N_A,
                                 int N_L, int N_G, cudaStream_t st);
// AF rows f*N_L.. = A rows fail_list[f]*N_L.. (stack A_a of failing atoms).
cudaError_t hs_launch_gather_af(const double2* A, int ldA, const int* fail_list, int N_f,
                                int N_L, int N_G, double2* AF, cudaStream_t st);
// Lower-triangle tiles of C = sum_seg L^H diag(u^2) R, FP64 (C column-major, ld ldC).
cudaError_t hs_launch_contract_fp64(const SegList& segs, double2* C, int N_G, int ldC,
                                    cudaStream_t st);
// Upper triangle := conj(lower), Im(diag) := 0.
cudaError_t hs_launch_mirror(double2* C, int N_G, int ldC, cudaStream_t st);

// ---- generalized-eigenproblem reduction (k_reduce.cu) --------------------------
// All n x n column-major with leading dimension n; *fail is the failure word (0 =
// positive definite so far); every kernel does nothing once it is set.
// S <- L (Cholesky, strict upper zeroed); *fail = failing column (1-based).
cudaError_t hs_launch_cholesky(double2* S, int n, int* fail, cudaStream_t st);
// W <- L^{-1}.
cudaError_t hs_launch_tri_inverse(const double2* L, double2* W, int n, const int* fail,
                                  cudaStream_t st);
// P <- W tril_h(H) (lower triangle of H, diagonal halved).
cudaError_t hs_launch_reduce_p(const double2* W, const double2* H, double2* P, int n,
                               const int* fail, cudaStream_t st);
// H <- P W^H (full).
cudaError_t hs_launch_reduce_g(const double2* P, const double2* W, double2* H, int n,
                               const int* fail, cudaStream_t st);
// H <- H + H^H (diagonal exactly real).
cudaError_t hs_launch_hermsum(double2* H, int n, const int* fail, cudaStream_t st);
// B (cols x rows, ldb) <- A^H (A rows x cols, lda).
cudaError_t hs_launch_ctrans(const double2* A, int lda, int rows, int cols, double2* B, int ldb,
                            cudaStream_t st);
// C -= T over m x nc (lower != 0: only r >= c).
cudaError_t hs_launch_sub(double2* C, int ldc, const double2* T, int ldt, int m, int nc, int lower,
                          const int* fail, cudaStream_t st);
// Pieces of the blocked Cholesky and inverse (the split form updates the trailing parts
// on the tensor cores between them): FP64 factorisation of the panel S[j0 :, j0 : j0 + pw)
// with updates inside the panel; strict upper triangle zeroed; W = I; FP64 block row
// [i0, i0 + pw) of L W = I with updates inside the block row.
cudaError_t hs_launch_cholesky_panel(double2* S, int n, int j0, int pw, int* fail,
                                     cudaStream_t st);
cudaError_t hs_launch_zero_upper(double2* S, int n, const int* fail, cudaStream_t st);
cudaError_t hs_launch_eye(double2* W, int n, const int* fail, cudaStream_t st);
cudaError_t hs_launch_inverse_blockrow(const double2* L, double2* W, int n, int i0, int pw,
                                       const int* fail, cudaStream_t st);

// ---- real-symmetric variant helpers (k_real.cu) --------------------------------
// y[i] = (x[i], 0) for i < n.
cudaError_t hs_launch_embed(const double* x, double2* y, size_t n, cudaStream_t st);
// y(r, c) = (x(r, c), 0), r < rows, c < cols, column-major.
cudaError_t hs_launch_embed2d(const double* x, int ldx, double2* y, int ldy, int rows, int cols,
                              cudaStream_t st);
// y = Re(x), n x n column-major.
cudaError_t hs_launch_real_part(const double2* x, int ldx, double* y, int ldy, int n,
                                cudaStream_t st);
// Real A_f gather (as hs_launch_gather_af).
cudaError_t hs_launch_gather_af_real(const double* A, int ldA, const int* fail_list, int N_f,
                                     int N_L, int N_G, double* AF, cudaStream_t st);
// Upper triangle := lower triangle.
cudaError_t hs_launch_mirror_real(double* C, int N_G, int ldC, cudaStream_t st);

// ---- split-precision kernels (k_split.cu) -------------------------------------
struct SliceSeg {
  // slices of one stacked operand segment: s arrays [rows_pad][kpad] bf16,
  // slice p at base + p * slice_stride (elements); row g holds column g.
  const uint16_t* base;
  const int* expo;      // per row (column g of the operand) power-of-two exponent
  int64_t slice_stride;
  int kpad;             // padded real K (multiple of 16)
};
