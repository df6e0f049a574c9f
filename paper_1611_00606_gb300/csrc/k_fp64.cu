// FP64 kernels: per-atom products (Algorithm 1 loops), the stacked Hermitian
// contractions of the plain FP64 form, and the final mirror.
//
// GB300 runs FP64 on the CUDA cores only (tcgen05 has no FP64 kind), so these
// kernels are bound by the FP64 pipe; smem tiles keep global traffic small.
#include "hs_internal.h"

namespace {

__device__ __forceinline__ void cfma_conj(double2& acc, double2 l, double2 r) {
  // acc += conj(l) * r
  acc.x = fma(l.x, r.x, acc.x);
  acc.x = fma(l.y, r.y, acc.x);
  acc.y = fma(l.x, r.y, acc.y);
  acc.y = fma(-l.y, r.x, acc.y);
}
__device__ __forceinline__ void cfma(double2& acc, double2 m, double2 x) {
  // acc += m * x
  acc.x = fma(m.x, x.x, acc.x);
  acc.x = fma(-m.y, x.y, acc.x);
  acc.y = fma(m.x, x.y, acc.y);
  acc.y = fma(m.y, x.x, acc.y);
}

// ---------------------------------------------------------------------------
// Per-atom products.  blockIdx.z = 2*a + job.
//   job 0:  Z[a*N_L + r, g]       = sum_k MZ[a](r, k) [A_a; B_a](k, g)      (k < 2N_L)
//   job 1:  W2[slot[a]*N_L + r, g] = sum_k M2[a](r, k) A_a(k, g)            (k < N_L)
// M2[a] is upper triangular when fail[a] == 0 (L^H): K tiles left of the
// diagonal block are skipped.  CTA tile: 32 rows x 64 columns, K step 16.
constexpr int AT_R = 32, AT_C = 64, AT_K = 16;

__global__ void __launch_bounds__(256) k_atoms(const double2* __restrict__ MZ,
                                               const double2* __restrict__ M2,
                                               const int* __restrict__ fail,
                                               const int* __restrict__ slot,
                                               const double2* __restrict__ A,
                                               const double2* __restrict__ B, int ldAB,
                                               double2* __restrict__ Z, double2* __restrict__ W2,
                                               int ldW, int N_L, int N_G) {
  __shared__ double2 Ms[AT_K][AT_R + 1];
  __shared__ double2 Xs[AT_K][AT_C + 1];
  const int a = blockIdx.z >> 1, job = blockIdx.z & 1;
  const int r0 = blockIdx.y * AT_R, g0 = blockIdx.x * AT_C;
  const int tid = threadIdx.x;
  const double2* M;
  int Kb, ldM = N_L, kstart = 0;
  double2* C;
  if (job == 0) {
    M = MZ + (size_t)a * 2 * N_L * N_L;
    Kb = 2 * N_L;
    C = Z + (size_t)a * N_L;
  } else {
    M = M2 + (size_t)a * N_L * N_L;
    Kb = N_L;
    C = W2 + (size_t)slot[a] * N_L;
    if (fail[a] == 0) kstart = (r0 / AT_K) * AT_K;  // L^H is upper triangular
  }
  const double2* X0 = A + (size_t)a * N_L;
  const double2* X1 = B + (size_t)a * N_L;

  // thread -> outputs: rows tr, tr+16 ; cols tc + 16*c (c < 4)
  const int tr = tid >> 4, tc = tid & 15;
  double2 acc[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = kstart; k0 < Kb; k0 += AT_K) {
    // M tile: AT_R x AT_K, column-major source (rows contiguous)
    for (int idx = tid; idx < AT_R * AT_K; idx += 256) {
      const int rr = idx % AT_R, kk = idx / AT_R;
      const int r = r0 + rr, k = k0 + kk;
      Ms[kk][rr] = (r < N_L && k < Kb) ? M[r + (size_t)k * ldM] : make_double2(0.0, 0.0);
    }
    // X tile: AT_K x AT_C, column g contiguous in k
    for (int idx = tid; idx < AT_K * AT_C; idx += 256) {
      const int kk = idx % AT_K, cc = idx / AT_K;
      const int k = k0 + kk, g = g0 + cc;
      double2 v = make_double2(0.0, 0.0);
      if (g < N_G && k < Kb) {
        v = (k < N_L) ? X0[k + (size_t)g * ldAB] : X1[(k - N_L) + (size_t)g * ldAB];
      }
      Xs[kk][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < AT_K; ++kk) {
      const double2 m0 = Ms[kk][tr], m1 = Ms[kk][tr + 16];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const double2 x = Xs[kk][tc + 16 * j];
        cfma(acc[0][j], m0, x);
        cfma(acc[1][j], m1, x);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int r = r0 + tr + 16 * i;
    if (r >= N_L) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int g = g0 + tc + 16 * j;
      if (g < N_G) C[r + (size_t)g * ldW] = acc[i][j];
    }
  }
}

__global__ void k_gather_af(const double2* __restrict__ A, int ldA,
                            const int* __restrict__ fail_list, int N_L, int N_G,
                            double2* __restrict__ AF, int ldAF) {
  const int f = blockIdx.y;
  const int a = fail_list[f];
  for (int g = blockIdx.x; g < N_G; g += gridDim.x)
    for (int r = threadIdx.x; r < N_L; r += blockDim.x)
      AF[(size_t)f * N_L + r + (size_t)g * ldAF] = A[(size_t)a * N_L + r + (size_t)g * ldA];
}

// ---------------------------------------------------------------------------
// FP64 stacked contraction, lower-triangle tiles only:
//   C(i, j) = sum_seg sum_k conj(L(k, i)) u(k)^2 R(k, j)
// Tile 64 x 64 complex, 256 threads (4 x 4 outputs each), K step 16.
constexpr int CT = 64, CK = 16;

__device__ __forceinline__ void tri_index(int t, int& bi, int& bj) {
  int b = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((b + 1) * (b + 2) / 2 <= t) ++b;
  while (b * (b + 1) / 2 > t) --b;
  bi = b;
  bj = t - b * (b + 1) / 2;
}

__global__ void __launch_bounds__(256) k_contract_fp64(SegList segs, double2* __restrict__ C,
                                                       int N_G, int ldC) {
  __shared__ double2 Ls[CK][CT + 1];
  __shared__ double2 Rs[CK][CT + 1];
  int bi, bj;
  tri_index(blockIdx.x, bi, bj);
  const int i0 = bi * CT, j0 = bj * CT;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  double2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_double2(0.0, 0.0);

  for (int s = 0; s < segs.n; ++s) {
    const Seg sg = segs.s[s];
    for (int k0 = 0; k0 < sg.K; k0 += CK) {
      for (int idx = tid; idx < CK * CT; idx += 256) {
        const int kk = idx % CK, cc = idx / CK;
        const int k = k0 + kk;
        double2 l = make_double2(0.0, 0.0), r = make_double2(0.0, 0.0);
        if (k < sg.K) {
          if (i0 + cc < N_G) {
            l = sg.L[k + (size_t)(i0 + cc) * sg.ldL];
            if (sg.u) {
              const double w = sg.u[k] * sg.u[k];
              l.x *= w;
              l.y *= w;
            }
          }
          if (j0 + cc < N_G) r = sg.R[k + (size_t)(j0 + cc) * sg.ldR];
        }
        Ls[kk][cc] = l;
        Rs[kk][cc] = r;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < CK; ++kk) {
        double2 lv[4], rv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) lv[r] = Ls[kk][ty + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) rv[c] = Rs[kk][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) cfma_conj(acc[r][c], lv[r], rv[c]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 16 * r;
    if (i >= N_G) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx + 16 * c;
      if (j < N_G) C[i + (size_t)j * ldC] = acc[r][c];
    }
  }
}

// Upper triangle := conj(lower); Im(diag) := 0.  32 x 32 blocks via smem.
__global__ void k_mirror(double2* __restrict__ C, int N, int ld) {
  __shared__ double2 t[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;  // source block (rows bi, cols bj), bi >= bj
  if (bi < bj) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int i = bi * 32 + tx, j = bj * 32 + k;
    t[k][tx] = (i < N && j < N) ? C[i + (size_t)j * ld] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  // destination (row j, col i) for source (i, j) with i > j
  for (int k = ty; k < 32; k += 8) {
    const int j = bj * 32 + tx, i = bi * 32 + k;  // dest element C(j, i)
    if (i < N && j < N) {
      const double2 v = t[tx][k];  // source C(i, j)
      if (i > j) {
        C[j + (size_t)i * ld] = make_double2(v.x, -v.y);
      } else if (i == j) {
        C[j + (size_t)i * ld] = make_double2(v.x, 0.0);
      }
    }
  }
}

}  // namespace

cudaError_t hs_launch_atoms_fp64(const double2* MZ, const double2* M2, const int* fail,
                                 const int* slot, const double2* A, const double2* B,
                                 int ldAB, double2* Z, double2* W2, int ldW, int N_A,
                                 int N_L, int N_G, cudaStream_t st) {
  dim3 grid((N_G + AT_C - 1) / AT_C, (N_L + AT_R - 1) / AT_R, 2 * N_A);
  k_atoms<<<grid, 256, 0, st>>>(MZ, M2, fail, slot, A, B, ldAB, Z, W2, ldW, N_L, N_G);
  return cudaGetLastError();
}

cudaError_t hs_launch_gather_af(const double2* A, int ldA, const int* fail_list, int N_f,
                                int N_L, int N_G, double2* AF, cudaStream_t st) {
  if (N_f == 0) return cudaSuccess;
  dim3 grid(N_G < 1024 ? N_G : 1024, N_f);
  k_gather_af<<<grid, 128, 0, st>>>(A, ldA, fail_list, N_L, N_G, AF, N_f * N_L);
  return cudaGetLastError();
}

cudaError_t hs_launch_contract_fp64(const SegList& segs, double2* C, int N_G, int ldC,
                                    cudaStream_t st) {
  const int nb = (N_G + CT - 1) / CT;
  const int tiles = nb * (nb + 1) / 2;
  k_contract_fp64<<<tiles, 256, 0, st>>>(segs, C, N_G, ldC);
  return cudaGetLastError();
}

cudaError_t hs_launch_mirror(double2* C, int N_G, int ldC, cudaStream_t st) {
  const int nb = (N_G + 31) / 32;
  k_mirror<<<dim3(nb, nb), dim3(32, 8), 0, st>>>(C, N_G, ldC);
  return cudaGetLastError();
}
