// Factor step of H_AA (Algorithm 1, second part of H, "try Cholesky"):
// batched FP64 Cholesky of every T^AA_a with the failure test, plus the
// per-atom operators used by the per-k-point products.  T does not depend on
// the k-point, so the plan runs this once and caches the result.
#include "hs_internal.h"

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// Start of column c in the packed (column-major) lower triangle of an n x n matrix.
__device__ __forceinline__ int col0(int c, int n) { return c * n - (c * (c - 1)) / 2; }

// One CTA factorises T^AA_a = L L^H (L lower, real positive diagonal) in
// shared memory, right-looking, column by column.  The failure test is the
// zpotrf one: the pivot Re(T_jj) - sum_k |L_jk|^2 must be > 0 (NaN fails).
// Output: fail[a]; M2[a] = L^H (upper triangular) on success, else the full
// Hermitian T^AA_a rebuilt from its lower triangle (fallback operator).
__global__ void __launch_bounds__(256) k_cholesky(const double2* __restrict__ T_AA, int N,
                                                  double2* __restrict__ M2,
                                                  int* __restrict__ fail) {
  extern __shared__ double2 P[];
  __shared__ int s_fail;
  __shared__ double s_inv;
  const int a = blockIdx.x;
  const double2* T = T_AA + (size_t)a * N * N;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  for (int c = 0; c < N; ++c)
    for (int r = c + tid; r < N; r += nt) P[col0(c, N) + (r - c)] = T[r + (size_t)c * N];
  if (tid == 0) s_fail = 0;
  __syncthreads();

  for (int j = 0; j < N; ++j) {
    if (tid == 0) {
      const double d = P[col0(j, N)].x;
      if (!(d > 0.0)) {
        s_fail = 1;
      } else {
        const double l = sqrt(d);
        P[col0(j, N)] = make_double2(l, 0.0);
        s_inv = 1.0 / l;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const double inv = s_inv;
    const int cj = col0(j, N);
    for (int r = j + 1 + tid; r < N; r += nt) {
      double2 v = P[cj + (r - j)];
      P[cj + (r - j)] = make_double2(v.x * inv, v.y * inv);
    }
    __syncthreads();
    // trailing update  P(r,c) -= L(r,j) conj(L(c,j)),  c > j, r >= c
    for (int c = j + 1 + warp; c < N; c += nw) {
      const double2 lcj = cconj(P[cj + (c - j)]);
      const int cc = col0(c, N);
      for (int r = c + lane; r < N; r += 32) {
        const double2 t = cmul(P[cj + (r - j)], lcj);
        double2 v = P[cc + (r - c)];
        v.x -= t.x;
        v.y -= t.y;
        P[cc + (r - c)] = v;
      }
    }
    __syncthreads();
  }

  double2* M = M2 + (size_t)a * N * N;
  if (!s_fail) {
    for (int idx = tid; idx < N * N; idx += nt) {
      const int r = idx % N, c = idx / N;
      M[idx] = (c >= r) ? cconj(P[col0(r, N) + (c - r)]) : make_double2(0.0, 0.0);
    }
  } else {
    for (int idx = tid; idx < N * N; idx += nt) {
      const int r = idx % N, c = idx / N;
      M[idx] = (r >= c) ? T[r + (size_t)c * N] : cconj(T[c + (size_t)r * N]);
    }
  }
  if (tid == 0) fail[a] = s_fail;
}

// MZ[a] = [T^BA_a | 1/2 T^BB_a] with T^BA = (T^AB)^H (Sec. 2) and T^BB the
// Hermitian matrix rebuilt from its lower triangle.  N x 2N column-major.
__global__ void k_prep_mz(const double2* __restrict__ T_AB, const double2* __restrict__ T_BB,
                          int N_A, int N, double2* __restrict__ MZ) {
  const size_t per = (size_t)2 * N * N;
  const size_t total = per * N_A;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / per);
    const int rem = (int)(idx % per);
    const int r = rem % N, c = rem / N;
    const double2* tab = T_AB + (size_t)a * N * N;
    const double2* tbb = T_BB + (size_t)a * N * N;
    double2 v;
    if (c < N) {
      v = cconj(tab[c + (size_t)r * N]);
    } else {
      const int cb = c - N;
      const double2 t = (r >= cb) ? tbb[r + (size_t)cb * N] : cconj(tbb[cb + (size_t)r * N]);
      v = make_double2(0.5 * t.x, 0.5 * t.y);
    }
    MZ[idx] = v;
  }
}

}  // namespace

cudaError_t hs_launch_factor(const double2* T_AA, const double2* T_AB, const double2* T_BB,
                             int N_A, int N_L, double2* M2, double2* MZ, int* fail,
                             cudaStream_t st) {
  const size_t smem = (size_t)N_L * (N_L + 1) / 2 * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_cholesky<<<N_A, 256, smem, st>>>(T_AA, N_L, M2, fail);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t total = (size_t)2 * N_L * N_L * N_A;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_prep_mz<<<blocks, 256, 0, st>>>(T_AB, T_BB, N_A, N_L, MZ);
  return cudaGetLastError();
}
