// Helpers of the real-symmetric variant (real A, B, T, U; Sec. 1.1 notes that H
// and S are real symmetric for systems with inversion symmetry): embedding of
// real arrays as complex ones (the factorisation and the FP64 form reuse the
// complex kernels, whose imaginary parts then stay exactly zero), the real part
// of a complex result, the real A_f gather and the real symmetric mirror.
#include "hs_internal.h"

namespace {

__global__ void k_embed(const double* __restrict__ x, double2* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = make_double2(x[i], 0.0);
}

// y(r, c) = x(r, c) for r < rows, c < cols (column-major, leading dimensions ldx, ldy)
__global__ void k_embed2d(const double* __restrict__ x, int ldx, double2* __restrict__ y, int ldy,
                          int rows, int cols) {
  for (int c = blockIdx.x; c < cols; c += gridDim.x)
    for (int r = threadIdx.x; r < rows; r += blockDim.x)
      y[r + (size_t)c * ldy] = make_double2(x[r + (size_t)c * ldx], 0.0);
}

__global__ void k_real_part(const double2* __restrict__ x, int ldx, double* __restrict__ y,
                            int ldy, int n) {
  for (int c = blockIdx.x; c < n; c += gridDim.x)
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      y[r + (size_t)c * ldy] = x[r + (size_t)c * ldx].x;
}

__global__ void k_gather_af_real(const double* __restrict__ A, int ldA,
                                 const int* __restrict__ fail_list, int N_L, int N_G,
                                 double* __restrict__ AF, int ldAF) {
  const int f = blockIdx.y;
  const int a = fail_list[f];
  for (int g = blockIdx.x; g < N_G; g += gridDim.x)
    for (int r = threadIdx.x; r < N_L; r += blockDim.x)
      AF[(size_t)f * N_L + r + (size_t)g * ldAF] = A[(size_t)a * N_L + r + (size_t)g * ldA];
}

// Upper triangle := lower triangle (32 x 32 blocks through shared memory).
__global__ void k_mirror_real(double* __restrict__ C, int N, int ld) {
  __shared__ double t[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;  // source block (rows bi, cols bj), bi >= bj
  if (bi < bj) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int i = bi * 32 + tx, j = bj * 32 + k;
    t[k][tx] = (i < N && j < N) ? C[i + (size_t)j * ld] : 0.0;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int j = bj * 32 + tx, i = bi * 32 + k;  // dest element C(j, i) = source C(i, j)
    if (i < N && j < N && i > j) C[j + (size_t)i * ld] = t[tx][k];
  }
}

int grid_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t hs_launch_embed(const double* x, double2* y, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_embed<<<grid_for(n), 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t hs_launch_embed2d(const double* x, int ldx, double2* y, int ldy, int rows, int cols,
                              cudaStream_t st) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  k_embed2d<<<cols < 4096 ? cols : 4096, 256, 0, st>>>(x, ldx, y, ldy, rows, cols);
  return cudaGetLastError();
}

cudaError_t hs_launch_real_part(const double2* x, int ldx, double* y, int ldy, int n,
                                cudaStream_t st) {
  k_real_part<<<n < 4096 ? n : 4096, 256, 0, st>>>(x, ldx, y, ldy, n);
  return cudaGetLastError();
}

cudaError_t hs_launch_gather_af_real(const double* A, int ldA, const int* fail_list, int N_f,
                                     int N_L, int N_G, double* AF, cudaStream_t st) {
  if (N_f == 0) return cudaSuccess;
  dim3 grid(N_G < 1024 ? N_G : 1024, N_f);
  k_gather_af_real<<<grid, 128, 0, st>>>(A, ldA, fail_list, N_L, N_G, AF, N_f * N_L);
  return cudaGetLastError();
}

cudaError_t hs_launch_mirror_real(double* C, int N_G, int ldC, cudaStream_t st) {
  const int nb = (N_G + 31) / 32;
  k_mirror_real<<<dim3(nb, nb), dim3(32, 8), 0, st>>>(C, N_G, ldC);
  return cudaGetLastError();
}
