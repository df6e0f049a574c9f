// hs_assemble_static: the FP64 assembly for small problems without any device
// allocation.
//
// Some callers cannot call cudaMalloc at all: code inside a memory pool or arena
// owned by someone else that forbids side allocations, or hosts whose allocator is
// locked down (for example an embedding that has to keep its device footprint fixed
// after start-up).  hs_plan() allocates its workspace, so those callers cannot use
// it.  This entry point instead keeps the whole per-call workspace (per-atom
// operators, Cholesky flags, Z, [Y; X], the stacked A rows of failing atoms) in one
// statically sized device array that the CUDA runtime reserves when the library is
// loaded.
//
// The array is a file-scope __device__ symbol: in host code its name is only
// a host-side stand-in, not a device address, so the first call on each device
// asks the runtime for the real address with cudaGetSymbolAddress (with that
// device current) and caches it.
#include <cuda_runtime.h>

#include <mutex>

#include "hs_internal.h"

namespace {

// Maximum bytes of per-call workspace (see hs.h for the size formula).
constexpr size_t kStaticScratchBytes = (size_t)HS_STATIC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// Address of g_scratch on the current device (set up once per device).
cudaError_t scratch_ptr(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Slot map from the Cholesky flags, on the device: HPD atoms first (rows of Y),
// then failing atoms (rows of X); counts[0] = number of failing atoms.
__global__ void k_slots(const int* __restrict__ fail, int N_A, int* __restrict__ slot,
                        int* __restrict__ fail_list, int* __restrict__ counts) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int nh = 0;
  for (int a = 0; a < N_A; ++a)
    if (!fail[a]) slot[a] = nh++;
  int nf = 0;
  for (int a = 0; a < N_A; ++a)
    if (fail[a]) {
      slot[a] = nh + nf;
      fail_list[nf++] = a;
    }
  counts[0] = nf;
}

// Bytes of g_scratch one call needs (the formula documented in hs.h).
size_t scratch_bytes(int N_A, int N_L, int N_G) {
  if (N_A < 1 || N_L < 1 || N_G < 1) return 0;
  const size_t K = (size_t)N_A * N_L;
  size_t b = 0;
  b += align256((size_t)16 * N_A * N_L * N_L);      // M2
  b += align256((size_t)32 * N_A * N_L * N_L);      // MZ
  b += 3 * align256(sizeof(int) * (size_t)N_A);     // fail, slot, fail list
  b += align256(sizeof(int) * 4);                   // counts
  b += 3 * align256((size_t)16 * K * N_G);          // Z, W2, A rows of failing atoms
  return b;
}

}  // namespace

extern "C" int hs_assemble_static(const hs_z* A, const hs_z* B, const hs_z* T_AA,
                                  const hs_z* T_AB, const hs_z* T_BB, const double* U, int N_A,
                                  int N_L, int N_G, hs_z* H, hs_z* S, void* stream) {
  if (!A || !B || !T_AA || !T_AB || !T_BB || !U || !H || !S || H == S) return HS_EINVAL;
  if (N_A < 1 || N_L < 1 || N_L > 168 || N_G < 1) return HS_EINVAL;
  const size_t need = scratch_bytes(N_A, N_L, N_G);
  if (need == 0 || need > kStaticScratchBytes) return HS_ESCRATCH;
  void* base = nullptr;
  HS_CUDA_TRY(scratch_ptr(&base));
  cudaStream_t st = (cudaStream_t)stream;
  const int K = N_A * N_L;

  unsigned char* p = (unsigned char*)base;
  auto take = [&](size_t bytes) {
    unsigned char* q = p;
    p += align256(bytes);
    return (void*)q;
  };
  double2* M2 = (double2*)take((size_t)16 * N_A * N_L * N_L);
  double2* MZ = (double2*)take((size_t)32 * N_A * N_L * N_L);
  int* fail = (int*)take(sizeof(int) * (size_t)N_A);
  int* slot = (int*)take(sizeof(int) * (size_t)N_A);
  int* flist = (int*)take(sizeof(int) * (size_t)N_A);
  int* counts = (int*)take(sizeof(int) * 4);
  double2* Z = (double2*)take((size_t)16 * K * N_G);
  double2* W2 = (double2*)take((size_t)16 * K * N_G);
  double2* AF = (double2*)take((size_t)16 * K * N_G);

  // Every region above is fully written before it is read, so no clearing is
  // needed; only the failure count is reset so a failed launch cannot leave a
  // stale value from an earlier call.
  HS_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int), st));
  HS_CUDA_TRY(hs_launch_factor((const double2*)T_AA, (const double2*)T_AB, (const double2*)T_BB,
                               N_A, N_L, M2, MZ, fail, st));
  k_slots<<<1, 32, 0, st>>>(fail, N_A, slot, flist, counts);
  HS_CUDA_TRY(cudaGetLastError());
  int N_f = 0;
  HS_CUDA_TRY(cudaMemcpyAsync(&N_f, counts, sizeof(int), cudaMemcpyDeviceToHost, st));
  HS_CUDA_TRY(cudaStreamSynchronize(st));
  const int N_h = N_A - N_f;

  const double2* dA = (const double2*)A;
  const double2* dB = (const double2*)B;
  HS_CUDA_TRY(hs_launch_atoms_fp64(MZ, M2, fail, slot, dA, dB, K, Z, W2, K, N_A, N_L, N_G, st));
  HS_CUDA_TRY(hs_launch_gather_af(dA, K, flist, N_f, N_L, N_G, AF, st));
  SegList sS{}, sH{};
  sS.s[0] = Seg{dA, dA, nullptr, K, K, K};
  sS.s[1] = Seg{dB, dB, U, K, K, K};
  sS.n = 2;
  int n = 0;
  sH.s[n++] = Seg{Z, dB, nullptr, K, K, K};
  sH.s[n++] = Seg{dB, Z, nullptr, K, K, K};
  if (N_h > 0) sH.s[n++] = Seg{W2, W2, nullptr, K, K, N_h * N_L};
  if (N_f > 0) sH.s[n++] = Seg{AF, W2 + (size_t)N_h * N_L, nullptr, N_f * N_L, K, N_f * N_L};
  sH.n = n;
  HS_CUDA_TRY(hs_launch_contract_fp64(sS, (double2*)S, N_G, N_G, st));
  HS_CUDA_TRY(hs_launch_contract_fp64(sH, (double2*)H, N_G, N_G, st));
  HS_CUDA_TRY(hs_launch_mirror((double2*)S, N_G, N_G, st));
  HS_CUDA_TRY(hs_launch_mirror((double2*)H, N_G, N_G, st));
  HS_CUDA_TRY(cudaStreamSynchronize(st));
  return HS_OK;
}
