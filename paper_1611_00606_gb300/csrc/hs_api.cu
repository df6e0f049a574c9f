// C-ABI of libhs: plans, the synchronous assembly and the host-buffer variant.
// See include/hs.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "hs_internal.h"
#include "plan.h"

static thread_local cudaError_t g_last_cuda = cudaSuccess;
void hs_last_cuda_error(cudaError_t e) { g_last_cuda = e; }

extern "C" const char* hs_strerror(int code) {
  switch (code) {
    case HS_OK: return "ok";
    case HS_PENDING: return "pending";
    case HS_EINVAL: return "invalid argument";
    case HS_ENOMEM: return "out of device memory or above the HBM budget";
    case HS_ECUDA: return "CUDA runtime error";
    case HS_EBUSY: return "serving queue full";
    case HS_ETIMEDOUT: return "timed out";
    case HS_EDEVICE: return "device error word set (bounded wait expired)";
    case HS_ENOTSUP: return "not supported by this plan";
    case HS_ESCRATCH: return "problem larger than the static scratch of hs_assemble_static";
    default: return "unknown error";
  }
}

// ---------------------------------------------------------------------------
// workspace sizing

size_t hs_plan_s::workspace_bytes(int N_G) const {
  const size_t K = (size_t)N_A * N_L;
  size_t b = 0;
  b += 2 * 16 * K * (size_t)N_G;                    // Z, W2 (= [Y; X])
  b += 16 * (size_t)N_A * N_L * (size_t)N_G;          // AF (A rows of failing atoms), worst case
  b += split_bytes(N_G);
  return b;
}

size_t hs_plan_s::fixed_bytes() const {
  return (size_t)16 * N_A * N_L * N_L * 3 + (size_t)sizeof(int) * (3 * N_A + 16);
}

static void free_ptr(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void hs_plan_s::release() {
  free_ptr((void*&)Z);
  free_ptr((void*&)W2);
  free_ptr((void*&)AF);
  free_ptr((void*&)M2);
  free_ptr((void*&)MZ);
  free_ptr((void*&)fail_d);
  free_ptr((void*&)slot_d);
  free_ptr((void*&)fail_list_d);
  free_ptr((void*&)err_d);
  for (auto& p : stage) free_ptr(p);
  split_release();
  for (auto& e : ev)
    if (e) { cudaEventDestroy(e); e = nullptr; }
}

// ---------------------------------------------------------------------------

extern "C" int hs_plan(hs_plan_t* out, int N_A, int N_L, int N_G_max, int precision,
                       int slices, size_t hbm_budget_bytes, void* stream) {
  if (!out) return HS_EINVAL;
  *out = nullptr;
  if (N_A < 1 || N_L < 1 || N_L > kMaxNL || N_G_max < 1) return HS_EINVAL;
  if ((long long)N_A * N_L > (1LL << 30)) return HS_EINVAL;
  if (precision != HS_FP64 && precision != HS_SPLIT_BF16) return HS_EINVAL;
  if (precision == HS_SPLIT_BF16) {
    if (slices == 0) slices = kDefaultSlices;
    if (slices < 2 || slices > kMaxSlices) return HS_EINVAL;
  } else {
    slices = 0;
  }
  hs_plan_s* p = new (std::nothrow) hs_plan_s();
  if (!p) return HS_ENOMEM;
  p->N_A = N_A;
  p->N_L = N_L;
  p->N_G_max = N_G_max;
  p->precision = precision;
  p->slices = slices;
  p->budget = hbm_budget_bytes;
  p->stream = (cudaStream_t)stream;
  cudaGetDevice(&p->device);
  const size_t K = (size_t)N_A * N_L;
  const size_t need = p->workspace_bytes(N_G_max) + p->fixed_bytes();
  if (hbm_budget_bytes && need > hbm_budget_bytes) {
    delete p;
    return HS_ENOMEM;
  }
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (bytes == 0) bytes = 16;
    return cudaMalloc(ptr, bytes) == cudaSuccess;
  };
  bool ok = true;
  ok = ok && alloc((void**)&p->Z, 16 * K * N_G_max);
  ok = ok && alloc((void**)&p->W2, 16 * K * N_G_max);
  ok = ok && alloc((void**)&p->M2, (size_t)16 * N_A * N_L * N_L);
  ok = ok && alloc((void**)&p->MZ, (size_t)32 * N_A * N_L * N_L);
  ok = ok && alloc((void**)&p->fail_d, sizeof(int) * N_A);
  ok = ok && alloc((void**)&p->slot_d, sizeof(int) * N_A);
  ok = ok && alloc((void**)&p->fail_list_d, sizeof(int) * N_A);
  ok = ok && alloc((void**)&p->err_d, sizeof(int) * 16);
  ok = ok && (p->split_alloc() == HS_OK);
  for (auto& e : p->ev) ok = ok && (cudaEventCreate(&e) == cudaSuccess);
  if (!ok) {
    cudaGetLastError();
    p->release();
    delete p;
    return HS_ENOMEM;
  }
  cudaMemset(p->err_d, 0, sizeof(int) * 16);
  *out = p;
  return HS_OK;
}

extern "C" size_t hs_footprint(hs_plan_t p, int N_G) {
  if (!p || N_G < 1 || N_G > p->N_G_max) return 0;
  return p->workspace_bytes(N_G) + p->fixed_bytes() + (size_t)2 * 16 * N_G * (size_t)N_G;
}

int hs_plan_s::factor(const double2* T_AA, const double2* T_AB, const double2* T_BB) {
  HS_CUDA_TRY(cudaEventRecord(ev[1], stream));
  HS_CUDA_TRY(hs_launch_factor(T_AA, T_AB, T_BB, N_A, N_L, M2, MZ, fail_d, stream));
  fail_h.assign(N_A, 0);
  HS_CUDA_TRY(cudaMemcpyAsync(fail_h.data(), fail_d, sizeof(int) * N_A, cudaMemcpyDeviceToHost,
                              stream));
  HS_CUDA_TRY(cudaEventRecord(ev[2], stream));
  HS_CUDA_TRY(cudaStreamSynchronize(stream));
  // slot map: HPD atoms first (rows of Y), then failing atoms (rows of X)
  std::vector<int> slot(N_A), flist;
  int nh = 0;
  for (int a = 0; a < N_A; ++a)
    if (!fail_h[a]) slot[a] = nh++;
  for (int a = 0; a < N_A; ++a)
    if (fail_h[a]) {
      slot[a] = nh + (int)flist.size();
      flist.push_back(a);
    }
  N_f = (int)flist.size();
  HS_CUDA_TRY(cudaMemcpy(slot_d, slot.data(), sizeof(int) * N_A, cudaMemcpyHostToDevice));
  if (N_f)
    HS_CUDA_TRY(cudaMemcpy(fail_list_d, flist.data(), sizeof(int) * N_f, cudaMemcpyHostToDevice));
  // AF holds the A rows of the failing atoms: (N_f*N_L) x N_G_max
  if (N_f > af_atoms) {
    free_ptr((void*&)AF);
    if (cudaMalloc((void**)&AF, (size_t)16 * N_f * N_L * N_G_max) != cudaSuccess) {
      cudaGetLastError();
      af_atoms = 0;
      return HS_ENOMEM;
    }
    af_atoms = N_f;
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev[1], ev[2]);
  last_factor_ms = ms;
  tAA = T_AA;
  tAB = T_AB;
  tBB = T_BB;
  t_valid = true;
  return HS_OK;
}

extern "C" int hs_set_t(hs_plan_t p, const hs_z* T_AA, const hs_z* T_AB, const hs_z* T_BB) {
  if (!p || !T_AA || !T_AB || !T_BB) return HS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  return p->factor((const double2*)T_AA, (const double2*)T_AB, (const double2*)T_BB);
}

// Enqueue the per-k-point path on p->stream (the T factor must be current).
// ev[3..8] bracket the phases for hs_info.
int hs_plan_s::enqueue(const double2* A, const double2* B, int ldAB, const double* U, int N_G,
                       double2* H, double2* S, double2* Zw, double2* W2w, double2* AFw,
                       cudaStream_t st, bool timed) {
  const int K = N_A * N_L;
  const int N_h = N_A - N_f;
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[3], st));
  HS_CUDA_TRY(hs_launch_atoms_fp64(MZ, M2, fail_d, slot_d, A, B, ldAB, Zw, W2w, K, N_A, N_L,
                                   N_G, st));
  HS_CUDA_TRY(hs_launch_gather_af(A, ldAB, fail_list_d, N_f, N_L, N_G, AFw, st));
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[4], st));
  SegList sS{}, sH{};
  sS.s[0] = Seg{A, A, nullptr, ldAB, ldAB, K};
  sS.s[1] = Seg{B, B, U, ldAB, ldAB, K};
  sS.n = 2;
  int n = 0;
  sH.s[n++] = Seg{Zw, B, nullptr, K, ldAB, K};
  sH.s[n++] = Seg{B, Zw, nullptr, ldAB, K, K};
  if (N_h > 0) sH.s[n++] = Seg{W2w, W2w, nullptr, K, K, N_h * N_L};
  if (N_f > 0) sH.s[n++] = Seg{AFw, W2w + (size_t)N_h * N_L, nullptr, N_f * N_L, K, N_f * N_L};
  sH.n = n;
  if (precision == HS_FP64) {
    if (timed) HS_CUDA_TRY(cudaEventRecord(ev[5], st));
    HS_CUDA_TRY(hs_launch_contract_fp64(sS, S, N_G, N_G, st));
    if (timed) HS_CUDA_TRY(cudaEventRecord(ev[6], st));
    HS_CUDA_TRY(hs_launch_contract_fp64(sH, H, N_G, N_G, st));
    if (timed) HS_CUDA_TRY(cudaEventRecord(ev[7], st));
  } else {
    int rc = split_enqueue(sS, sH, N_G, H, S, st, timed);
    if (rc != HS_OK) return rc;
  }
  HS_CUDA_TRY(hs_launch_mirror(S, N_G, N_G, st));
  HS_CUDA_TRY(hs_launch_mirror(H, N_G, N_G, st));
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[8], st));
  return HS_OK;
}

int hs_plan_s::check_device_error() {
  int h = 0;
  HS_CUDA_TRY(cudaMemcpy(&h, err_d, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    cudaMemset(err_d, 0, sizeof(int) * 16);
    return HS_EDEVICE;
  }
  return HS_OK;
}

void hs_plan_s::fill_info(hs_info* info, bool factored) {
  if (!info) return;
  std::memset(info, 0, sizeof(*info));
  info->n_fallback = N_f;
  info->slices = slices;
  auto el = [&](int a, int b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[a], ev[b]) != cudaSuccess) {
      cudaGetLastError();
      return 0.0;
    }
    return (double)ms;
  };
  info->ms_factor = factored ? last_factor_ms : 0.0;
  info->ms_atoms = el(3, 4);
  if (precision == HS_FP64) {
    info->ms_slice = 0.0;
    info->ms_S = el(5, 6);
    info->ms_H = el(6, 7);
  } else {
    info->ms_slice = el(4, 5);
    info->ms_S = el(5, 6);
    info->ms_H = el(6, 7);
  }
  info->ms_finalize = el(7, 8);
  info->ms_total = el(3, 8) + info->ms_factor;
}

static int check_args(hs_plan_t p, const void* A, const void* B, const void* T_AA,
                      const void* T_AB, const void* T_BB, const void* U, int N_A, int N_L,
                      int N_G, const void* H, const void* S) {
  if (!p || !A || !B || !T_AA || !T_AB || !T_BB || !U || !H || !S) return HS_EINVAL;
  if (N_A != p->N_A || N_L != p->N_L || N_G < 1 || N_G > p->N_G_max) return HS_EINVAL;
  if (H == S) return HS_EINVAL;
  return HS_OK;
}

extern "C" int hs_assemble(hs_plan_t p, const hs_z* A, const hs_z* B, const hs_z* T_AA,
                           const hs_z* T_AB, const hs_z* T_BB, const double* U, int N_A,
                           int N_L, int N_G, hs_z* H, hs_z* S, hs_info* info) {
  int rc = check_args(p, A, B, T_AA, T_AB, T_BB, U, N_A, N_L, N_G, H, S);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(p->mu);
  bool factored = false;
  if (!p->t_valid || p->tAA != (const void*)T_AA || p->tAB != (const void*)T_AB ||
      p->tBB != (const void*)T_BB) {
    rc = p->factor((const double2*)T_AA, (const double2*)T_AB, (const double2*)T_BB);
    if (rc) return rc;
    factored = true;
  }
  const int K = N_A * N_L;
  rc = p->enqueue((const double2*)A, (const double2*)B, K, U, N_G, (double2*)H, (double2*)S, p->Z,
                  p->W2, p->AF, p->stream, true);
  if (rc) return rc;
  HS_CUDA_TRY(cudaStreamSynchronize(p->stream));
  rc = p->check_device_error();
  if (rc) return rc;
  p->fill_info(info, factored);
  return HS_OK;
}

extern "C" int hs_assemble_host(hs_plan_t p, const hs_z* A, const hs_z* B, const hs_z* T_AA,
                                const hs_z* T_AB, const hs_z* T_BB, const double* U, int N_A,
                                int N_L, int N_G, hs_z* H, hs_z* S, hs_info* info) {
  int rc = check_args(p, A, B, T_AA, T_AB, T_BB, U, N_A, N_L, N_G, H, S);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(p->mu);
  const size_t K = (size_t)N_A * N_L;
  const size_t nT = (size_t)N_A * N_L * N_L;
  const size_t sz[7] = {16 * K * p->N_G_max, 16 * K * p->N_G_max, 16 * nT * 3,
                        8 * K, (size_t)16 * p->N_G_max * p->N_G_max,
                        (size_t)16 * p->N_G_max * p->N_G_max, 0};
  for (int i = 0; i < 6; ++i)
    if (!p->stage[i] && cudaMalloc(&p->stage[i], sz[i]) != cudaSuccess) {
      cudaGetLastError();
      return HS_ENOMEM;
    }
  double2* dA = (double2*)p->stage[0];
  double2* dB = (double2*)p->stage[1];
  double2* dT = (double2*)p->stage[2];
  double* dU = (double*)p->stage[3];
  double2* dH = (double2*)p->stage[4];
  double2* dS = (double2*)p->stage[5];
  cudaStream_t st = p->stream;
  HS_CUDA_TRY(cudaMemcpyAsync(dA, A, 16 * K * N_G, cudaMemcpyHostToDevice, st));
  HS_CUDA_TRY(cudaMemcpyAsync(dB, B, 16 * K * N_G, cudaMemcpyHostToDevice, st));
  HS_CUDA_TRY(cudaMemcpyAsync(dU, U, 8 * K, cudaMemcpyHostToDevice, st));
  bool factored = false;
  if (!p->t_valid || p->host_tAA != (const void*)T_AA || p->host_tAB != (const void*)T_AB ||
      p->host_tBB != (const void*)T_BB) {
    HS_CUDA_TRY(cudaMemcpyAsync(dT, T_AA, 16 * nT, cudaMemcpyHostToDevice, st));
    HS_CUDA_TRY(cudaMemcpyAsync(dT + nT, T_AB, 16 * nT, cudaMemcpyHostToDevice, st));
    HS_CUDA_TRY(cudaMemcpyAsync(dT + 2 * nT, T_BB, 16 * nT, cudaMemcpyHostToDevice, st));
    rc = p->factor(dT, dT + nT, dT + 2 * nT);
    if (rc) return rc;
    p->host_tAA = T_AA;
    p->host_tAB = T_AB;
    p->host_tBB = T_BB;
    factored = true;
  }
  rc = p->enqueue(dA, dB, (int)K, dU, N_G, dH, dS, p->Z, p->W2, p->AF, st, true);
  if (rc) return rc;
  HS_CUDA_TRY(cudaMemcpyAsync(H, dH, (size_t)16 * N_G * N_G, cudaMemcpyDeviceToHost, st));
  HS_CUDA_TRY(cudaMemcpyAsync(S, dS, (size_t)16 * N_G * N_G, cudaMemcpyDeviceToHost, st));
  HS_CUDA_TRY(cudaStreamSynchronize(st));
  rc = p->check_device_error();
  if (rc) return rc;
  p->fill_info(info, factored);
  return HS_OK;
}

extern "C" int hs_fallback_flags(hs_plan_t p, int* flags_host) {
  if (!p || !flags_host) return HS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  if (!p->t_valid) return HS_EINVAL;
  std::copy(p->fail_h.begin(), p->fail_h.end(), flags_host);
  return HS_OK;
}

extern "C" int hs_destroy(hs_plan_t p) {
  if (!p) return HS_EINVAL;
  p->serve_shutdown();
  {
    std::lock_guard<std::mutex> lk(p->mu);
    cudaStreamSynchronize(p->stream);
    p->release();
  }
  delete p;
  return HS_OK;
}
