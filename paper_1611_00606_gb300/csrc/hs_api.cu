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
    case HS_ENOTPD: return "S is not positive definite";
    default: return "unknown error";
  }
}

// ---------------------------------------------------------------------------
// workspace sizing and allocation

size_t hs_plan_s::ws_bytes(int N_G, int n_fail) const {
  const size_t K = (size_t)N_A * N_L;
  const size_t nf = (size_t)(n_fail > 0 ? n_fail : 1);
  size_t b = 0;
  b += 2 * ws_elem() * K * (size_t)N_G;     // Z, W2 (= [Y; X])
  b += ws_elem() * nf * N_L * (size_t)N_G;  // AF (A rows of failing atoms)
  b += split_ws_bytes(N_G, n_fail);
  return b;
}

size_t hs_plan_s::fixed_bytes() const {
  size_t b = (size_t)16 * N_A * N_L * N_L * 3 + (size_t)sizeof(int) * (3 * N_A + 16) +
             split_fixed_bytes();
  if (real) {
    b += (size_t)16 * N_A * N_L * N_L * 3;  // Tc
    if (precision == HS_FP64)               // Ac, Bc, Hc, Sc
      b += (size_t)2 * 16 * N_A * N_L * N_G_max + (size_t)2 * 16 * N_G_max * (size_t)N_G_max;
  }
  return b;
}

static void free_ptr(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

static void free_ws_ptr(void*& p, bool async, cudaStream_t st) {
  if (p) {
    if (async) cudaFreeAsync(p, st);
    else cudaFree(p);
  }
  p = nullptr;
}

int hs_plan_s::ws_alloc(Workspace& w, int N_G, int n_fail, cudaStream_t st, bool async) {
  const size_t K = (size_t)N_A * N_L;
  const size_t nf = (size_t)(n_fail > 0 ? n_fail : 1);
  w = Workspace{};
  w.async = async;
  w.N_G = N_G;
  w.n_fail = (int)nf;
  auto al = [&](void** ptr, size_t bytes) -> bool {
    if (bytes == 0) bytes = 256;
    return (async ? hs_malloc_async(ptr, bytes, st, hs_serve_pool(this)) : cudaMalloc(ptr, bytes)) ==
           cudaSuccess;
  };
  const size_t e = ws_elem();
  bool ok = al((void**)&w.Z, e * K * N_G) && al((void**)&w.W2, e * K * N_G) &&
            al((void**)&w.AF, e * nf * N_L * N_G);
  if (ok) ok = split_ws_alloc(w, N_G, (int)nf, st, async) == HS_OK;
  if (!ok) {
    cudaGetLastError();
    ws_free(w, st);
    return HS_ENOMEM;
  }
  return HS_OK;
}

void hs_plan_s::ws_free(Workspace& w, cudaStream_t st) {
  free_ws_ptr((void*&)w.Z, w.async, st);
  free_ws_ptr((void*&)w.W2, w.async, st);
  free_ws_ptr((void*&)w.AF, w.async, st);
  for (auto& b : w.sb) {
    free_ws_ptr((void*&)b.plain, w.async, st);
    free_ws_ptr((void*&)b.expo, w.async, st);
    b.rot = false;
  }
  w.N_G = 0;
  w.n_fail = 0;
}

void hs_plan_s::release() {
  ws_free(ws, stream);
  free_ptr((void*&)M2);
  free_ptr((void*&)MZ);
  free_ptr((void*&)fail_d);
  free_ptr((void*&)slot_d);
  free_ptr((void*&)fail_list_d);
  free_ptr((void*&)err_d);
  free_ptr((void*&)Tc);
  free_ptr((void*&)Ac);
  free_ptr((void*&)Bc);
  free_ptr((void*&)Hc);
  free_ptr((void*&)Sc);
  split_plan_release();
  for (auto& p : stage) free_ptr(p);
  free_ptr((void*&)red_W);
  free_ptr((void*&)red_P);
  free_ptr((void*&)red_fail);
  red_cap = 0;
  split_reduce_release();
  for (auto& e : red_ev)
    if (e) { cudaEventDestroy(e); e = nullptr; }
  for (auto& e : real_ev)
    if (e) { cudaEventDestroy(e); e = nullptr; }
  for (auto& e : copy_ev)
    if (e) { cudaEventDestroy(e); e = nullptr; }
  if (copy_stream) { cudaStreamDestroy(copy_stream); copy_stream = nullptr; }
  if (s_stream) { cudaStreamDestroy(s_stream); s_stream = nullptr; }
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
  const bool real = (precision & HS_REAL) != 0;
  precision &= ~HS_REAL;
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
  p->real = real;
  p->slices = slices;
  p->budget = hbm_budget_bytes;
  p->stream = (cudaStream_t)stream;
  cudaGetDevice(&p->device);
  if (hbm_budget_bytes && p->fixed_bytes() + p->ws_bytes(1, 1) > hbm_budget_bytes) {
    delete p;
    return HS_ENOMEM;
  }
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (bytes == 0) bytes = 16;
    return cudaMalloc(ptr, bytes) == cudaSuccess;
  };
  bool ok = true;
  ok = ok && alloc((void**)&p->M2, (size_t)16 * N_A * N_L * N_L);
  ok = ok && alloc((void**)&p->MZ, (size_t)32 * N_A * N_L * N_L);
  ok = ok && alloc((void**)&p->fail_d, sizeof(int) * N_A);
  ok = ok && alloc((void**)&p->slot_d, sizeof(int) * N_A);
  ok = ok && alloc((void**)&p->fail_list_d, sizeof(int) * N_A);
  ok = ok && alloc((void**)&p->err_d, sizeof(int) * 16);
  ok = ok && (p->split_plan_alloc() == HS_OK);
  if (real) {
    ok = ok && alloc((void**)&p->Tc, (size_t)3 * 16 * N_A * N_L * N_L);
    if (precision == HS_FP64) {
      const size_t K = (size_t)N_A * N_L;
      ok = ok && alloc((void**)&p->Ac, 16 * K * N_G_max) && alloc((void**)&p->Bc, 16 * K * N_G_max);
      ok = ok && alloc((void**)&p->Hc, (size_t)16 * N_G_max * N_G_max) &&
           alloc((void**)&p->Sc, (size_t)16 * N_G_max * N_G_max);
    }
  }
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
  const int nf = p->t_valid ? p->N_f : p->N_A;
  return p->ws_bytes(N_G, nf) + (size_t)2 * (p->real ? 8 : 16) * N_G * (size_t)N_G;
}

int hs_plan_s::factor(const double2* T_AA, const double2* T_AB, const double2* T_BB) {
  HS_CUDA_TRY(cudaEventRecord(ev[1], stream));
  HS_CUDA_TRY(hs_launch_factor(T_AA, T_AB, T_BB, N_A, N_L, M2, MZ, fail_d, stream));
  int rc = split_factor(stream);
  if (rc != HS_OK) return rc;
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
  if (!p || !T_AA || !T_AB || !T_BB || p->real) return HS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  if (p->serve_busy()) return HS_EBUSY;  // requests in flight use the cached factor
  int rc = p->factor((const double2*)T_AA, (const double2*)T_AB, (const double2*)T_BB);
  if (rc == HS_OK) p->factor_pending_info = true;
  return rc;
}

// Enqueue the per-k-point path on stream st using workspace w (the T factor
// must be current).  ev[3..8] bracket the phases for hs_info when timed.
int hs_plan_s::enqueue(const double2* A, const double2* B, int ldAB, const double* U, int N_G,
                       double2* H, double2* S, Workspace& w, cudaStream_t st, bool timed,
                       cudaEvent_t s_done, bool presliced, bool mirror) {
  const int K = N_A * N_L;
  const int N_h = N_A - N_f;
  if (w.N_G < N_G || w.n_fail < N_f) return HS_EINVAL;
  if (timed && !presliced) HS_CUDA_TRY(cudaEventRecord(ev[3], st));
  if (precision == HS_SPLIT_BF16) {
    int rc = split_enqueue(A, B, ldAB, U, N_G, H, S, w, st, timed, s_done, presliced, mirror);
    if (rc != HS_OK) return rc;
  } else {
    HS_CUDA_TRY(hs_launch_atoms_fp64(MZ, M2, fail_d, slot_d, A, B, ldAB, w.Z, w.W2, K, N_A, N_L,
                                     N_G, st));
    HS_CUDA_TRY(hs_launch_gather_af(A, ldAB, fail_list_d, N_f, N_L, N_G, w.AF, st));
    if (timed) HS_CUDA_TRY(cudaEventRecord(ev[4], st));
    SegList sS{}, sH{};
    sS.s[0] = Seg{A, A, nullptr, ldAB, ldAB, K};
    sS.s[1] = Seg{B, B, U, ldAB, ldAB, K};
    sS.n = 2;
    int n = 0;
    sH.s[n++] = Seg{w.Z, B, nullptr, K, ldAB, K};
    sH.s[n++] = Seg{B, w.Z, nullptr, ldAB, K, K};
    if (N_h > 0) sH.s[n++] = Seg{w.W2, w.W2, nullptr, K, K, N_h * N_L};
    if (N_f > 0)
      sH.s[n++] = Seg{w.AF, w.W2 + (size_t)N_h * N_L, nullptr, N_f * N_L, K, N_f * N_L};
    sH.n = n;
    if (timed) HS_CUDA_TRY(cudaEventRecord(ev[5], st));
    HS_CUDA_TRY(hs_launch_contract_fp64(sS, S, N_G, N_G, st));
    if (mirror) HS_CUDA_TRY(hs_launch_mirror(S, N_G, N_G, st));  // S final: it can leave
    if (s_done) HS_CUDA_TRY(cudaEventRecord(s_done, st));
    if (timed) HS_CUDA_TRY(cudaEventRecord(ev[6], st));
    HS_CUDA_TRY(hs_launch_contract_fp64(sH, H, N_G, N_G, st));
    if (timed) HS_CUDA_TRY(cudaEventRecord(ev[7], st));
  }
  // (S was mirrored right after its contraction)
  if (!mirror) {
  } else if (real && precision == HS_SPLIT_BF16) {
    HS_CUDA_TRY(hs_launch_mirror_real((double*)H, N_G, N_G, st));
  } else {
    HS_CUDA_TRY(hs_launch_mirror(H, N_G, N_G, st));
  }
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
  info->ms_factor = (factored || factor_pending_info) ? last_factor_ms : 0.0;
  factor_pending_info = false;
  if (precision == HS_FP64) {
    info->ms_atoms = el(3, 4);
    info->ms_slice = 0.0;
  } else {  // slice inputs [3, 9], per-atom products [9, 4], slice outputs [4, 5]
    info->ms_atoms = el(9, 4);
    info->ms_slice = el(3, 9) + el(4, 5);
  }
  info->ms_S = el(5, 6);
  info->ms_H = el(6, 7);
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

// The synchronous workspace: allocated on first use for N_G_max, regrown when
// more atoms fail than it has room for.
static int ensure_sync_ws(hs_plan_t p) {
  if (p->ws.N_G == p->N_G_max && p->ws.n_fail >= p->N_f) return HS_OK;
  HS_CUDA_TRY(cudaStreamSynchronize(p->stream));
  p->ws_free(p->ws, p->stream);
  return p->ws_alloc(p->ws, p->N_G_max, p->N_f, p->stream, false);
}

extern "C" int hs_assemble(hs_plan_t p, const hs_z* A, const hs_z* B, const hs_z* T_AA,
                           const hs_z* T_AB, const hs_z* T_BB, const double* U, int N_A,
                           int N_L, int N_G, hs_z* H, hs_z* S, hs_info* info) {
  int rc = check_args(p, A, B, T_AA, T_AB, T_BB, U, N_A, N_L, N_G, H, S);
  if (rc) return rc;
  if (p->real) return HS_EINVAL;  // real plans: hs_assemble_real
  std::lock_guard<std::mutex> lk(p->mu);
  bool factored = false;
  if (!p->t_valid || p->tAA != (const void*)T_AA || p->tAB != (const void*)T_AB ||
      p->tBB != (const void*)T_BB) {
    if (p->serve_busy()) return HS_EBUSY;
    rc = p->factor((const double2*)T_AA, (const double2*)T_AB, (const double2*)T_BB);
    if (rc) return rc;
    factored = true;
  }
  rc = ensure_sync_ws(p);
  if (rc) return rc;
  const int K = N_A * N_L;
  rc = p->enqueue((const double2*)A, (const double2*)B, K, U, N_G, (double2*)H, (double2*)S, p->ws,
                  p->stream, true);
  if (rc) return rc;
  HS_CUDA_TRY(cudaStreamSynchronize(p->stream));
  rc = p->check_device_error();
  if (rc) return rc;
  p->fill_info(info, factored);
  return HS_OK;
}

// K-split over atoms (the multi-GPU form of Sec. 4, one atom range per rank): the terms
// of this plan's atoms, lower triangles only; the caller sums the partials of all atom
// ranges and calls hs_finalize.
extern "C" int hs_assemble_partial(hs_plan_t p, const hs_z* A, const hs_z* B, int ld_AB,
                                   const hs_z* T_AA, const hs_z* T_AB, const hs_z* T_BB,
                                   const double* U, int N_A, int N_L, int N_G, hs_z* H,
                                   hs_z* S, hs_info* info) {
  int rc = check_args(p, A, B, T_AA, T_AB, T_BB, U, N_A, N_L, N_G, H, S);
  if (rc) return rc;
  if (p->real || ld_AB < N_A * N_L) return HS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  bool factored = false;
  if (!p->t_valid || p->tAA != (const void*)T_AA || p->tAB != (const void*)T_AB ||
      p->tBB != (const void*)T_BB) {
    if (p->serve_busy()) return HS_EBUSY;
    rc = p->factor((const double2*)T_AA, (const double2*)T_AB, (const double2*)T_BB);
    if (rc) return rc;
    factored = true;
  }
  rc = ensure_sync_ws(p);
  if (rc) return rc;
  rc = p->enqueue((const double2*)A, (const double2*)B, ld_AB, U, N_G, (double2*)H, (double2*)S,
                  p->ws, p->stream, true, nullptr, false, /*mirror=*/false);
  if (rc) return rc;
  HS_CUDA_TRY(cudaStreamSynchronize(p->stream));
  rc = p->check_device_error();
  if (rc) return rc;
  p->fill_info(info, factored);
  return HS_OK;
}

extern "C" int hs_finalize(hs_plan_t p, hs_z* H, hs_z* S, int N_G) {
  if (!p || !H || !S || H == S || p->real || N_G < 1 || N_G > p->N_G_max) return HS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  HS_CUDA_TRY(hs_launch_mirror((double2*)H, N_G, N_G, p->stream));
  HS_CUDA_TRY(hs_launch_mirror((double2*)S, N_G, N_G, p->stream));
  HS_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return HS_OK;
}

extern "C" int hs_assemble_host(hs_plan_t p, const hs_z* A, const hs_z* B, const hs_z* T_AA,
                                const hs_z* T_AB, const hs_z* T_BB, const double* U, int N_A,
                                int N_L, int N_G, hs_z* H, hs_z* S, hs_info* info) {
  int rc = check_args(p, A, B, T_AA, T_AB, T_BB, U, N_A, N_L, N_G, H, S);
  if (rc) return rc;
  if (p->real) return HS_EINVAL;  // real plans: hs_assemble_real (device buffers)
  std::lock_guard<std::mutex> lk(p->mu);
  const size_t K = (size_t)N_A * N_L;
  const size_t nT = (size_t)N_A * N_L * N_L;
  const size_t sz[6] = {16 * K * p->N_G_max, 16 * K * p->N_G_max, 16 * nT * 3,
                        8 * K, (size_t)16 * p->N_G_max * p->N_G_max,
                        (size_t)16 * p->N_G_max * p->N_G_max};
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
  // Copies run on a copy stream of their own: A and B in column chunks, each sliced
  // (split form) as soon as it has landed; T first, so the factorisation, whose host
  // step waits for it, does not wait for A and B; S leaves while H is computed.
  if (!p->copy_stream) {
    HS_CUDA_TRY(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
    HS_CUDA_TRY(cudaStreamCreateWithFlags(&p->s_stream, cudaStreamNonBlocking));
    for (auto& e : p->copy_ev) HS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  cudaStream_t cs = p->copy_stream;
  // copy_ev[0..3]: chunks landed; [4]: start; [5]: S final; [6..9]: chunks sliced
  constexpr int kChunks = 4;
  HS_CUDA_TRY(cudaEventRecord(p->copy_ev[4], st));  // after everything already queued on st
  HS_CUDA_TRY(cudaStreamWaitEvent(cs, p->copy_ev[4], 0));
  HS_CUDA_TRY(cudaMemcpyAsync(dU, U, 8 * K, cudaMemcpyHostToDevice, st));
  bool factored = false;
  if (!p->t_valid || p->host_tAA != (const void*)T_AA || p->host_tAB != (const void*)T_AB ||
      p->host_tBB != (const void*)T_BB) {
    if (p->serve_busy()) return HS_EBUSY;
    HS_CUDA_TRY(cudaMemcpyAsync(dT, T_AA, 16 * nT, cudaMemcpyHostToDevice, st));
    HS_CUDA_TRY(cudaMemcpyAsync(dT + nT, T_AB, 16 * nT, cudaMemcpyHostToDevice, st));
    HS_CUDA_TRY(cudaMemcpyAsync(dT + 2 * nT, T_BB, 16 * nT, cudaMemcpyHostToDevice, st));
  }
  // chunk boundaries on 128-column (row-block) multiples; the last chunk ends at N_G
  int c0[kChunks + 1];
  for (int c = 0; c <= kChunks; ++c)
    c0[c] = (int)(((long long)N_G * c / kChunks + 127) / 128 * 128);
  c0[kChunks] = N_G;
  for (int c = 0; c < kChunks; ++c) {
    const size_t off = K * (size_t)std::min(c0[c], N_G);
    const size_t n = K * (size_t)(std::min(c0[c + 1], N_G) - std::min(c0[c], N_G));
    if (n) {
      HS_CUDA_TRY(cudaMemcpyAsync(dA + off, A + off, 16 * n, cudaMemcpyHostToDevice, cs));
      HS_CUDA_TRY(cudaMemcpyAsync(dB + off, B + off, 16 * n, cudaMemcpyHostToDevice, cs));
    }
    HS_CUDA_TRY(cudaEventRecord(p->copy_ev[c], cs));
  }
  if (p->host_tAA != (const void*)T_AA || p->host_tAB != (const void*)T_AB ||
      p->host_tBB != (const void*)T_BB || !p->t_valid) {
    rc = p->factor(dT, dT + nT, dT + 2 * nT);
    if (rc) return rc;
    p->host_tAA = T_AA;
    p->host_tAB = T_AB;
    p->host_tBB = T_BB;
    factored = true;
  }
  rc = ensure_sync_ws(p);
  if (rc) return rc;
  const bool split = p->precision == HS_SPLIT_BF16;
  if (split) {
    // slice each chunk as it lands; on the S stream, the S tiles of its row blocks (a
    // lower-triangle tile of row block b reads A, U.B columns below 128 (b + 1) only),
    // so S fills the time the copies leave and the other kernels fill the S launches'
    // tails; S is mirrored and copied back as soon as its last chunk is done
    cudaStream_t ss = p->s_stream;
    HS_CUDA_TRY(cudaEventRecord(p->ev[3], st));
    const int nbi = (N_G + 127) / 128;
    for (int c = 0; c < kChunks; ++c) {
      HS_CUDA_TRY(cudaStreamWaitEvent(st, p->copy_ev[c], 0));
      const int g0 = std::min(c0[c], N_G), g1 = std::min(c0[c + 1], N_G);
      // the last chunk also writes the zero rows past N_G (ng = -1: up to the padding)
      if (g1 > g0 || c == kChunks - 1) {
        rc = p->split_inputs(dA, dB, (int)K, dU, N_G, p->ws, st, g0,
                             c == kChunks - 1 ? -1 : g1 - g0);
        if (rc) return rc;
      }
      HS_CUDA_TRY(cudaEventRecord(p->copy_ev[6 + c], st));
      HS_CUDA_TRY(cudaStreamWaitEvent(ss, p->copy_ev[6 + c], 0));
      const int b0 = std::min(c0[c], N_G) / 128;
      const int b1 = c == kChunks - 1 ? nbi : std::min(c0[c + 1], N_G) / 128;
      rc = p->split_contract_S_rows(N_G, dS, p->ws, ss, b0, b1);
      if (rc) return rc;
    }
    HS_CUDA_TRY(hs_launch_mirror(dS, N_G, N_G, ss));
    HS_CUDA_TRY(cudaEventRecord(p->copy_ev[5], ss));
  } else {
    HS_CUDA_TRY(cudaStreamWaitEvent(st, p->copy_ev[kChunks - 1], 0));
  }
  rc = p->enqueue(dA, dB, (int)K, dU, N_G, dH, dS, p->ws, st, true,
                  split ? nullptr : p->copy_ev[5], split);
  if (rc) return rc;
  HS_CUDA_TRY(cudaStreamWaitEvent(cs, p->copy_ev[5], 0));
  HS_CUDA_TRY(cudaMemcpyAsync(S, dS, (size_t)16 * N_G * N_G, cudaMemcpyDeviceToHost, cs));
  HS_CUDA_TRY(cudaMemcpyAsync(H, dH, (size_t)16 * N_G * N_G, cudaMemcpyDeviceToHost, st));
  HS_CUDA_TRY(cudaStreamSynchronize(cs));  // (after the S stream, whose S-final event it waited for)
  HS_CUDA_TRY(cudaStreamSynchronize(st));
  rc = p->check_device_error();
  if (rc) return rc;
  p->fill_info(info, factored);
  return HS_OK;
}

// ---------------------------------------------------------------------------
// Real-symmetric variant

int hs_plan_s::factor_real(const double* T_AA, const double* T_AB, const double* T_BB) {
  const size_t n = (size_t)N_A * N_L * N_L;
  HS_CUDA_TRY(hs_launch_embed(T_AA, Tc, n, stream));
  HS_CUDA_TRY(hs_launch_embed(T_AB, Tc + n, n, stream));
  HS_CUDA_TRY(hs_launch_embed(T_BB, Tc + 2 * n, n, stream));
  int rc = factor(Tc, Tc + n, Tc + 2 * n);
  if (rc) return rc;
  tAA = T_AA;  // the cache is keyed by the caller's real arrays
  tAB = T_AB;
  tBB = T_BB;
  return HS_OK;
}

extern "C" int hs_set_t_real(hs_plan_t p, const double* T_AA, const double* T_AB,
                             const double* T_BB) {
  if (!p || !T_AA || !T_AB || !T_BB || !p->real) return HS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  int rc = p->factor_real(T_AA, T_AB, T_BB);
  if (rc == HS_OK) p->factor_pending_info = true;
  return rc;
}

extern "C" int hs_assemble_real(hs_plan_t p, const double* A, const double* B,
                                const double* T_AA, const double* T_AB, const double* T_BB,
                                const double* U, int N_A, int N_L, int N_G, double* H, double* S,
                                hs_info* info) {
  int rc = check_args(p, A, B, T_AA, T_AB, T_BB, U, N_A, N_L, N_G, H, S);
  if (rc) return rc;
  if (!p->real) return HS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  bool factored = false;
  if (!p->t_valid || p->tAA != (const void*)T_AA || p->tAB != (const void*)T_AB ||
      p->tBB != (const void*)T_BB) {
    rc = p->factor_real(T_AA, T_AB, T_BB);
    if (rc) return rc;
    factored = true;
  }
  rc = ensure_sync_ws(p);
  if (rc) return rc;
  const int K = N_A * N_L;
  if (p->precision == HS_SPLIT_BF16) {
    // native real: the double arrays travel through the double2-typed plumbing
    rc = p->enqueue((const double2*)A, (const double2*)B, K, U, N_G, (double2*)H, (double2*)S,
                    p->ws, p->stream, true);
    if (rc) return rc;
  } else {
    // FP64 form: the complex kernels on A, B embedded as complex, then Re(H), Re(S)
    HS_CUDA_TRY(hs_launch_embed2d(A, K, p->Ac, K, K, N_G, p->stream));
    HS_CUDA_TRY(hs_launch_embed2d(B, K, p->Bc, K, K, N_G, p->stream));
    rc = p->enqueue(p->Ac, p->Bc, K, U, N_G, p->Hc, p->Sc, p->ws, p->stream, true);
    if (rc) return rc;
    HS_CUDA_TRY(hs_launch_real_part(p->Hc, N_G, H, N_G, N_G, p->stream));
    HS_CUDA_TRY(hs_launch_real_part(p->Sc, N_G, S, N_G, N_G, p->stream));
  }
  HS_CUDA_TRY(cudaStreamSynchronize(p->stream));
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

// ---------------------------------------------------------------------------
// Generalized-eigenproblem reduction (Sec. 1.1): S <- L, H <- L^{-1} H L^{-H}.

// The reduction of complex device buffers dH, dS (arguments checked, plan locked).
static int reduce_locked(hs_plan_s* p, double2* dH, double2* dS, int N_G, hs_reduce_info* info) {
  if (p->red_cap < N_G) {
    free_ptr((void*&)p->red_W);
    free_ptr((void*&)p->red_P);
    p->red_cap = 0;
    const size_t bytes = (size_t)16 * N_G * N_G;
    if (cudaMalloc((void**)&p->red_W, bytes) != cudaSuccess ||
        cudaMalloc((void**)&p->red_P, bytes) != cudaSuccess) {
      cudaGetLastError();
      free_ptr((void*&)p->red_W);
      free_ptr((void*&)p->red_P);
      return HS_ENOMEM;
    }
    p->red_cap = N_G;
  }
  if (!p->red_fail) {
    if (cudaMalloc((void**)&p->red_fail, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return HS_ENOMEM;
    }
  }
  for (auto& e : p->red_ev)
    if (!e) HS_CUDA_TRY(cudaEventCreate(&e));
  const bool split = p->precision == HS_SPLIT_BF16;
  if (split) {
    const int rc = p->split_reduce_alloc(N_G);
    if (rc) return rc;
  }
  cudaStream_t st = p->stream;
  int fail = 0;
  HS_CUDA_TRY(cudaMemsetAsync(p->red_fail, 0, sizeof(int), st));
  HS_CUDA_TRY(cudaEventRecord(p->red_ev[0], st));
  if (split) {
    // the Cholesky on the plan's stream; the inverse on the S stream, block row i as soon
    // as the Cholesky's panel i is final (both chains are narrow FP64 launches between
    // tensor-core updates, so they overlap)
    if (!p->s_stream) HS_CUDA_TRY(cudaStreamCreateWithFlags(&p->s_stream, cudaStreamNonBlocking));
    cudaStream_t s2 = p->s_stream;
    HS_CUDA_TRY(cudaEventRecord(p->red_ev[5], st));  // after the failure word's reset
    HS_CUDA_TRY(cudaStreamWaitEvent(s2, p->red_ev[5], 0));
    int rc = p->split_cholesky(dS, N_G, p->red_fail, st);
    if (rc) return rc;
    HS_CUDA_TRY(cudaEventRecord(p->red_ev[1], st));
    rc = p->split_inverse(dS, p->red_W, N_G, p->red_fail, s2);
    if (rc) return rc;
    HS_CUDA_TRY(cudaEventRecord(p->red_ev[6], s2));
    HS_CUDA_TRY(cudaStreamWaitEvent(st, p->red_ev[6], 0));
    // the slice path does not read the failure word: stop here if S failed
    HS_CUDA_TRY(cudaMemcpyAsync(&fail, p->red_fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    HS_CUDA_TRY(cudaStreamSynchronize(st));
    if (fail) {
      if (info) info->fail_col = fail;
      return HS_ENOTPD;
    }
  } else {
    HS_CUDA_TRY(hs_launch_cholesky(dS, N_G, p->red_fail, st));
    HS_CUDA_TRY(cudaEventRecord(p->red_ev[1], st));
    HS_CUDA_TRY(hs_launch_tri_inverse(dS, p->red_W, N_G, p->red_fail, st));
  }
  HS_CUDA_TRY(cudaEventRecord(p->red_ev[2], st));
  if (split) {
    // B = W^H; H completed from its lower triangle; then H <- B^H H B on the tensor cores
    HS_CUDA_TRY(hs_launch_ctrans(p->red_W, N_G, N_G, N_G, p->red_P, N_G, st));
    HS_CUDA_TRY(hs_launch_mirror(dH, N_G, N_G, st));
    const int rc = p->split_reduce_transform(p->red_P, dH, N_G, st, p->red_ev[3]);
    if (rc) return rc;
  } else {
    HS_CUDA_TRY(hs_launch_reduce_p(p->red_W, dH, p->red_P, N_G, p->red_fail, st));
    HS_CUDA_TRY(cudaEventRecord(p->red_ev[3], st));
    HS_CUDA_TRY(hs_launch_reduce_g(p->red_P, p->red_W, dH, N_G, p->red_fail, st));
    HS_CUDA_TRY(hs_launch_hermsum(dH, N_G, p->red_fail, st));
  }
  HS_CUDA_TRY(cudaEventRecord(p->red_ev[4], st));
  HS_CUDA_TRY(cudaMemcpyAsync(&fail, p->red_fail, sizeof(int), cudaMemcpyDeviceToHost, st));
  HS_CUDA_TRY(cudaStreamSynchronize(st));
  if (split) {
    const int rc = p->check_device_error();
    if (rc) return rc;
  }
  if (info) {
    auto el = [&](int a, int b) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p->red_ev[a], p->red_ev[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
      }
      return (double)ms;
    };
    info->fail_col = fail;
    info->ms_cholesky = el(0, 1);
    info->ms_inverse = el(1, 2);
    info->ms_p = el(2, 3);
    info->ms_g = el(3, 4);
    info->ms_total = el(0, 4);
  }
  return fail ? HS_ENOTPD : HS_OK;
}

extern "C" int hs_reduce(hs_plan_t p, hs_z* H, hs_z* S, int N_G, hs_reduce_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (!p || !H || !S || N_G < 0 || N_G > p->N_G_max || p->real) return HS_EINVAL;
  if (N_G == 0) return HS_OK;
  if (H == S) return HS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  return reduce_locked(p, (double2*)H, (double2*)S, N_G, info);
}

// Real symmetric pairs (Sec. 1.1): embedded as complex in the FP64 real plan's complex
// H, S buffers, reduced by the complex FP64 kernels (imaginary parts stay exactly zero),
// real parts copied back.
extern "C" int hs_reduce_real(hs_plan_t p, double* H, double* S, int N_G, hs_reduce_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (!p || !H || !S || N_G < 0 || N_G > p->N_G_max || !p->real) return HS_EINVAL;
  if (N_G == 0) return HS_OK;
  if (H == S) return HS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  if (!p->Hc || !p->Sc) {  // split real plans: the complex embedding on first use
    const size_t bytes = (size_t)16 * p->N_G_max * p->N_G_max;
    if ((!p->Hc && cudaMalloc((void**)&p->Hc, bytes) != cudaSuccess) ||
        (!p->Sc && cudaMalloc((void**)&p->Sc, bytes) != cudaSuccess)) {
      cudaGetLastError();
      free_ptr((void*&)p->Hc);
      free_ptr((void*&)p->Sc);
      return HS_ENOMEM;
    }
  }
  cudaStream_t st = p->stream;
  for (auto& e : p->real_ev)
    if (!e) HS_CUDA_TRY(cudaEventCreate(&e));
  HS_CUDA_TRY(cudaEventRecord(p->real_ev[0], st));
  HS_CUDA_TRY(hs_launch_embed2d(H, N_G, p->Hc, N_G, N_G, N_G, st));
  HS_CUDA_TRY(hs_launch_embed2d(S, N_G, p->Sc, N_G, N_G, N_G, st));
  const int rc = reduce_locked(p, p->Hc, p->Sc, N_G, info);
  if (rc) return rc;  // HS_ENOTPD included: H and S are left unchanged
  HS_CUDA_TRY(hs_launch_real_part(p->Hc, N_G, H, N_G, N_G, st));
  HS_CUDA_TRY(hs_launch_real_part(p->Sc, N_G, S, N_G, N_G, st));
  HS_CUDA_TRY(cudaEventRecord(p->real_ev[1], st));
  HS_CUDA_TRY(cudaStreamSynchronize(st));
  if (info) {  // the whole call's device time: the embedding and the copies back included
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->real_ev[0], p->real_ev[1]) == cudaSuccess)
      info->ms_total = ms;
    else
      cudaGetLastError();
  }
  return HS_OK;
}
