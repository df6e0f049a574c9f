// The plan object behind hs_plan_t (internal).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "hs_internal.h"

constexpr int kMaxNL = 168;       // packed lower triangle of T^AA fits in 227 KB smem
constexpr int kDefaultSlices = 5;
constexpr int kMaxSlices = 7;  // 7 + 9*(s-1) bits must fit an int64 digit word

struct SplitWork;   // k_split.cu
struct ServeState;  // serve.cu

struct hs_plan_s {
  std::mutex mu;
  int device = 0;
  int N_A = 0, N_L = 0, N_G_max = 0, precision = HS_FP64, slices = 0;
  size_t budget = 0;
  cudaStream_t stream = nullptr;

  // per-k-point workspace (FP64)
  double2* Z = nullptr;   // K x N_G_max   (Z_a stacked)
  double2* W2 = nullptr;  // K x N_G_max   (Y_HPD rows, then X_notHPD rows)
  double2* AF = nullptr;  // (N_f N_L) x N_G_max  (A_notHPD)
  int af_atoms = 0;

  // factor cache (k-independent)
  double2* M2 = nullptr;  // N_A x N_L x N_L : L_a^H or T^AA_a
  double2* MZ = nullptr;  // N_A x N_L x 2N_L : [T^BA_a | 1/2 T^BB_a]
  int* fail_d = nullptr;
  int* slot_d = nullptr;
  int* fail_list_d = nullptr;
  std::vector<int> fail_h;
  int N_f = 0;
  const void *tAA = nullptr, *tAB = nullptr, *tBB = nullptr;
  const void *host_tAA = nullptr, *host_tAB = nullptr, *host_tBB = nullptr;
  bool t_valid = false;
  double last_factor_ms = 0.0;

  int* err_d = nullptr;  // device error word (bounded waits)
  cudaEvent_t ev[10] = {};
  void* stage[6] = {};   // host-call staging: A, B, T, U, H, S

  SplitWork* split = nullptr;
  ServeState* serve = nullptr;

  size_t workspace_bytes(int N_G) const;
  size_t fixed_bytes() const;
  size_t split_bytes(int N_G) const;
  int split_alloc();
  void split_release();
  void release();
  int factor(const double2* T_AA, const double2* T_AB, const double2* T_BB);
  int enqueue(const double2* A, const double2* B, int ldAB, const double* U, int N_G, double2* H,
              double2* S, double2* Zw, double2* W2w, double2* AFw, cudaStream_t st, bool timed);
  int split_enqueue(const SegList& sS, const SegList& sH, int N_G, double2* H, double2* S,
                    cudaStream_t st, bool timed);
  int check_device_error();
  void fill_info(hs_info* info, bool factored);
  void serve_shutdown();
};
