// Autotuner of the split kernels' launch knobs and the test-only stall switch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "split_common.h"

namespace hs_split {

// Test-only stall injection (HS_TEST_STALL=1): every slice-GEMM launch arms no stage and
// issues no copy, so its bounded waits give up (2 s) and the kernel sets the device error
// word and returns (the host sees HS_EDEVICE).  Read at every launch.
bool stall_injection() {
  const char* e = std::getenv("HS_TEST_STALL");
  return e && e[0] == '1';
}

// ---------------------------------------------------------------- autotuner
// Launch knobs tuned on the real work: the first synchronous assembly with an untuned
// key times every candidate value (the trial launches compute the same result as the
// final one) and keeps the fastest; a candidate other than the first must win by 2 %.
//  * ring depth (TMA pipeline stages) of each kernel mode, key "mode:s:N_L:bucket";
//  * the contraction's band width (row blocks per band of its tile order, which sets
//    how compact the block of tiles resident at one time is and so the L2 reuse of
//    the slice boxes), key "band:mode:s:N_L:bucket", candidates 8, 4, 16, 32;
//  * the slicer's block size (threads per operand column), key
//    "slice:real:s:N_L:bucket", candidates 256, 128.
// bucket = N_G / 1024 rounded up.  Serving requests use tuned values when there are
// some and the defaults otherwise.  HS_AUTOTUNE=0 disables tuning; HS_TUNE_CACHE=<file>
// loads (whenever the name changes) and appends "key value" lines.  The per-atom kernel's grid is not a knob: its
// ring fills an SM's shared memory, so it runs one CTA per SM by construction.
namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
std::string g_tune_path;  // the HS_TUNE_CACHE file read last ("" = none yet)

std::string tune_key(int mode, int s, int N_L, int N_G) {
  return std::to_string(mode) + ":" + std::to_string(s) + ":" + std::to_string(N_L) + ":" +
         std::to_string((N_G + 1023) / 1024);
}

// Reads the cache file named by HS_TUNE_CACHE whenever that name changes (its values
// override the ones in memory).
void tune_load_locked() {
  const char* path = std::getenv("HS_TUNE_CACHE");
  if (!path || g_tune_path == path) return;
  g_tune_path = path;
  std::FILE* f = std::fopen(path, "r");
  if (!f) return;
  char key[128];
  int v;
  while (std::fscanf(f, "%127s %d", key, &v) == 2) g_tune[key] = v;
  std::fclose(f);
}

void tune_store_locked(const std::string& key, int v) {
  g_tune[key] = v;
  const char* path = std::getenv("HS_TUNE_CACHE");
  if (!path) return;
  std::FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d\n", key.c_str(), v);
  std::fclose(f);
}

}  // namespace

size_t smem_for(int mode, int n_stage, int stage_bytes) {
  const size_t ring = (size_t)n_stage * stage_bytes;
  return (is_contract(mode) ? std::max(ring, (size_t)STAGING_CONTRACT) : ring) + 1024 + 256;
}

namespace {

// The cached value of `key` if any; else, when tuning is allowed, the fastest of
// `cand` (cand[0] is the default) timed with `trial(value)`, which enqueues the real
// work; else cand[0].  `found` tells whether the value came from the cache.
int tuned_choice(const std::string& key, const std::vector<int>& cand, bool allow,
                 cudaStream_t st, const std::function<int(int)>& trial, bool* found = nullptr) {
  if (found) *found = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      if (found) *found = true;
      return it->second;
    }
  }
  const char* env = std::getenv("HS_AUTOTUNE");
  if (!allow || cand.size() < 2 || (env && env[0] == '0') || stall_injection()) return cand[0];
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cand[0];
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cand[0];
  }
  int best = cand[0];
  float best_ms = 1e30f;
  for (int v : cand) {
    float ms = 0.f;
    if (cudaEventRecord(e0, st) != cudaSuccess || trial(v) != HS_OK ||
        cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    if (ms < 0.98f * best_ms) {  // a later candidate must win clearly
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_store_locked(key, best);
  return best;
}

}  // namespace

// Depth for this launch; `trial(depth)` enqueues the real work with that depth.
int tuned_depth(int mode, int s, int N_L, int N_G, int max_depth, bool allow, cudaStream_t st,
                const std::function<int(int)>& trial) {
  std::vector<int> cand;
  for (int d = max_depth; d >= 2; --d) cand.push_back(d);
  const int v = tuned_choice(tune_key(mode, s, N_L, N_G), cand, allow, st, trial);
  return std::min(std::max(v, 2), max_depth);
}

// Row blocks per band of the contraction's tile order: tuned per key (8 by default:
// 152 resident CTAs then span about 8 row blocks x 19 column blocks); HS_BAND > 0 fixes it.
static int band_override() {
  static const int band = []() {
    const char* e = std::getenv("HS_BAND");
    const int v = e ? std::atoi(e) : 0;
    return v >= 1 ? v : 0;
  }();
  return band;
}
int contract_band(int mode, int s, int N_L, int N_G) {
  if (band_override()) return band_override();
  if (s == 0) return 8;
  bool found = false;
  const int v = tuned_choice("band:" + tune_key(mode, s, N_L, N_G), {8}, false, nullptr,
                             [](int) { return HS_OK; }, &found);
  return found && v >= 1 ? v : 8;
}
int tuned_band(int mode, int s, int N_L, int N_G, bool allow, cudaStream_t st,
               const std::function<int(int)>& trial) {
  if (band_override()) return band_override();
  const int v = tuned_choice("band:" + tune_key(mode, s, N_L, N_G), {8, 4, 16, 32}, allow, st,
                             trial);
  return v >= 1 ? v : 8;
}

// Threads per slicer block (one block per operand column).
int slice_threads(bool real, int s, int N_L, int N_G, bool allow, cudaStream_t st,
                  const std::function<int(int)>& trial) {
  const int v = tuned_choice("slice:" + std::to_string(real ? 1 : 0) + ":" + std::to_string(s) +
                                 ":" + std::to_string(N_L) + ":" +
                                 std::to_string((N_G + 1023) / 1024),
                             {256, 128}, allow, st, trial);
  return v == 128 ? v : 256;
}


}  // namespace hs_split
