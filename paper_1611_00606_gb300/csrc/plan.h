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
constexpr int kRedPanel = 128;  // hs_reduce, split plans: FP64 panel width

// Slice buffers of one operand source: s BF16 arrays [p][rows_pad][kpad] of
// (re, im) pairs and one exponent per row (= column of the operand).  With `rot`
// the same buffer also holds the slices of the (im, -re) pairs, interleaved by
// plane: plane 2p = plain slice p, plane 2p + 1 = rotated slice p (one 2 KB TMA
// tile row of the right operand then covers both).
struct SliceBuf {
  uint16_t* plain = nullptr;
  bool rot = false;
  int* expo = nullptr;
};
// Operand sources of the two contractions.
enum { SRC_A = 0, SRC_UB, SRC_Z, SRC_B, SRC_Y, SRC_AF, SRC_X, NSRC };

// Per-k-point device workspace.  The synchronous path owns one sized for
// N_G_max; every admitted serving request gets its own, sized exactly.
struct Workspace {
  double2* Z = nullptr;   // K x N_G (Z_a stacked)
  double2* W2 = nullptr;  // K x N_G (Y_HPD rows, then X_notHPD rows)
  double2* AF = nullptr;  // (N_f N_L) x N_G (A rows of failing atoms)
  int N_G = 0;            // capacity in columns
  int n_fail = 0;         // capacity of AF and of the A_f / X_f slices, in atoms
  SliceBuf sb[NSRC];      // split form only
  bool async = false;     // allocated with cudaMallocAsync (serving)
};

struct ServeState;  // serve.cu
struct AtomsGraph;  // k_split.cu: graph holding the grouped per-atom launch
AtomsGraph* hs_atoms_graph_new();
void hs_atoms_graph_free(AtomsGraph* a);
// One k-point of a grouped per-atom launch.
struct AtomsJob {
  Workspace* w;
  int N_G;
};
struct hs_plan_s;
// Stream-ordered pool for serving workspaces (null before the first hs_submit).
cudaMemPool_t hs_serve_pool(hs_plan_s* p);
// cudaMallocAsync from the serving pool when there is one.
inline cudaError_t hs_malloc_async(void** ptr, size_t bytes, cudaStream_t st, cudaMemPool_t pool) {
  return pool ? cudaMallocFromPoolAsync(ptr, bytes, pool, st) : cudaMallocAsync(ptr, bytes, st);
}

struct hs_plan_s {
  std::mutex mu;
  int device = 0;
  int N_A = 0, N_L = 0, N_G_max = 0, precision = HS_FP64, slices = 0;
  // HS_REAL plan (real-symmetric variant, hs_assemble_real): T embedded as complex for
  // the factorisation; the split form is native real (real Z, W2, A_f and slices), the
  // FP64 form runs the complex kernels on embedded A, B into complex H, S buffers
  bool real = false;
  double2* Tc = nullptr;                                          // 3 x N_A x N_L^2
  double2 *Ac = nullptr, *Bc = nullptr, *Hc = nullptr, *Sc = nullptr;  // FP64 real plans
  size_t budget = 0;
  cudaStream_t stream = nullptr;

  Workspace ws;  // synchronous calls

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
  bool factor_pending_info = false;  // hs_set_t ran since the last hs_assemble

  // split form: BF16 slices of MZ (job 0) and M2 (job 1), [a][p][n_pad][Kop], and
  // one exponent per (atom, operator row); refreshed with every factorisation
  uint16_t* op_slices[2] = {nullptr, nullptr};
  int* op_expo[2] = {nullptr, nullptr};

  int* err_d = nullptr;  // device error word (bounded waits)
  // hs_assemble_host: copy stream and S stream (created on first use) and their events
  cudaStream_t copy_stream = nullptr, s_stream = nullptr;
  cudaEvent_t copy_ev[10] = {};
  cudaEvent_t ev[10] = {};
  void* stage[6] = {};   // host-call staging: A, B, T, U, H, S
  // hs_reduce: W = L^{-1} and P (n x n each, n = red_cap), failure word, events
  double2 *red_W = nullptr, *red_P = nullptr;
  int red_cap = 0;
  int* red_fail = nullptr;
  cudaEvent_t red_ev[7] = {};
  cudaEvent_t real_ev[2] = {};  // hs_reduce_real: around its copies in and out
  // hs_reduce, split plans: slices of M = [L^{-H} | 0 | H] and of Z = H L^{-H} / 2,
  // 2 Z in FP64 (n x (n_pad + n)), the row weight 1/2; sized for red_split_cap
  SliceBuf red_M, red_Zs;
  double2* red_Z = nullptr;
  double* red_half = nullptr;
  int red_split_cap = 0;
  // the inverse's own scratch (it runs on s_stream beside the Cholesky): slices,
  // transposed L block, product; one event per Cholesky panel (its L columns final)
  SliceBuf red_M2;
  double2 *red_P2 = nullptr, *red_Z2 = nullptr;
  std::vector<cudaEvent_t> red_pev;

  ServeState* serve = nullptr;

  // workspace sizing and allocation (hs_api.cu / k_split.cu)
  size_t ws_bytes(int N_G, int n_fail) const;      // exact bytes of one workspace
  size_t split_ws_bytes(int N_G, int n_fail) const;
  int ws_alloc(Workspace& w, int N_G, int n_fail, cudaStream_t st, bool async);
  int split_ws_alloc(Workspace& w, int N_G, int n_fail, cudaStream_t st, bool async);
  void ws_free(Workspace& w, cudaStream_t st);
  size_t fixed_bytes() const;
  size_t split_fixed_bytes() const;
  int split_plan_alloc();
  void split_plan_release();
  int split_factor(cudaStream_t st);
  void release();
  int factor(const double2* T_AA, const double2* T_AB, const double2* T_BB);
  int factor_real(const double* T_AA, const double* T_AB, const double* T_BB);
  // bytes of one element of Z, W2, A_f: real doubles for real split plans
  size_t ws_elem() const { return real && precision == HS_SPLIT_BF16 ? 8 : 16; }
  // s_done (optional): recorded on st once S (mirrored) is final, while H is still being
  // computed; presliced (split form): the caller already sliced the inputs and contracted
  // and mirrored S (the host call's streamed path); mirror = false: the lower triangles of
  // H and S only, the upper triangles left as the contraction leaves them (partial sums
  // over an atom range, mirrored after they are added up)
  int enqueue(const double2* A, const double2* B, int ldAB, const double* U, int N_G, double2* H,
              double2* S, Workspace& w, cudaStream_t st, bool timed, cudaEvent_t s_done = nullptr,
              bool presliced = false, bool mirror = true);
  int split_enqueue(const double2* A, const double2* B, int ldAB, const double* U, int N_G,
                    double2* H, double2* S, Workspace& w, cudaStream_t st, bool timed,
                    cudaEvent_t s_done = nullptr, bool presliced = false, bool mirror = true);
  int split_geometry(int& n_stage, size_t& smem) const;
  // g0, ng: slice only operand columns [g0, g0 + ng) (ng < 0: every column and the zero
  // rows up to the padded row count)
  int split_inputs(const double2* A, const double2* B, int ldAB, const double* U, int N_G,
                   Workspace& w, cudaStream_t st, int g0 = 0, int ng = -1, bool tune = false);
  int split_atoms(const AtomsJob* jobs, int n, cudaStream_t st, AtomsGraph* graph);
  // also mirrors S (right after its contraction, then records s_done if given);
  // skip_S: S was already contracted and mirrored by the caller
  int split_outputs(const double2* A, int ldAB, int N_G, double2* H, double2* S, Workspace& w,
                    cudaStream_t st, bool timed, cudaEvent_t s_done = nullptr,
                    bool skip_S = false, bool mirror = true);
  // S contraction tiles of row blocks [bi0, bi1) only (no mirror)
  int split_contract_S_rows(int N_G, double2* S, Workspace& w, cudaStream_t st, int bi0,
                            int bi1);
  // hs_reduce's two-sided transform on the slice path: H <- B^H H B with B = L^{-H}
  // (n x n column-major, upper triangular); records `mid` between its two contractions
  int split_reduce_transform(const double2* B, double2* H, int n, cudaStream_t st,
                             cudaEvent_t mid);
  int split_reduce_alloc(int n);
  void split_reduce_release();
  // the Cholesky and the inverse of hs_reduce on split plans: FP64 panels of kRedPanel
  // columns (rows), trailing updates as slice contractions.  The Cholesky (scratch
  // red_M, red_P, red_Z) records red_pev[p] once panel p is factored; the inverse
  // (scratch red_M2, red_P2, red_Z2), on another stream, waits for it before block row p.
  int split_cholesky(double2* S, int n, int* fail, cudaStream_t st);
  int split_inverse(const double2* L, double2* W, int n, const int* fail, cudaStream_t st);
  // lower(X^H X) and A^H B for K-major operands on the slice path (slices in sb)
  int split_herk_lower(const double2* X, int ldX, int K, int nc, double2* out, SliceBuf& sb,
                       cudaStream_t st);
  int split_gemm_ahb(const double2* A, int ldA, int m, const double2* B, int ldB, int nc, int K,
                     double2* out, SliceBuf& sb, cudaStream_t st);
  int check_device_error();
  void fill_info(hs_info* info, bool factored);
  bool serve_busy();
  void serve_shutdown();
};
