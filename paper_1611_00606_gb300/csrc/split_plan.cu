// Split-precision form, host side of the assembly: tensor maps over the blocked slice
// arrays, the slice workspaces and the launch sequence of one k-point (slice the
// inputs, the per-atom products, slice their outputs, the S and H contractions).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "split_common.h"

using namespace hs_split;

namespace hs_split {


PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000)p;
    cudaGetLastError();
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

// Tensor map over a blocked slice array: dims (16 elements, 64 rows, NKB K blocks,
// NRB row blocks, planes `plane_tiles` tiles of 2 KB apart), box (16, 64, 1, box_rb,
// box_planes): every (row block, plane) of a box is one contiguous 2 KB tile, so a box
// lands in shared memory as [plane][row block] 2 KB tiles.
bool encode_tiles(CUtensorMap* m, const uint16_t* base, int NKB, int NRB, int planes,
                  size_t plane_tiles, int box_rb, int box_planes) {
  auto fn = get_encode();
  if (!fn) return false;
  if (box_rb < 1 || box_rb > NRB || box_planes < 1 || box_planes > planes) return false;
  cuuint64_t dims[5] = {(cuuint64_t)KB, 64u, (cuuint64_t)NKB, (cuuint64_t)NRB, (cuuint64_t)planes};
  cuuint64_t strides[4] = {(cuuint64_t)KB * 2, (cuuint64_t)TILE_BYTES,
                           (cuuint64_t)NKB * TILE_BYTES, (cuuint64_t)plane_tiles * TILE_BYTES};
  cuuint32_t box[5] = {(cuuint32_t)KB, 64u, 1u, (cuuint32_t)box_rb, (cuuint32_t)box_planes};
  cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Maps over the slices of one operand source with NKB K blocks and NRB 64-row blocks.
// A source with a rotated copy stores plain and rotated slices interleaved by plane
// (plane 2p: slice p of (re, im) pairs, plane 2p + 1: slice p of (im, -re) pairs).
//  * left role: the s plain slices of two row blocks (128 rows) per box;
//  * right role, complex: the plain and rotated slices of one row block (64 columns)
//    per box (2 s planes); right role, real: as the left role (128 columns).
bool encode_left(CUtensorMap* m, const uint16_t* base, int NKB, int NRB, int s, bool rot) {
  const size_t plane = (size_t)NRB * NKB * (rot ? 2 : 1);
  return encode_tiles(m, base, NKB, NRB, s, plane, 2, s);
}
bool encode_right(CUtensorMap* m, const uint16_t* base, int NKB, int NRB, int s, bool rot) {
  if (!rot) return encode_left(m, base, NKB, NRB, s, false);
  return encode_tiles(m, base, NKB, NRB, 2 * s, (size_t)NRB * NKB, 1, 2 * s);
}


}  // namespace hs_split

// Blocks (of N_L complex rows) of each source and whether it needs the rotated copy.
static void source_shape(int src, int N_A, int n_fail, bool real, int& nblk, bool& rot) {
  rot = !real && (src != SRC_AF);
  nblk = (src == SRC_AF || src == SRC_X) ? n_fail : N_A;
}

size_t hs_plan_s::split_ws_bytes(int N_G, int n_fail) const {
  if (precision != HS_SPLIT_BF16) return 0;
  const int nf = n_fail > 0 ? n_fail : 1;
  const int rp = rows_pad_of(N_G, real);
  size_t b = 0;
  for (int src = 0; src < NSRC; ++src) {
    int nblk;
    bool rot;
    source_shape(src, N_A, nf, real, nblk, rot);
    const size_t one = (size_t)slices * rp * kpad_of(nblk, N_L, real) * 2;
    b += (rot ? 2 : 1) * one + sizeof(int) * rp;
  }
  return b;
}

int hs_plan_s::split_ws_alloc(Workspace& w, int N_G, int n_fail, cudaStream_t st, bool async) {
  if (precision != HS_SPLIT_BF16) return HS_OK;
  if (!get_encode()) return HS_ECUDA;
  const int rp = rows_pad_of(N_G, real);
  auto al = [&](void** ptr, size_t bytes) -> bool {
    return (async ? hs_malloc_async(ptr, bytes, st, hs_serve_pool(this)) : cudaMalloc(ptr, bytes)) ==
           cudaSuccess;
  };
  for (int src = 0; src < NSRC; ++src) {
    int nblk;
    bool rot;
    source_shape(src, N_A, n_fail, real, nblk, rot);
    const size_t one = (size_t)slices * rp * kpad_of(nblk, N_L, real) * 2;
    if (!al((void**)&w.sb[src].plain, (rot ? 2 : 1) * one)) return HS_ENOMEM;
    w.sb[src].rot = rot;
    if (!al((void**)&w.sb[src].expo, sizeof(int) * rp)) return HS_ENOMEM;
  }
  return HS_OK;
}

size_t hs_plan_s::split_fixed_bytes() const {
  if (precision != HS_SPLIT_BF16) return 0;
  const size_t P = (size_t)op_part_k(N_A, N_L, real), np = (size_t)op_rows_pad(N_L, real);
  return (size_t)N_A * slices * np * (3 * P) * 2 + 2 * sizeof(int) * N_A * np;
}

int hs_plan_s::split_plan_alloc() {
  if (precision != HS_SPLIT_BF16) return HS_OK;
  if (!get_encode()) return HS_ECUDA;
  const size_t P = (size_t)op_part_k(N_A, N_L, real), np = (size_t)op_rows_pad(N_L, real);
  const size_t zb = (size_t)N_A * slices * np * 2 * P * 2, wb = zb / 2;
  if (cudaMalloc((void**)&op_slices[0], zb) != cudaSuccess ||
      cudaMalloc((void**)&op_slices[1], wb) != cudaSuccess ||
      cudaMalloc((void**)&op_expo[0], sizeof(int) * N_A * np) != cudaSuccess ||
      cudaMalloc((void**)&op_expo[1], sizeof(int) * N_A * np) != cudaSuccess) {
    cudaGetLastError();
    return HS_ENOMEM;
  }
  return HS_OK;
}

void hs_plan_s::split_plan_release() {
  for (int j = 0; j < 2; ++j) {
    if (op_slices[j]) cudaFree(op_slices[j]);
    if (op_expo[j]) cudaFree(op_expo[j]);
    op_slices[j] = nullptr;
    op_expo[j] = nullptr;
  }
}

// Slice MZ and M2 (k-independent) after every factorisation.
int hs_plan_s::split_factor(cudaStream_t st) {
  if (precision != HS_SPLIT_BF16) return HS_OK;
  const int P = op_part_k(N_A, N_L, real), np = op_rows_pad(N_L, real);
  for (int job = 0; job < 2; ++job) {
    const double2* M = job == 0 ? MZ : M2;
    const int rc = slice_op_launch(M, job, N_A, N_L, P, np, slices, op_slices[job], op_expo[job],
                                   real, st);
    if (rc) return rc;
  }
  return HS_OK;
}


int hs_plan_s::split_geometry(int& n_stage, size_t& smem) const {
  const int stage_bytes = 4 * slices * TILE_BYTES;
  const int budget = 227 * 1024 - 1024 - 256;
  n_stage = budget / stage_bytes;
  if (n_stage > 8) n_stage = 8;
  if (n_stage < 2) return HS_EINVAL;
  smem = smem_for(MODE_CONTRACT, n_stage, stage_bytes);
  return HS_OK;
}

static void slice_job(SliceParams& sp, int& nj, Workspace& w, int src, const double2* X, int ldX,
                      int nblk, const double* u) {
  SliceBuf& b = w.sb[src];
  sp.job[nj++] = SliceJob{X, u, b.plain, b.rot, b.expo, ldX, nblk};
}

// 1. slice the inputs A, U.B, B of one k-point (tune: time the slicer's block sizes on
//    this work if its key is untuned)
int hs_plan_s::split_inputs(const double2* A, const double2* B, int ldAB, const double* U,
                            int N_G, Workspace& w, cudaStream_t st, int g0, int ng, bool tune) {
  const int rp = rows_pad_of(N_G, real);
  if (rows_pad_of(w.N_G, real) < rp || w.n_fail < N_f || !w.sb[SRC_A].plain) return HS_EINVAL;
  SliceParams sp{};
  int nj = 0;
  slice_job(sp, nj, w, SRC_A, A, ldAB, N_A, nullptr);
  slice_job(sp, nj, w, SRC_UB, B, ldAB, N_A, U);
  slice_job(sp, nj, w, SRC_B, B, ldAB, N_A, nullptr);
  const int threads = slice_threads(real, slices, N_L, N_G, tune && g0 == 0 && ng < 0, st,
                                    [&](int t) {
                                      return slice_launch(sp, nj, slices, N_G, rp, N_L, real, st,
                                                          g0, ng, t);
                                    });
  return slice_launch(sp, nj, slices, N_G, rp, N_L, real, st, g0, ng, threads);
}

// 2. per-atom products of up to kMaxBatch k-points in one grouped launch: Z and
//    W2 = [Y; X] in FP64.  With `graph`, the launch is the (re-parameterised) kernel
//    node of the plan's captured graph.
int hs_plan_s::split_atoms(const AtomsJob* jobs, int n, cudaStream_t st, AtomsGraph* graph) {
  if (n < 1 || n > kMaxBatch) return HS_EINVAL;
  const int s = slices, Pp = op_part_k(N_A, N_L, real), np = op_rows_pad(N_L, real);
  const int mode = real ? MODE_ATOMS_R : MODE_ATOMS;
  int n_stage;
  size_t smem;
  int rc = split_geometry(n_stage, smem);
  if (rc) return rc;
  SplitParams* PA = new (std::nothrow) SplitParams;
  if (!PA) return HS_ENOMEM;
  std::memset(PA, 0, sizeof(*PA));
  AtomsArgs& at = PA->at;
  // operator slices [a][p][n_pad][Kop]: the right operand, two row blocks x s planes
  bool ok = encode_tiles(&PA->maps[0], op_slices[0], 2 * Pp / KB, np / 64, N_A * s,
                         (size_t)(np / 64) * (2 * Pp / KB), 2, s) &&
            encode_tiles(&PA->maps[1], op_slices[1], Pp / KB, np / 64, N_A * s,
                         (size_t)(np / 64) * (Pp / KB), 2, s);
  at.mOp[0] = 0;
  at.mOp[1] = 1;
  int grid = 0;
  for (int r = 0; r < n && ok; ++r) {
    Workspace& w = *jobs[r].w;
    const int rp = rows_pad_of(jobs[r].N_G, real);
    AtomsReq& R = at.rq[r];
    R.mA = 2 + 2 * r;
    R.mB = 3 + 2 * r;
    const int nkb = kpad_of(N_A, N_L, real) / KB;
    ok = encode_left(&PA->maps[R.mA], w.sb[SRC_A].plain, nkb, rp / 64, s, w.sb[SRC_A].rot) &&
         encode_left(&PA->maps[R.mB], w.sb[SRC_B].plain, nkb, rp / 64, s, w.sb[SRC_B].rot);
    R.eA = w.sb[SRC_A].expo;
    R.eB = w.sb[SRC_B].expo;
    R.Z = w.Z;
    R.W2 = w.W2;
    R.N_G = jobs[r].N_G;
    R.ngblk = rp / BM;
    R.tile0 = grid;
    grid += R.ngblk * (np / BN) * 2 * N_A;
  }
  if (!ok) {
    delete PA;
    return HS_ECUDA;
  }
  at.nreq = n;
  // persistent: one CTA per SM, each running every gridDim.x-th tile
  PA->ntiles = grid;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
      delete PA;
      return HS_ECUDA;
    }
    grid = std::min(grid, nsm);
  }
  at.eOp[0] = op_expo[0];
  at.eOp[1] = op_expo[1];
  at.slot = slot_d;
  at.ld = N_A * N_L;
  at.N_A = N_A;
  at.N_L = N_L;
  at.P = Pp;
  at.n_pad = np;
  at.ntile = np / BN;
  PA->s = s;
  PA->err = err_d;
  const int stage_bytes = 4 * s * TILE_BYTES;
  const int depth = tuned_depth(mode, s, N_L, jobs[0].N_G, n_stage, graph == nullptr, st,
                                [&](int d) {
                                  PA->n_stage = d;
                                  return launch_gemm(mode, s, grid, smem_for(mode, d, stage_bytes),
                                                     st, *PA);
                                });
  PA->n_stage = depth;
  smem = smem_for(mode, depth, stage_bytes);
  rc = graph ? graph_launch_atoms(*graph, s, grid, smem, st, *PA)
             : launch_gemm(mode, s, grid, smem, st, *PA);
  delete PA;
  return rc;
}

// 3. gather A_f, slice the per-atom outputs, and the two stacked contractions
int hs_plan_s::split_outputs(const double2* A, int ldAB, int N_G, double2* H, double2* S,
                             Workspace& w, cudaStream_t st, bool timed, cudaEvent_t s_done,
                             bool skip_S, bool mirror) {
  const int K = N_A * N_L;
  const int N_h = N_A - N_f;
  const int s = slices;
  const int rp = rows_pad_of(N_G, real);
  const int mode = real ? MODE_CONTRACT_R : MODE_CONTRACT;
  int n_stage;
  size_t smem;
  int rc = split_geometry(n_stage, smem);
  if (rc) return rc;
  if (real)
    HS_CUDA_TRY(hs_launch_gather_af_real((const double*)A, ldAB, fail_list_d, N_f, N_L, N_G,
                                         (double*)w.AF, st));
  else
    HS_CUDA_TRY(hs_launch_gather_af(A, ldAB, fail_list_d, N_f, N_L, N_G, w.AF, st));
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[4], st));
  {
    SliceParams sp{};
    int nj = 0;
    slice_job(sp, nj, w, SRC_Z, w.Z, K, N_A, nullptr);
    if (N_h > 0) slice_job(sp, nj, w, SRC_Y, w.W2, K, N_h, nullptr);
    if (N_f > 0) {
      slice_job(sp, nj, w, SRC_AF, w.AF, N_f * N_L, N_f, nullptr);
      const double2* X = real ? (const double2*)((const double*)w.W2 + (size_t)N_h * N_L)
                              : w.W2 + (size_t)N_h * N_L;
      slice_job(sp, nj, w, SRC_X, X, K, N_f, nullptr);
    }
    const int threads = slice_threads(real, s, N_L, N_G, false, st, [](int) { return HS_OK; });
    rc = slice_launch(sp, nj, s, N_G, rp, N_L, real, st, 0, -1, threads);
    if (rc) return rc;
  }
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[5], st));

  SplitParams* PP = new (std::nothrow) SplitParams;
  if (!PP) return HS_ENOMEM;
  SplitParams& P = *PP;
  std::memset(&P, 0, sizeof(P));
  int map_of[NSRC][2];
  int nm = 0;
  auto add_map = [&](int src, int nblk) -> bool {  // [0]: left role, [1]: right role
    SliceBuf& b = w.sb[src];
    const int nkb = kpad_of(nblk, N_L, real) / KB;
    map_of[src][0] = nm;
    if (!encode_left(&P.maps[nm++], b.plain, nkb, rp / 64, s, b.rot)) return false;
    map_of[src][1] = nm;
    return encode_right(&P.maps[nm++], b.plain, nkb, rp / 64, s, b.rot);
  };
  bool ok = add_map(SRC_A, N_A) && add_map(SRC_UB, N_A) && add_map(SRC_Z, N_A) &&
            add_map(SRC_B, N_A);
  if (N_h > 0) ok = ok && add_map(SRC_Y, N_h);
  if (N_f > 0) ok = ok && add_map(SRC_AF, N_f) && add_map(SRC_X, N_f);
  if (!ok) {
    delete PP;
    return HS_ECUDA;
  }
  P.s = s;
  P.n_stage = n_stage;
  P.N_G = N_G;
  P.ldC = N_G;
  P.nbj = (N_G + (real ? BN : BNC) - 1) / (real ? BN : BNC);  // output column tiles
  P.rows_pad = rp;
  P.err = err_d;
  const int nbi = (N_G + BM - 1) / BM;
  int tiles = 0;
  for (int b = 0; b < nbi; ++b)  // CTA pairs: column pair c from row block c (2c if real)
    tiles += 2 * std::min((real ? b / 2 : b) + 1, (P.nbj + 1) / 2);
  P.nbi = nbi;
  P.band = contract_band(mode, s, N_L, N_G);
  P.ntiles = tiles;  // one tile per CTA
  auto seg = [&](int srcL, int srcR, int nblk) {
    SplitSeg g;
    g.mL = map_of[srcL][0];
    g.mR = map_of[srcR][1];
    g.kblocks = kpad_of(nblk, N_L, real) / KB;
    g.eL = w.sb[srcL].expo;
    g.eR = w.sb[srcR].expo;
    return g;
  };
  // S = A^H A + (UB)^H (UB)
  P.nseg = 2;
  P.seg[0] = seg(SRC_A, SRC_A, N_A);
  P.seg[1] = seg(SRC_UB, SRC_UB, N_A);
  P.C = S;
  {
    const int stage_bytes = 4 * s * TILE_BYTES;
    // trials re-run the S contraction: not when the caller already made S (its mirror
    // may be running on another stream)
    const bool tune = timed && !skip_S;
    const int depth = tuned_depth(mode, s, N_L, N_G, n_stage, tune, st, [&](int d) {
      P.n_stage = d;
      return launch_gemm(mode, s, tiles, smem_for(mode, d, stage_bytes), st, P);
    });
    P.n_stage = depth;
    smem = smem_for(mode, depth, stage_bytes);
    P.band = tuned_band(mode, s, N_L, N_G, tune, st, [&](int b) {
      P.band = b;
      return launch_gemm(mode, s, tiles, smem, st, P);
    });
  }
  if (!skip_S) rc = launch_gemm(mode, s, tiles, smem, st, P);
  if (rc == HS_OK && !skip_S && mirror) {  // S is final once mirrored: it can leave while H runs
    const cudaError_t e = real ? hs_launch_mirror_real((double*)S, N_G, N_G, st)
                               : hs_launch_mirror(S, N_G, N_G, st);
    if (e != cudaSuccess || (s_done && cudaEventRecord(s_done, st) != cudaSuccess)) rc = HS_ECUDA;
  }
  if (rc == HS_OK && timed && cudaEventRecord(ev[6], st) != cudaSuccess) rc = HS_ECUDA;
  if (rc == HS_OK) {
    // H = Z^H B + B^H Z + Y^H Y + A_f^H X_f
    int n = 0;
    P.seg[n++] = seg(SRC_Z, SRC_B, N_A);
    P.seg[n++] = seg(SRC_B, SRC_Z, N_A);
    if (N_h > 0) P.seg[n++] = seg(SRC_Y, SRC_Y, N_h);
    if (N_f > 0) P.seg[n++] = seg(SRC_AF, SRC_X, N_f);
    P.nseg = n;
    P.C = H;
    rc = launch_gemm(mode, s, tiles, smem, st, P);
    if (rc == HS_OK && timed && cudaEventRecord(ev[7], st) != cudaSuccess) rc = HS_ECUDA;
  }
  delete PP;
  return rc;
}

// The S contraction restricted to the lower-triangle tiles of row blocks [bi0, bi1):
// they read only A and U.B slice rows below 128 * bi1, so a caller that slices column
// chunks as they arrive can run them before the later chunks exist.
int hs_plan_s::split_contract_S_rows(int N_G, double2* S, Workspace& w, cudaStream_t st, int bi0,
                                     int bi1) {
  const int s = slices;
  const int rp = rows_pad_of(N_G, real);
  const int mode = real ? MODE_CONTRACT_R : MODE_CONTRACT;
  const int nbi = (N_G + BM - 1) / BM;
  bi0 = std::max(bi0, 0);
  bi1 = std::min(bi1, nbi);
  if (bi1 <= bi0) return HS_OK;
  int n_stage;
  size_t smem;
  int rc = split_geometry(n_stage, smem);
  if (rc) return rc;
  SplitParams* PP = new (std::nothrow) SplitParams;
  if (!PP) return HS_ENOMEM;
  SplitParams& P = *PP;
  std::memset(&P, 0, sizeof(P));
  int map_of[2][2];
  int nm = 0;
  bool ok = true;
  for (int i = 0; i < 2 && ok; ++i) {
    SliceBuf& b = w.sb[i == 0 ? SRC_A : SRC_UB];
    const int nkb = kpad_of(N_A, N_L, real) / KB;
    map_of[i][0] = nm;
    ok = encode_left(&P.maps[nm++], b.plain, nkb, rp / 64, s, b.rot);
    map_of[i][1] = nm;
    ok = ok && encode_right(&P.maps[nm++], b.plain, nkb, rp / 64, s, b.rot);
  }
  if (!ok) {
    delete PP;
    return HS_ECUDA;
  }
  P.s = s;
  P.N_G = N_G;
  P.ldC = N_G;
  P.nbj = (N_G + (real ? BN : BNC) - 1) / (real ? BN : BNC);
  P.rows_pad = rp;
  P.err = err_d;
  int tiles = 0;
  for (int b = bi0; b < bi1; ++b) tiles += 2 * std::min((real ? b / 2 : b) + 1, (P.nbj + 1) / 2);
  P.bi0 = bi0;
  P.nbi = bi1;
  P.band = contract_band(mode, s, N_L, N_G);
  P.ntiles = tiles;
  for (int i = 0; i < 2; ++i) {
    SplitSeg& g = P.seg[i];
    g.mL = map_of[i][0];
    g.mR = map_of[i][1];
    g.kblocks = kpad_of(N_A, N_L, real) / KB;
    g.eL = g.eR = w.sb[i == 0 ? SRC_A : SRC_UB].expo;
  }
  P.nseg = 2;
  P.C = S;
  const int stage_bytes = 4 * s * TILE_BYTES;
  P.n_stage = tuned_depth(mode, s, N_L, N_G, n_stage, false, st, [](int) { return HS_OK; });
  rc = launch_gemm(mode, s, tiles, smem_for(mode, P.n_stage, stage_bytes), st, P);
  delete PP;
  return rc;
}

int hs_plan_s::split_enqueue(const double2* A, const double2* B, int ldAB, const double* U,
                             int N_G, double2* H, double2* S, Workspace& w, cudaStream_t st,
                             bool timed, cudaEvent_t s_done, bool presliced, bool mirror) {
  int rc = presliced ? HS_OK : split_inputs(A, B, ldAB, U, N_G, w, st, 0, -1, timed);
  if (rc) return rc;
  if (timed) HS_CUDA_TRY(cudaEventRecord(ev[9], st));
  AtomsJob job{&w, N_G};
  rc = split_atoms(&job, 1, st, nullptr);
  if (rc) return rc;
  return split_outputs(A, ldAB, N_G, H, S, w, st, timed, s_done, presliced, mirror);
}

