// Internal declarations shared by the split-precision translation units (not part
// of the ABI):
//   k_split.cu     the slice-GEMM kernel (contractions and per-atom products) and its
//                  launches;
//   k_slice.cu     the slicers (operands and per-atom operators to BF16 slices);
//   split_tune.cu  the autotuner of the launch knobs and the test-only stall switch;
//   split_plan.cu  tensor maps, slice workspaces and the assembly's launch sequence;
//   split_reduce.cu the slice-path products of the generalized-eigenproblem reduction.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <functional>

#include "plan.h"

namespace hs_split {

constexpr int BM = 128;        // complex rows per tile (MMA M)
constexpr int BNC = 64;        // complex columns per tile
constexpr int BN = 2 * BNC;    // MMA N (Re | Im)
constexpr int KB = 16;         // real K per pipeline stage (= one MMA K step)
constexpr int WIN = 8;         // stages per exact window (128 real K)
constexpr int ROWS_ALIGN = 128;
constexpr int kMaxBatch = 16;                 // requests per grouped per-atom launch
constexpr int kMaxMaps = 2 + 2 * kMaxBatch;   // >= 13 for a contraction
constexpr int kMaxJobs = 7;
constexpr int TILE_BYTES = 64 * KB * 2;  // one 64-row TMA box: 2 KB
constexpr int NUM_DRAIN_WARPS = 16;     // four per TMEM lane quarter
constexpr int NUM_THREADS = 64 + 32 * NUM_DRAIN_WARPS;  // warp 0 TMA, warp 1 MMA, then drain
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded waits: 2 s
// contraction epilogue staging in the (then idle) stage ring: (hi, lo) float2 as
// [2 strips x 64 columns][128 rows], plus 128 row and 128 column exponents
constexpr int STAGING_CONTRACT = 2 * 64 * 128 * 8 + 256 * 4;

// The _R modes are the real-symmetric variant (real A, B, T, U; H, S real symmetric,
// Sec. 1.1): operands hold one real K position per row, contraction tiles are
// 128 x 128 real outputs (B rows = 128 columns of R'), operator rows n = L.
enum { MODE_CONTRACT = 0, MODE_ATOMS = 1, MODE_CONTRACT_R = 2, MODE_ATOMS_R = 3 };
__host__ __device__ constexpr bool is_contract(int mode) { return (mode & 1) == 0; }
__host__ __device__ constexpr bool is_real(int mode) { return mode >= 2; }

struct SplitSeg {
  int mL, mR;       // tensor maps: L' as the left operand, R as the right one
                    // (complex: its plain and rotated slices, interleaved by plane)
  int kblocks;      // stages of KB real K
  const int* eL;    // exponents of the L source columns
  const int* eR;    // exponents of the R source columns
};

// One request of a grouped per-atom launch.
struct AtomsReq {
  int mA, mB;         // coefficient slice maps (plain) of this request
  const int* eA;      // column exponents of its A, B slices
  const int* eB;
  double2* Z;         // outputs, column-major, leading dimension AtomsArgs::ld
  double2* W2;
  int N_G;
  int ngblk;          // 128-row blocks of G
  int tile0;          // first CTA index of this request in the grouped grid
};

struct AtomsArgs {
  AtomsReq rq[kMaxBatch];
  int nreq;
  int mOp[2];             // operator slice maps: [0] Z job, [1] W2 job (shared by requests)
  const int* eOp[2];      // operator row exponents [a][n_pad]
  const int* slot;        // W2 slot of each atom
  int ld;
  int N_A, N_L, P;        // P: operator K per part (an atom's widest K block range)
  int n_pad, ntile;
};

struct SplitParams {
  CUtensorMap maps[kMaxMaps];
  SplitSeg seg[kMaxSeg];
  int nseg;
  int s;          // slices
  int n_stage;    // pipeline depth
  int N_G, ldC, nbj;
  int nbi, band;   // contraction: 128-row blocks, row blocks per band of the tile order
  int bi0;         // contraction: first row block of this launch (tiles of rows [bi0, nbi))
  int ntiles;      // tiles of the launch; a CTA runs tiles blockIdx.x, + gridDim.x, ...
  int rows_pad;   // slice p of a coefficient-side array starts at row p * rows_pad
  double2* C;
  int* err;
  int stall;  // test only: the producer arms no stage and issues no copy, so the MMA
              // thread's and the drain's waits run out (failure-path test)
  AtomsArgs at;
};

struct SliceJob {
  const double2* X;  // source: nblk * N_L complex rows x N_G, column-major, ld ldX
  const double* u;   // optional real row weight (the U norms), may be null
  uint16_t* plain;   // [s][rows_pad][kpad] BF16 slices of (re, im) pairs, or with rot
                     // [s][2][rows_pad][kpad]: (re, im) and (im, -re) slices interleaved
  int rot;           // nonzero: also write the (im, -re) slices
  int* expo;         // [rows_pad] column exponents
  int ldX, nblk;
};
struct SliceParams {
  SliceJob job[kMaxJobs];
  int s, N_G, rows_pad, N_L;
  int g0;  // first operand column of this launch (block x slices column g0 + x)
};


// ------------------------------------------------------------------ geometry
// Rows (operand columns g) of a slice array: whole 128-row blocks; 256 for real plans,
// whose contraction column pairs span 256 columns.
inline int rows_pad_of(int N_G, bool real = false) {
  const int al = real ? 2 * ROWS_ALIGN : ROWS_ALIGN;
  return ((N_G + al - 1) / al) * al;
}
// Packed real K of a source of nblk blocks of N_L rows (whole 16-wide blocks): two
// positions per complex row, one per real row.
inline int kpad_of(int nblk, int N_L, bool real = false) {
  return (((real ? 1 : 2) * nblk * N_L + KB - 1) / KB) * KB;
}
// Real K of one part of a per-atom operator: the most 16-wide K blocks any atom's
// rows [pr a N_L, pr (a+1) N_L) of the packed layout touch (pr positions per row).
inline int op_part_k(int N_A, int N_L, bool real = false) {
  const int pr = real ? 1 : 2;
  int nkb = 0;
  for (int a = 0; a < N_A; ++a)
    nkb = std::max(nkb, (pr * (a + 1) * N_L + KB - 1) / KB - (pr * a * N_L) / KB);
  return nkb * KB;
}
// Operator rows (2 N_L real rows; N_L for real plans) padded to whole 128-row tiles.
inline int op_rows_pad(int N_L, bool real = false) {
  return (((real ? 1 : 2) * N_L + BN - 1) / BN) * BN;
}

// ------------------------------------------------------------------ host helpers
// k_split.cu: one slice-GEMM launch (grid CTAs, smem bytes of dynamic shared memory),
// and the grouped per-atom launch as the kernel node of a captured graph
int launch_gemm(int mode, int s, int grid, size_t smem, cudaStream_t st, const SplitParams& P);
int graph_launch_atoms(AtomsGraph& G, int s, int grid, size_t smem, cudaStream_t st,
                       const SplitParams& P);
// k_slice.cu: slice nj jobs over operand columns [g0, g0 + ng) (ng < 0: up to rows_pad),
// and the per-atom operators (job 0: MZ, job 1: M2) of one factorisation
int slice_launch(SliceParams& sp, int nj, int s, int N_G, int rp, int N_L, bool real,
                 cudaStream_t st, int g0 = 0, int ng = -1, int threads = 256);
int slice_op_launch(const double2* M, int job, int N_A, int N_L, int Pk, int n_pad, int s,
                    uint16_t* out, int* expo, bool real, cudaStream_t st);
// split_tune.cu
bool stall_injection();
size_t smem_for(int mode, int n_stage, int stage_bytes);
int tuned_depth(int mode, int s, int N_L, int N_G, int max_depth, bool allow, cudaStream_t st,
                const std::function<int(int)>& trial);
int contract_band(int mode = 0, int s = 0, int N_L = 0, int N_G = 0);
int tuned_band(int mode, int s, int N_L, int N_G, bool allow, cudaStream_t st,
               const std::function<int(int)>& trial);
int slice_threads(bool real, int s, int N_L, int N_G, bool allow, cudaStream_t st,
                  const std::function<int(int)>& trial);
// split_plan.cu: tensor maps over blocked slice arrays
PFN_cuTensorMapEncodeTiled_v12000 get_encode();
bool encode_tiles(CUtensorMap* m, const uint16_t* base, int NKB, int NRB, int planes,
                  size_t plane_tiles, int box_rb, int box_planes);
bool encode_left(CUtensorMap* m, const uint16_t* base, int NKB, int NRB, int s, bool rot);
bool encode_right(CUtensorMap* m, const uint16_t* base, int NKB, int NRB, int s, bool rot);

}  // namespace hs_split
