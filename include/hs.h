/*
 * libhs -- GB300 (sm_103a) assembly of the FLAPW Hamiltonian H and overlap S
 * for one k-point.
 *
 *   H = sum_a A_a^H T^AA_a A_a + A_a^H T^AB_a B_a + B_a^H T^BA_a A_a + B_a^H T^BB_a B_a   (Eq. (h))
 *   S = sum_a A_a^H A_a + B_a^H U_a^H U_a B_a                                              (Eq. (s))
 *
 * Shapes (Sec. 2, after Eq. (s)): A_a, B_a in C^{N_L x N_G}; T_a in C^{N_L x N_L};
 * H, S in C^{N_G x N_G}; U_a diagonal.  K = N_A * N_L.
 *
 * Method (Algorithm 1, restated for the GPU):
 *   Z_a = T^BA_a A_a + 1/2 T^BB_a B_a,   H  = Z^H B + B^H Z          (first part of H)
 *   S   = A^H A + (U B)^H (U B)                                        (S)
 *   T^AA_a = C_a C_a^H (Cholesky): Y_a = C_a^H A_a,  H += Y^H Y         (second part of H)
 *   Cholesky fails:                X_a = T^AA_a A_a, H += A_a^H X_a
 * T^BA is not an input: Sec. 2 states T^BA = (T^AB)^H and that T^BB is Hermitian.
 *
 * ---------------------------------------------------------------------------
 * Memory layout (all matrices column-major, BLAS order; complex = interleaved
 * re, im doubles, layout-compatible with cuDoubleComplex / std::complex<double>):
 *   A, B    : K x N_G, leading dimension K.  Atom a owns rows [a*N_L, (a+1)*N_L).
 *   T_AA, T_AB, T_BB : N_A consecutive N_L x N_L column-major blocks (stride N_L^2).
 *             Only the LOWER triangle of T_AA and T_BB is read (zpotrf / zhemm
 *             semantics); T_AB is read in full.
 *   U       : N_A x N_L reals, U[a*N_L + L] is the diagonal entry of U_a.
 *   H, S    : N_G x N_G, leading dimension N_G.  Both triangles are written;
 *             the result is exactly Hermitian with exactly real diagonal.
 *
 * Ownership: the caller owns every input and output buffer.  Buffers must stay
 * valid and unmodified until the call that uses them completes (hs_assemble
 * returns, or hs_poll returns HS_OK for the ticket).  The plan owns its device
 * workspace and a cache of the factorised T^AA blocks, keyed by the T pointers:
 * after changing T contents in place, call hs_set_t() (or pass new pointers).
 *
 * Errors: functions return HS_OK (0) or a negative code; no partial output is
 * guaranteed after an error.  An atom whose Cholesky factorisation fails is NOT
 * an error: it takes the fallback product and is counted in hs_info.n_fallback.
 * Non-finite inputs are not checked and propagate as NaN.  Device-side waits
 * are bounded; an expired wait returns HS_EDEVICE instead of hanging.
 * Every entry point is thread-safe per plan (calls on one plan serialise).
 */
#ifndef HS_H_
#define HS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hs_plan_s* hs_plan_t;

/* One complex double, interleaved. */
typedef struct { double re, im; } hs_z;

enum {
  HS_OK = 0,
  HS_PENDING = 1,      /* hs_poll: ticket not finished yet */
  HS_EINVAL = -1,      /* bad argument (sizes, null pointers, unknown precision) */
  HS_ENOMEM = -2,      /* device allocation failed, or request above the HBM budget */
  HS_ECUDA = -3,       /* a CUDA runtime call failed */
  HS_EBUSY = -4,       /* serving queue full */
  HS_ETIMEDOUT = -5,   /* hs_poll: timeout expired before completion */
  HS_EDEVICE = -6,     /* a kernel set the device error word (bounded wait expired) */
  HS_ENOTSUP = -7,     /* feature not available for this plan */
  HS_ESCRATCH = -8,    /* hs_assemble_static: problem larger than its static scratch */
  HS_ENOTPD = -9       /* hs_reduce: S is not positive definite */
};

/* Arithmetic of the big stacked contractions (the per-atom Cholesky and
 * the final H/S values are FP64 in every mode). */
enum {
  HS_FP64 = 0,        /* plain FP64 everywhere */
  HS_SPLIT_BF16 = 1,  /* Ozaki-style slices on BF16 tensor cores (tcgen05), FP32
                         exact windows, recombined in extended precision to FP64 */
  HS_REAL = 0x100     /* OR-ed into the precision of hs_plan: the real-symmetric
                         variant (hs_set_t_real / hs_assemble_real) */
};

typedef struct {
  int n_fallback;      /* atoms whose Cholesky failed (Algorithm 1 failure branch) */
  int slices;          /* slice count used (0 for HS_FP64) */
  double ms_total;     /* device time of the whole call (CUDA events) */
  double ms_factor;    /* Cholesky + T preparation (0 when served from the cache) */
  double ms_atoms;     /* per-atom products Z, Y, X */
  double ms_slice;     /* slicing of the contraction operands (split mode) */
  double ms_S;         /* S contraction */
  double ms_H;         /* H contraction */
  double ms_finalize;  /* mirror to the upper triangle, real diagonal */
  double ms_queue;     /* hs_poll: submit -> admission (host clock) */
  double ms_latency;   /* hs_poll: submit -> GPU completion (host clock) */
  double inflight_bytes; /* hs_poll: footprint of all admitted requests right after
                            this one was admitted (never above the budget) */
} hs_info;

/* Create a plan for problems with N_A atoms, N_L = (l_max+1)^2 and N_G <= N_G_max.
 * precision: HS_FP64 or HS_SPLIT_BF16, OR-ed with HS_REAL for the real-symmetric
 * variant (below).  slices: 2..7 for split mode (0 = default 5),
 * ignored for FP64.  hbm_budget_bytes: cap on the plan's device workspace plus the
 * H/S outputs of requests in flight (serving admission); 0 = no cap.
 * stream: cudaStream_t to run on (NULL = the legacy default stream).
 * Allocates the device workspace for N_G_max up front; returns HS_ENOMEM if it
 * does not fit.  Sizes: N_A >= 1, 1 <= N_L <= 168, N_G_max >= 1. */
int hs_plan(hs_plan_t* out, int N_A, int N_L, int N_G_max, int precision, int slices,
            size_t hbm_budget_bytes, void* stream);

/* Exact device bytes one assembly of width N_G needs: the plan's workspace share
 * plus the caller's H and S (2 * 16 * N_G^2).  0 for a bad plan or N_G. */
size_t hs_footprint(hs_plan_t plan, int N_G);

/* Factorise T^AA (batched FP64 Cholesky, Algorithm 1 "try Cholesky") and prepare
 * the per-atom operators from device pointers T_AA, T_AB, T_BB (layout above).
 * Called implicitly by hs_assemble when the T pointers differ from the cached
 * ones; call it explicitly after changing T contents in place. */
int hs_set_t(hs_plan_t plan, const hs_z* T_AA, const hs_z* T_AB, const hs_z* T_BB);

/* Assemble H and S for one k-point (Eqs. (h), (s)).  All pointers are DEVICE
 * pointers (layout above).  Blocks until H and S are complete.  N_A and N_L
 * must equal the plan's; 1 <= N_G <= N_G_max.  info may be NULL. */
int hs_assemble(hs_plan_t plan, const hs_z* A, const hs_z* B,
                const hs_z* T_AA, const hs_z* T_AB, const hs_z* T_BB, const double* U,
                int N_A, int N_L, int N_G, hs_z* H, hs_z* S, hs_info* info);

/* Same as hs_assemble with HOST buffers: the call copies A, B, T, U to the device
 * (staging buffers owned by the plan, allocated on first use), assembles, and
 * copies H and S back.  Pinned host memory gives the fastest copies. */
int hs_assemble_host(hs_plan_t plan, const hs_z* A, const hs_z* B,
                     const hs_z* T_AA, const hs_z* T_AB, const hs_z* T_BB, const double* U,
                     int N_A, int N_L, int N_G, hs_z* H, hs_z* S, hs_info* info);

/* K-split over atoms (the paper's multi-GPU experiments, Sec. 4, split one k-point's
 * work; here each rank of a process group takes one range of atoms).  Eqs. (h) and (s)
 * are sums over atoms, so H = sum_r H_r and S = sum_r S_r over disjoint atom ranges r.
 * hs_assemble_partial computes the terms of the plan's N_A atoms only: A and B point at
 * the first row of the range inside the full stacked arrays (row a0 * N_L of a
 * K_total x N_G array, ld_AB = K_total >= N_A * N_L), T_AA, T_AB, T_BB at the range's
 * first N_L x N_L block, U at its first row (U + a0 * N_L).  It writes the LOWER
 * triangles (diagonal included) of H_r and S_r; the strict upper triangles are left
 * undefined (they may hold parts of the contraction's diagonal tiles or whatever the
 * buffers held before).  The caller adds the partials of all ranges element by element
 * (for example one collective sum over the ranks' H and S buffers), then calls
 * hs_finalize on the sums, which fills the upper triangles as the conjugates of the
 * lower ones and sets Im(diag) = 0: the result equals hs_assemble's up to the rounding
 * of the additions.  Failing Cholesky factorisations are found and counted per range
 * (hs_info.n_fallback counts this range's).  Pointers are DEVICE pointers; both calls
 * block until done; complex plans only (real plans: HS_EINVAL). */
int hs_assemble_partial(hs_plan_t plan, const hs_z* A, const hs_z* B, int ld_AB,
                        const hs_z* T_AA, const hs_z* T_AB, const hs_z* T_BB, const double* U,
                        int N_A, int N_L, int N_G, hs_z* H, hs_z* S, hs_info* info);
int hs_finalize(hs_plan_t plan, hs_z* H, hs_z* S, int N_G);

/* Serving: enqueue one k-point request (device pointers, layout above; A and B
 * may be column-truncated views of wider arrays: ld_AB >= K is their leading
 * dimension).  T and U must be the plan's current T (hs_set_t) and a U of the
 * plan's shape.  Returns at once with a ticket.  The request is admitted to the
 * device when its footprint fits the HBM budget and a slot is free; admitted
 * requests run concurrently.  HS_ENOMEM: footprint above the whole budget (can
 * never be admitted).  HS_EBUSY: queue full. */
int hs_submit(hs_plan_t plan, const hs_z* A, const hs_z* B, int ld_AB, const double* U,
              int N_G, hs_z* H, hs_z* S, int64_t* ticket);

/* Wait up to timeout_us microseconds (0 = just test, <0 = no limit) for a ticket.
 * HS_OK: done (info filled if non-NULL; the ticket is retired).  HS_PENDING /
 * HS_ETIMEDOUT: not yet.  Negative: the request failed. */
int hs_poll(hs_plan_t plan, int64_t ticket, int64_t timeout_us, hs_info* info);

/* Copy the per-atom Cholesky failure flags of the cached factorisation to
 * flags_host[N_A] (1 = fallback product used). */
int hs_fallback_flags(hs_plan_t plan, int* flags_host);

/* Free the plan and its workspace (waits for requests in flight). */
int hs_destroy(hs_plan_t plan);

/* ---------------------------------------------------------------------------
 * Real-symmetric variant.  Sec. 1.1: for systems with inversion symmetry H and S
 * are real symmetric.  Here A, B are real K x N_G (leading dimension K), T_AA,
 * T_AB, T_BB real N_A x N_L x N_L blocks (column-major; only the lower triangles of
 * T_AA and T_BB are read, T^BA = (T^AB)^T), U as above, and H, S real symmetric
 * N_G x N_G (leading dimension N_G, both triangles written).  All pointers are
 * DEVICE pointers.  The plan must be created with precision | HS_REAL; such a plan
 * accepts only these two calls (hs_assemble, hs_assemble_host and hs_set_t return
 * HS_EINVAL, hs_submit HS_ENOTSUP).  With HS_SPLIT_BF16 every operand is sliced as
 * a real array (one K position per row, no rotated copy: half the slice bytes and a
 * quarter of the tensor work of the complex form at equal sizes).  With HS_FP64 the
 * call embeds A, B as complex and runs the complex FP64 kernels (reference form).
 * The factorisation embeds T as complex and uses the complex kernels; imaginary
 * parts stay exactly zero.  Errors and blocking as hs_assemble. */
int hs_set_t_real(hs_plan_t plan, const double* T_AA, const double* T_AB, const double* T_BB);
int hs_assemble_real(hs_plan_t plan, const double* A, const double* B, const double* T_AA,
                     const double* T_AB, const double* T_BB, const double* U, int N_A, int N_L,
                     int N_G, double* H, double* S, hs_info* info);

/* ---------------------------------------------------------------------------
 * Allocation-free FP64 assembly (a library addition; the paper has no
 * counterpart).  For callers that may not allocate device memory: code that runs
 * inside someone else's fixed memory arena, or in a host process that locks its
 * device footprint after start-up, cannot create a plan, because hs_plan allocates
 * its workspace.  This call runs the plain FP64 path of hs_assemble (same kernels,
 * same results) without a plan: all intermediate buffers live in one file-scope
 * device array of HS_STATIC_SCRATCH_BYTES that every GPU loading the library holds
 * until the process exits.  Nothing is allocated and nothing is cached between calls.
 *
 * Pointers are DEVICE pointers with the layout above; stream is a cudaStream_t
 * (NULL = legacy default stream).  The call synchronises that stream once midway
 * (it reads the number of atoms whose Cholesky failed back to the host to size the
 * fallback segment) and again at the end; it returns after H and S are complete.
 * Size limit: the call needs
 *   align256(16 N_A N_L^2) + align256(32 N_A N_L^2) + 3 align256(4 N_A) + 256
 *   + 3 align256(16 N_A N_L N_G)
 * bytes of scratch; above HS_STATIC_SCRATCH_BYTES it returns HS_ESCRATCH without
 * touching the device.  1 <= N_L <= 168.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it: make that
 * first call before any stream capture begins.  All calls on a device share
 * the one array and each call overwrites it, so calls whose GPU work overlaps
 * (other streams, other host threads) race and give wrong results: serialise
 * them. */
#define HS_STATIC_SCRATCH_BYTES (32u << 20)
int hs_assemble_static(const hs_z* A, const hs_z* B, const hs_z* T_AA, const hs_z* T_AB,
                       const hs_z* T_BB, const double* U, int N_A, int N_L, int N_G,
                       hs_z* H, hs_z* S, void* stream);

/* ---------------------------------------------------------------------------
 * Reduction of the generalized eigenproblem to standard form.  Sec. 1.1: the H and
 * S of one k-point define the generalized eigenvalue problem
 *   sum_G' [H_GG' - lambda S_GG'] c_G' = 0,
 * with S (an overlap) Hermitian positive definite.  hs_reduce computes, in place,
 *   S <- L        the Cholesky factor, S = L L^H: L lower triangular with a real
 *                 positive diagonal; the strict upper triangle is set to zero;
 *   H <- C        C = L^{-1} H L^{-H}, Hermitian (both triangles written, diagonal
 *                 exactly real); C y = lambda y has the eigenvalues of the pair and
 *                 c = L^{-H} y.
 * H and S are DEVICE pointers, N_G x N_G column-major with leading dimension N_G
 * (the layout hs_assemble writes).  Only the lower triangles are read (H's
 * diagonal as its real part).  HS_FP64 plans: FP64 (DFMA) throughout, blocked
 * Cholesky, triangular inverse W = L^{-1} and the products C = G + G^H with
 * G = W tril(H) W^H.  HS_SPLIT_BF16 plans: the Cholesky and the inverse factor
 * 128-wide panels in FP64 and run their trailing updates, and the two-sided products
 * (H L^{-H}, then C = Z^H B + B^H Z with B = L^{-H} and Z = H B / 2), as BF16 slice
 * contractions on the tensor cores with the plan's slice count; relative error about
 * 1e-10 kappa(S) instead of FP64's.  Complex plans
 * only (real plans: HS_EINVAL).  0 <= N_G <= N_G_max.  The plan allocates 32 N_G^2
 * bytes of device workspace on first use (split plans also about (24 s + 64) N_G^2
 * bytes of slices and products), grown on demand and
 * freed by hs_destroy; HS_ENOMEM if that fails.  Runs on the plan's stream and
 * returns when done.
 * HS_ENOTPD: a Cholesky pivot of S is zero, negative or NaN; info->fail_col is that
 * column (1-based), H is unchanged and S holds a partial factor.
 * info may be NULL. */
typedef struct {
  int fail_col;          /* 0, or the failing column of the Cholesky (1-based) */
  double ms_total;       /* device time of the call (CUDA events) */
  double ms_cholesky;    /* S = L L^H */
  double ms_inverse;     /* W = L^{-1} (split plans: the part not overlapped with the
                            Cholesky, which it follows panel by panel on another stream) */
  double ms_p;           /* P = W tril_h(H) (tril_h: lower triangle, diagonal halved) */
  double ms_g;           /* G = P W^H and C = G + G^H */
} hs_reduce_info;
int hs_reduce(hs_plan_t plan, hs_z* H, hs_z* S, int N_G, hs_reduce_info* info);
/* The same for the real-symmetric variant: real symmetric H and S (DEVICE pointers,
 * N_G x N_G column-major, leading dimension N_G) on a plan made with HS_REAL;
 * S <- L (real), H <- C (real symmetric).  The pair is embedded as complex and reduced
 * by the plan's form (FP64 plans: the FP64 kernels; split plans: the split form's,
 * with its error bound), imaginary parts staying exactly zero; split real plans
 * allocate the two complex N_G_max x N_G_max buffers of the embedding on first use.
 * Complex plans: HS_EINVAL.  HS_ENOTPD leaves H and S unchanged. */
int hs_reduce_real(hs_plan_t plan, double* H, double* S, int N_G, hs_reduce_info* info);

/* ---------------------------------------------------------------------------
 * Matching coefficients A, B (the inputs of hs_assemble), Sec. 1.1.  The basis
 * function of plane wave g, wave vector K_g = k + G_g, is e^{i K.r} / sqrt(Omega)
 * between the spheres and, in the sphere of atom a (centre tau_a, radius R_a),
 *   sum_{l,m} [A_{aL,g} u^a_l(r) + B_{aL,g} udot^a_l(r)] Y_lm(r^),   L = l^2 + l + m;
 * A and B make the function and its radial derivative continuous at r = R_a.  With
 * the Rayleigh expansion of the plane wave,
 *   c = (4 pi / sqrt(Omega)) e^{i K.tau_a} i^l conj(Y_lm(K^)),   x = |K| R_a,
 *   A = c (j_l(x) udot'_l - |K| j_l'(x) udot_l) / W,
 *   B = c (|K| j_l'(x) u_l - j_l(x) u'_l) / W,      W = u_l udot'_l - u'_l udot_l,
 * Y_lm orthonormal with the Condon-Shortley phase, j_l spherical Bessel functions;
 * a zero K takes the direction theta = phi = 0.
 * Inputs (DEVICE pointers, doubles, row-major):
 *   Kvec : N_G x 3 Cartesian wave vectors k + G;   tau : N_A x 3 atom positions;
 *   R    : N_A sphere radii;
 *   ufun : N_A x (l_max + 1) x 4 radial boundary values at R_a, in the order
 *          u_l(R), u_l'(R), udot_l(R), udot_l'(R);   omega : cell volume (> 0).
 * Outputs: A, B (distinct, not overlapping the inputs) in the layout of hs_assemble,
 *   (N_A N_L) x N_G column-major with leading dimension ld_AB >= N_A N_L; only rows
 *   [0, N_A N_L) of each column are written.
 * 0 <= l_max <= 11 (N_L <= 144); N_G = 0 returns HS_OK at once.  A zero W gives
 * non-finite coefficients (not checked).  stream is a cudaStream_t (NULL = legacy
 * default stream); the call returns after A and B are complete.  It takes
 * 48 N_A (l_max + 1) bytes of stream-ordered device scratch (cudaMallocAsync on that
 * stream, freed before it returns) for the factors that do not depend on the plane
 * wave; HS_ENOMEM if that allocation fails. */
int hs_matching(const double* Kvec, const double* tau, const double* R, const double* ufun,
                double omega, int N_A, int l_max, int N_G, hs_z* A, hs_z* B, int ld_AB,
                void* stream);

/* Static description of an error code. */
const char* hs_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* HS_H_ */
