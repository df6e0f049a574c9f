// Matching coefficients A, B of the basis (Sec. 1.1): inside the muffin-tin sphere of
// atom a the basis function of plane wave G (wave vector K = k + G) is
//   sum_{l,m} [A^{a,G}_{lm} u^a_l(r) + B^{a,G}_{lm} udot^a_l(r)] Y_lm(r^_a),
// and A, B make it and its radial derivative continuous with e^{i K.r} / sqrt(Omega)
// on the sphere r = R_a.  By the Rayleigh expansion of the plane wave around tau_a,
//   c_lm = (4 pi / sqrt(Omega)) e^{i K.tau_a} i^l conj(Y_lm(K^)),
//   A = c_lm (j_l(KR) udot'(R) - K j_l'(KR) udot(R)) / W,
//   B = c_lm (K j_l'(KR) u(R) - j_l(KR) u'(R)) / W,   W = u udot' - u' udot,
// with j_l the spherical Bessel functions (K = |K|).
//
// GB300 runs FP64 at 2 operations per clock per SM, so this kernel is bound by its
// FP64 arithmetic, not by the stores of A and B; it is arranged to spend as few FP64
// operations per output element as the formula allows.  With conj(Y_lm) written as
// Pbar_l|m|(cos theta) e^{-i m phi} (times (-1)^m for m < 0), each element is the
// product of three factors:
//   A_{aL} = [scale_a e^{i K.tau_a} e^{-i m phi}] * i^l [pref sigma Pbar]_L * f^A_{al},
// a complex one per (atom, m), a real one per row L and a real radial one per
// (atom, l), shared with B (f^B in place of f^A).  The factor i^l is a sign, kept in
// the row table P2, and a swap of the real and imaginary parts of E, so an element
// costs 2 FP64 products for X = i^l E P_L and 2 each for A and B, with no additions
// and no negations.
//
// A pre-pass kernel computes the factors that do not depend on the plane wave (the
// radial boundary values over the Wronskian W, l / R_a).  Then one CTA per plane
// wave g, all atoms: the per-row factors P2_L and e^{-i m phi} in shared memory
// (normalised associated Legendre functions by their l recurrence with compile-time
// coefficients, Condon-Shortley phase); per chunk of atoms, one thread per atom
// computes E_{a,m} and the radial factors (j_l for all l by Miller's downward
// recurrence, or upwards when |K| R_a exceeds l_max + 8), then consecutive threads
// write the chunk's rows of the column, which are contiguous in the column-major
// layout.
#include <cuda_runtime.h>

#include <cmath>

#include "hs_internal.h"

namespace {

constexpr int kMaxL = 11;               // l_max: (l_max + 1)^2 <= 144 rows per atom
constexpr int kMaxNL = (kMaxL + 1) * (kMaxL + 1);
constexpr int kMaxM = 2 * kMaxL + 1;    // m = -l_max .. l_max
constexpr int kAtomChunk = 64;          // atoms whose factors sit in smem at once
constexpr int kThreads = 256;

// ---- constant tables of the normalised associated Legendre functions
// Pbar_lm = N_lm P_lm (Condon-Shortley phase), N_lm = sqrt((2l + 1) / (4 pi) (l - m)! / (l + m)!),
// obey (standard recurrences, from the ones of P_lm with the ratios of the N_lm):
//   Pbar_00 = 1 / sqrt(4 pi),   Pbar_mm = c_m sin(theta) Pbar_{m-1,m-1},  c_m = -sqrt((2m + 1) / (2m)),
//   Pbar_lm = a_lm (cos(theta) Pbar_{l-1,m} - b_lm Pbar_{l-2,m})  (l > m, Pbar_{m-1,m} = 0),
//   a_lm = sqrt((4 l^2 - 1) / (l^2 - m^2)),  b_lm = sqrt(((l - 1)^2 - m^2) / (4 (l - 1)^2 - 1)).
// The coefficients are evaluated at compile time (Newton's iteration for the square
// root, run until it stops decreasing: within an ulp), so the kernel spends no FP64
// divisions or square roots on them.
constexpr double ce_sqrt(double x) {
  if (x <= 0.0) return 0.0;
  double r = x > 1.0 ? x : 1.0;  // start above sqrt(x): Newton then decreases monotonically
  for (int i = 0; i < 2000; ++i) {
    const double n = 0.5 * (r + x / r);
    if (!(n < r)) break;
    r = n;
  }
  return r;
}

struct LegendreTab {
  double a[kMaxNL], b[kMaxNL];  // at index l^2 + l + m, 0 <= m < l
  double c[kMaxL + 1];          // c_m, m >= 1
  double p00;
};

constexpr LegendreTab make_legendre_tab() {
  LegendreTab t{};
  for (int l = 0; l <= kMaxL; ++l) {
    for (int m = 0; m < l; ++m) {
      const double l2 = (double)l * l, m2 = (double)m * m, lm1 = l - 1.0;
      t.a[l * l + l + m] = ce_sqrt((4.0 * l2 - 1.0) / (l2 - m2));
      t.b[l * l + l + m] = ce_sqrt((lm1 * lm1 - m2) / (4.0 * lm1 * lm1 - 1.0));
    }
  }
  for (int m = 1; m <= kMaxL; ++m) t.c[m] = -ce_sqrt((2.0 * m + 1.0) / (2.0 * m));
  t.p00 = 1.0 / ce_sqrt(4.0 * 3.14159265358979323846);
  return t;
}

__constant__ LegendreTab kLeg = make_legendre_tab();

// Unnormalised j_l(x), l = 0 .. lmax + 1, and the factor that normalises them,
// j_l = scale f_l; rx = 1 / x.  The recurrence f_{n-1} + f_{n+1} = (2n + 1) / x f_n
// of the spherical Bessel functions is run
// * upwards from j_0 = sin x / x and j_1 = sin x / x^2 - cos x / x when x > lmax + 8:
//   every order needed is below x, where the upward direction is stable (scale = 1);
// * otherwise downwards (Miller's method) from n0 = max(lmax + x + 6, x + 4.5 sqrt(x) + 6),
//   where j_n decays fast in n, rescaled when it nears overflow, and normalised by
//   whichever of j_0, j_1 is larger in magnitude.
// Below x = 1e-30, f = (1, 0, ...) and scale = 1: j_l(x) = x^l / (2l + 1)!! (1 + O(x^2))
// is below 1e-30 of j_0 there for l > 0.
__device__ double miller(double x, double rx, int lmax, double* f) {
  for (int l = 0; l < kMaxL + 2; ++l) f[l] = 0.0;
  if (x < 1e-30) {
    f[0] = 1.0;
    return 1.0;
  }
  if (x > lmax + 8.0) {
    double s, c;
    sincos(x, &s, &c);
    f[0] = s * rx;
    f[1] = (s * rx - c) * rx;
    for (int l = 1; l <= lmax; ++l) f[l + 1] = (2.0 * l + 1.0) * rx * f[l] - f[l - 1];
    return 1.0;
  }
  const int n0 = (int)fmax(lmax + x + 6.0, x + 4.5 * sqrt(x) + 6.0);
  // 2n + 1 as an exact double counter; (2n + 1) * rx formed afresh each step (a
  // coefficient stepped down by 2 / x drifts, and the drift costs ~1e-13 at x ~ 11)
  double tn = 2.0 * n0 + 1.0;
  double fp1 = 0.0, fn = 1e-200;  // f_{n+1}, f_n
  for (int n = n0; n >= 1; --n) {
    const double fm1 = tn * rx * fn - fp1;
    tn -= 2.0;
    fp1 = fn;
    fn = fm1;
    // rescale when |f| passes 2^664 (exponent field of the high word: no FP64 compare)
    if (((__double2hiint(fn) >> 20) & 0x7ff) > 1023 + 664) {
      fp1 *= 0x1p-1328;
      fn *= 0x1p-1328;
      for (int l = 0; l < kMaxL + 2; ++l) f[l] *= 0x1p-1328;
    }
    if (n - 1 <= lmax + 1) f[n - 1] = fn;
  }
  double s, c;
  sincos(x, &s, &c);
  const double j0 = s * rx, j1 = (s * rx - c) * rx;
  return fabs(j0) >= fabs(j1) ? j0 / f[0] : j1 / f[1];
}

// Per (atom, l) factors that do not depend on the plane wave, one thread each:
//   rad = (udot'/W, udot/W, u/W, u'/W, l / R_a, 1 / R_a),   W = u udot' - u' udot.
constexpr int kRad = 6;
__global__ void k_matching_radial(const double* __restrict__ R, const double* __restrict__ ufun,
                                  int N_A, int lmax, double* __restrict__ rad) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N_A * (lmax + 1)) return;
  const int a = idx / (lmax + 1), l = idx - a * (lmax + 1);
  const double u = ufun[4 * idx], du = ufun[4 * idx + 1], ud = ufun[4 * idx + 2],
               dud = ufun[4 * idx + 3];
  const double rW = 1.0 / (u * dud - du * ud);
  const double rR = 1.0 / R[a];
  double* o = rad + (size_t)idx * kRad;
  o[0] = dud * rW;
  o[1] = ud * rW;
  o[2] = u * rW;
  o[3] = du * rW;
  o[4] = l * rR;
  o[5] = rR;
}

__global__ void __launch_bounds__(kThreads) k_matching(const double* __restrict__ Kvec,
                                                       const double* __restrict__ tau,
                                                       const double* __restrict__ R,
                                                       const double* __restrict__ rad,
                                                       double pref, int N_A, int lmax, int N_G,
                                                       size_t ld, double2* __restrict__ A,
                                                       double2* __restrict__ B) {
  __shared__ double2 P2[kMaxNL];                // (v, v) for even l, (-v, v) for odd l,
                                                // v = (-1)^{floor(l/2)} pref sigma_m Pbar
  __shared__ unsigned char l_of[kMaxNL], mi_of[kMaxNL];
  __shared__ double2 w_m[kMaxM];                // e^{-i m phi} at index lmax + m
  __shared__ double2 E[kAtomChunk][kMaxM];      // scale_a e^{i K.tau_a} e^{-i m phi}
  __shared__ double fa[kAtomChunk][kMaxL + 1];  // radial factor of A over scale_a
  __shared__ double fb[kAtomChunk][kMaxL + 1];  // radial factor of B over scale_a
  const int g = blockIdx.x;
  if (g >= N_G) return;
  const int N_L = (lmax + 1) * (lmax + 1);
  const int NM = 2 * lmax + 1;
  const double kx = Kvec[3 * g], ky = Kvec[3 * g + 1], kz = Kvec[3 * g + 2];
  // |K|, 1/|K| and the direction of K, computed once per column by one thread (the
  // square roots and divisions cost tens of FP64 operations, which every thread of the
  // CTA repeating them would multiply by 256); a zero vector (or one on the z axis)
  // takes theta = 0 (phi = 0)
  __shared__ double col[6];  // |K|, 1/|K|, cos theta, sin theta, cos phi, sin phi
  if (threadIdx.x == 0) {
    const double rho = sqrt(kx * kx + ky * ky);
    const double kn = sqrt(rho * rho + kz * kz);
    col[0] = kn;
    col[1] = kn > 0.0 ? 1.0 / kn : 0.0;
    col[2] = kn > 0.0 ? kz / kn : 1.0;
    col[3] = kn > 0.0 ? rho / kn : 0.0;
    col[4] = rho > 0.0 ? kx / rho : 1.0;
    col[5] = rho > 0.0 ? ky / rho : 0.0;
  }
  __syncthreads();
  const double Kn = col[0], rK = col[1];
  const double ct = col[2], st = col[3], cp = col[4], sp = col[5];

  // ---- per-row factors: thread m runs the l recurrence of order m
  if (threadIdx.x <= lmax) {
    const int m = threadIdx.x;
    // Pbar_mm from Pbar_00 by the c_m steps
    double pmm = kLeg.p00;
    for (int i = 1; i <= m; ++i) pmm *= kLeg.c[i] * st;
    // e^{i m phi} by repeated rotation; e^{-i m phi} is its conjugate
    double er = 1.0, ei = 0.0;
    for (int i = 0; i < m; ++i) {
      const double t = er * cp - ei * sp;
      ei = er * sp + ei * cp;
      er = t;
    }
    w_m[lmax + m] = make_double2(er, -ei);
    w_m[lmax - m] = make_double2(er, ei);
    double p_lm2 = 0.0, p_lm1 = pmm;
    for (int l = m; l <= lmax; ++l) {
      double p = pmm;
      if (l > m) {
        const int L = l * l + l + m;
        p = kLeg.a[L] * (ct * p_lm1 - kLeg.b[L] * p_lm2);
        p_lm2 = p_lm1;
        p_lm1 = p;
      }
      // i^l = (-1)^{floor(l/2)} i^{l mod 2}: the sign here, the factor i in the output
      const double v = ((l & 2) ? -pref : pref) * p;
      // conj(Y_lm) = Pbar_lm e^{-i m phi};  conj(Y_{l,-m}) = (-1)^m Y_lm = (-1)^m Pbar_lm e^{i m phi}
      const int Lp = l * l + l + m, Lm = l * l + l - m;
      P2[Lp] = make_double2((l & 1) ? -v : v, v);
      l_of[Lp] = (unsigned char)l;
      mi_of[Lp] = (unsigned char)(lmax + m);
      if (m > 0) {
        const double vm = (m & 1) ? -v : v;
        P2[Lm] = make_double2((l & 1) ? -vm : vm, vm);
        l_of[Lm] = (unsigned char)l;
        mi_of[Lm] = (unsigned char)(lmax - m);
      }
    }
  }
  __syncthreads();

  // ---- per chunk of atoms: E and the radial factors, then the chunk's rows
  const int step_i = kThreads / N_L, step_L = kThreads % N_L;
  for (int a0 = 0; a0 < N_A; a0 += kAtomChunk) {
    const int na = min(kAtomChunk, N_A - a0);
    for (int i = threadIdx.x; i < na; i += kThreads) {
      const int a = a0 + i;
      const double* rd = rad + (size_t)a * (lmax + 1) * kRad;
      // radial part: j_l = scale f_l and, with K / x = 1 / R_a,
      //   K j_l' = scale (l / R_a f_l - K f_{l+1}) = scale d_l;
      //   f^A = scale (f_l udot' - d_l udot) / W,  f^B = scale (d_l u - f_l u') / W,
      // the common factor scale moved into E
      double f[kMaxL + 2];
      const double scale = miller(Kn * R[a], rK * rd[5], lmax, f);
      for (int l = 0; l <= lmax; ++l) {
        const double* q = rd + l * kRad;
        const double d = q[4] * f[l] - Kn * f[l + 1];
        fa[i][l] = f[l] * q[0] - d * q[1];
        fb[i][l] = d * q[2] - f[l] * q[3];
      }
      double s, c;
      sincos(kx * tau[3 * a] + ky * tau[3 * a + 1] + kz * tau[3 * a + 2], &s, &c);
      s *= scale;
      c *= scale;
      for (int k = 0; k < NM; ++k) {
        const double2 w = w_m[k];
        E[i][k] = make_double2(c * w.x - s * w.y, c * w.y + s * w.x);
      }
    }
    __syncthreads();
    double2* Ac = A + (size_t)g * ld + (size_t)a0 * N_L;
    double2* Bc = B + (size_t)g * ld + (size_t)a0 * N_L;
    const int nr = na * N_L;
    int i = threadIdx.x / N_L, L = threadIdx.x % N_L;  // row r = i N_L + L
    for (int r = threadIdx.x; r < nr; r += kThreads) {
      const double2 e = E[i][mi_of[L]];
      const double2 p = P2[L];
      const int l = l_of[L];
      // times i for odd l: (e.x, e.y) p -> (-e.y p, e.x p), the sign taken from P2
      const bool odd = l & 1;
      const double xr = (odd ? e.y : e.x) * p.x, xi = (odd ? e.x : e.y) * p.y;
      const double fA = fa[i][l], fB = fb[i][l];
      Ac[r] = make_double2(xr * fA, xi * fA);
      Bc[r] = make_double2(xr * fB, xi * fB);
      i += step_i;
      L += step_L;
      if (L >= N_L) {
        L -= N_L;
        ++i;
      }
    }
    __syncthreads();
  }
}

}  // namespace

extern "C" int hs_matching(const double* Kvec, const double* tau, const double* R,
                           const double* ufun, double omega, int N_A, int l_max, int N_G,
                           hs_z* A, hs_z* B, int ld_AB, void* stream) {
  if (!Kvec || !tau || !R || !ufun || !A || !B || A == B) return HS_EINVAL;
  if (N_A < 1 || l_max < 0 || l_max > kMaxL || N_G < 0 || !(omega > 0.0)) return HS_EINVAL;
  const long long K = (long long)N_A * (l_max + 1) * (l_max + 1);
  if (K > (1LL << 30) || ld_AB < K) return HS_EINVAL;
  if (N_G == 0) return HS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const double pref = 4.0 * M_PI / sqrt(omega);
  const int nrad = N_A * (l_max + 1);
  double* rad = nullptr;
  if (cudaMallocAsync((void**)&rad, sizeof(double) * kRad * nrad, st) != cudaSuccess) {
    cudaGetLastError();
    return HS_ENOMEM;
  }
  k_matching_radial<<<(nrad + 255) / 256, 256, 0, st>>>(R, ufun, N_A, l_max, rad);
  k_matching<<<N_G, kThreads, 0, st>>>(Kvec, tau, R, rad, pref, N_A, l_max, N_G,
                                       (size_t)ld_AB, (double2*)A, (double2*)B);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(rad, st);
  HS_CUDA_TRY(e);
  HS_CUDA_TRY(cudaStreamSynchronize(st));
  return HS_OK;
}
