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
// One CTA per plane wave g: the angular factors c_lm / e^{i K.tau_a} of the column in
// shared memory (normalised associated Legendre functions by the standard l recurrence,
// Condon-Shortley phase), then per chunk of atoms the phases and the radial factors
// (j_l for all l by Miller's downward recurrence, normalised to j_0 or j_1), then the
// column's K = N_A N_L rows of A and B, which are contiguous in the column-major
// layout, written by consecutive threads.
#include <cuda_runtime.h>

#include <cmath>

#include "hs_internal.h"

namespace {

constexpr int kMaxL = 11;               // l_max: (l_max + 1)^2 <= 168 rows per atom
constexpr int kMaxNL = (kMaxL + 1) * (kMaxL + 1);
constexpr int kAtomChunk = 64;          // atoms whose radial factors sit in smem at once
constexpr int kThreads = 256;

// j_l(x) for l = 0 .. lmax (x >= 0) and j_l'(x).  Miller's method: the recurrence
// f_{n-1} = (2n + 1) / x f_n - f_{n+1}, run downwards from n0 = m + 8 + sqrt(40 m),
// m = max(lmax, x) (where j_n decays fast in n), is stable; the sequence is rescaled
// when it nears overflow and normalised by whichever of j_0 = sin x / x and
// j_1 = sin x / x^2 - cos x / x is larger in magnitude.  j_l' = (l / x) j_l - j_{l+1}.
__device__ void sph_bessel(double x, int lmax, double* j, double* dj) {
  if (x == 0.0) {
    for (int l = 0; l <= lmax; ++l) {
      j[l] = l == 0 ? 1.0 : 0.0;
      dj[l] = l == 1 ? 1.0 / 3.0 : 0.0;
    }
    return;
  }
  double f[kMaxL + 2];
  for (int l = 0; l < kMaxL + 2; ++l) f[l] = 0.0;
  const double m = fmax((double)lmax, x);
  const int n0 = (int)(m + 8.0 + sqrt(40.0 * m));
  const double rx = 1.0 / x;
  double fp1 = 0.0, fn = 1e-200;  // f_{n+1}, f_n
  for (int n = n0; n >= 1; --n) {
    const double fm1 = (2.0 * n + 1.0) * rx * fn - fp1;
    fp1 = fn;
    fn = fm1;
    if (fabs(fn) > 1e200) {  // rescale the sequence, the part kept so far included
      fp1 *= 1e-200;
      fn *= 1e-200;
      for (int l = 0; l < kMaxL + 2; ++l) f[l] *= 1e-200;
    }
    if (n - 1 <= lmax + 1) f[n - 1] = fn;
  }
  double s, c;
  sincos(x, &s, &c);
  const double j0 = s * rx, j1 = (s * rx - c) * rx;
  const double scale = fabs(j0) >= fabs(j1) ? j0 / f[0] : j1 / f[1];
  for (int l = 0; l <= lmax + 1; ++l) f[l] *= scale;
  for (int l = 0; l <= lmax; ++l) {
    j[l] = f[l];
    dj[l] = l * rx * f[l] - f[l + 1];
  }
}

__global__ void __launch_bounds__(kThreads) k_matching(const double* __restrict__ Kvec,
                                                       const double* __restrict__ tau,
                                                       const double* __restrict__ R,
                                                       const double* __restrict__ ufun,
                                                       double pref, int N_A, int lmax, int N_G, size_t ld,
                                                       double2* __restrict__ A,
                                                       double2* __restrict__ B) {
  __shared__ double2 c_L[kMaxNL];               // (4 pi / sqrt(Omega)) i^l conj(Y_lm(K^))
  __shared__ unsigned char l_of[kMaxNL];
  __shared__ double2 ph[kAtomChunk];            // e^{i K.tau_a}
  __shared__ double fa[kAtomChunk][kMaxL + 1];  // radial factor of A
  __shared__ double fb[kAtomChunk][kMaxL + 1];  // radial factor of B
  const int g = blockIdx.x;
  if (g >= N_G) return;
  const int N_L = (lmax + 1) * (lmax + 1);
  const double kx = Kvec[3 * g], ky = Kvec[3 * g + 1], kz = Kvec[3 * g + 2];
  const double rho = sqrt(kx * kx + ky * ky);
  const double Kn = sqrt(rho * rho + kz * kz);
  // direction of K; a zero vector (or one on the z axis) takes theta = 0 (phi = 0)
  const double ct = Kn > 0.0 ? kz / Kn : 1.0, st = Kn > 0.0 ? rho / Kn : 0.0;
  const double cp = rho > 0.0 ? kx / rho : 1.0, sp = rho > 0.0 ? ky / rho : 0.0;

  // ---- angular factors: thread m runs the l recurrence of order m
  if (threadIdx.x <= lmax) {
    const int m = threadIdx.x;
    // P_mm = (-1)^m (2m - 1)!! sin^m theta (Condon-Shortley phase included)
    double pmm = 1.0;
    for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * st;
    // e^{i m phi}
    double er = 1.0, ei = 0.0;
    for (int i = 0; i < m; ++i) {
      const double t = er * cp - ei * sp;
      ei = er * sp + ei * cp;
      er = t;
    }
    double p_lm2 = 0.0, p_lm1 = pmm;
    for (int l = m; l <= lmax; ++l) {
      double p;
      if (l == m) p = pmm;
      else if (l == m + 1) p = ct * (2.0 * m + 1.0) * pmm;
      else p = ((2.0 * l - 1.0) * ct * p_lm1 - (l + m - 1.0) * p_lm2) / (double)(l - m);
      if (l > m) {
        p_lm2 = p_lm1;
        p_lm1 = p;
      }
      // N_lm = sqrt((2l + 1) / (4 pi) (l - m)! / (l + m)!)
      double ratio = 1.0;
      for (int i = l - m + 1; i <= l + m; ++i) ratio /= (double)i;
      const double nrm = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * ratio);
      const double yr = nrm * p * er, yi = nrm * p * ei;  // Y_lm, m >= 0
      // i^l conj(Y): conj(Y) = (yr, -yi); i^l rotates by l quarter turns
      auto put = [&](int mm, double re, double im) {
        double cr = re, ci = -im;  // conj
        for (int q = 0; q < (l & 3); ++q) {
          const double t = -ci;
          ci = cr;
          cr = t;
        }
        const int L = l * l + l + mm;
        c_L[L] = make_double2(pref * cr, pref * ci);
        l_of[L] = (unsigned char)l;
      };
      put(m, yr, yi);
      if (m > 0) {  // Y_{l,-m} = (-1)^m conj(Y_lm)
        const double sgn = (m & 1) ? -1.0 : 1.0;
        put(-m, sgn * yr, -sgn * yi);
      }
    }
  }
  __syncthreads();

  // ---- per chunk of atoms: phases and radial factors, then the chunk's rows
  for (int a0 = 0; a0 < N_A; a0 += kAtomChunk) {
    const int na = min(kAtomChunk, N_A - a0);
    for (int i = threadIdx.x; i < na; i += blockDim.x) {
      const int a = a0 + i;
      double s, c;
      sincos(kx * tau[3 * a] + ky * tau[3 * a + 1] + kz * tau[3 * a + 2], &s, &c);
      ph[i] = make_double2(c, s);
      double j[kMaxL + 1], dj[kMaxL + 1];
      sph_bessel(Kn * R[a], lmax, j, dj);
      for (int l = 0; l <= lmax; ++l) {
        const double* uf = ufun + ((size_t)a * (lmax + 1) + l) * 4;
        const double u = uf[0], du = uf[1], ud = uf[2], dud = uf[3];
        const double rW = 1.0 / (u * dud - du * ud);  // 1 / Wronskian
        fa[i][l] = (j[l] * dud - Kn * dj[l] * ud) * rW;
        fb[i][l] = (Kn * dj[l] * u - j[l] * du) * rW;
      }
    }
    __syncthreads();
    double2* Ac = A + (size_t)g * ld + (size_t)a0 * N_L;
    double2* Bc = B + (size_t)g * ld + (size_t)a0 * N_L;
    for (int r = threadIdx.x; r < na * N_L; r += blockDim.x) {
      const int i = r / N_L, L = r - i * N_L;
      const double2 p = ph[i], cl = c_L[L];
      const double tr = p.x * cl.x - p.y * cl.y, ti = p.x * cl.y + p.y * cl.x;
      const int l = l_of[L];
      Ac[r] = make_double2(tr * fa[i][l], ti * fa[i][l]);
      Bc[r] = make_double2(tr * fb[i][l], ti * fb[i][l]);
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
  k_matching<<<N_G, kThreads, 0, st>>>(Kvec, tau, R, ufun, pref, N_A, l_max, N_G,
                                       (size_t)ld_AB, (double2*)A, (double2*)B);
  HS_CUDA_TRY(cudaGetLastError());
  HS_CUDA_TRY(cudaStreamSynchronize(st));
  return HS_OK;
}
