"""Matching coefficients A, B of the (L)APW basis, plain FP64 on the CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/hs_oracle.py``): used by tests and the
benchmark's CPU-baseline leg, never by the library.

Sec. 1.1 writes the basis function of plane wave G (wave vector K = k + G) as
e^{i K.r} in the interstitial region and, inside the muffin-tin sphere of atom a,

    sum_{l,m} [ A^{a,G}_{lm} u^a_l(r_a) + B^{a,G}_{lm} udot^a_l(r_a) ] Y_lm(r^_a),

r_a = r - tau_a, and states that A and B follow from the continuity of the function
and of its (radial) derivative on the sphere boundary r_a = R_a.  Written out:

* the plane wave around tau_a, with the normalisation 1 / sqrt(Omega) of the cell
  volume Omega, by the Rayleigh expansion (a textbook identity)

      e^{i K.r} / sqrt(Omega) = (4 pi / sqrt(Omega)) e^{i K.tau_a}
            sum_{l,m} i^l j_l(|K| r_a) conj(Y_lm(K^)) Y_lm(r^_a);

* per (a, l, m, G), with c = (4 pi / sqrt(Omega)) e^{i K.tau_a} i^l conj(Y_lm(K^)),
  the 2 x 2 system at r_a = R_a

      A u(R) + B udot(R)   = c j_l(|K| R)
      A u'(R) + B udot'(R) = c |K| j_l'(|K| R)

  solved with the Wronskian W = u udot' - u' udot:

      A = c (j udot' - |K| j' udot) / W,   B = c (|K| j' u - j u') / W.

Y_lm are the orthonormal complex spherical harmonics with the Condon-Shortley phase,
written out from their definition (Ferrers functions from the derivatives of the
Legendre polynomial, differentiated and evaluated in the Legendre basis; no
spherical-harmonic library routine); the spherical Bessel functions j_l and j_l'
are scipy's.  The row of (l, m) in a block of N_L = (l_max + 1)^2 rows is
L = l^2 + l + m, the order the assembly uses (angular momentum l = floor(sqrt(L))).
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg
from scipy.special import spherical_jn


def lm_of_L(N_L: int):
    """(l, m) of the compound index L = l^2 + l + m, L = 0 .. N_L - 1."""
    out = []
    for L in range(N_L):
        l = int(math.isqrt(L))
        out.append((l, L - l * l - l))
    return out


def ylm(l_max: int, theta, phi) -> np.ndarray:
    """Y_lm(theta, phi) for L = 0 .. (l_max+1)^2 - 1, shape (N_L,) + theta.shape.

    Y_lm = (-1)^m sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m(cos theta) e^{i m phi}
    for m >= 0, with the Ferrers function P_l^m(x) = (1-x^2)^{m/2} d^m P_l / dx^m,
    and Y_{l,-m} = (-1)^m conj(Y_lm)."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    x = np.cos(theta)
    sin_t = np.sin(theta)
    N_L = (l_max + 1) ** 2
    Y = np.zeros((N_L,) + x.shape, dtype=np.complex128)
    for l in range(l_max + 1):
        P = np.zeros(l + 1)
        P[l] = 1.0  # P_l in the Legendre basis
        for m in range(0, l + 1):
            # d^m P_l / dx^m kept in the Legendre basis and summed there (Clenshaw): the
            # power-series form of the same polynomial cancels to ~1e-12 at l = 11
            dm = npleg.legder(P, m) if m > 0 else P
            Plm = sin_t ** m * npleg.legval(x, dm)
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m)
                             / math.factorial(l + m))
            Ypos = (-1) ** m * norm * Plm * np.exp(1j * m * phi)
            Y[l * l + l + m] = Ypos
            if m > 0:
                Y[l * l + l - m] = (-1) ** m * np.conj(Ypos)
    return Y


def _angles(V):
    """(|V|, theta, phi) of vectors V (n, 3); direction of a zero vector: theta = phi = 0."""
    V = np.asarray(V, dtype=np.float64)
    r = np.linalg.norm(V, axis=1)
    safe = np.where(r > 0, r, 1.0)
    theta = np.arccos(np.clip(V[:, 2] / safe, -1.0, 1.0))
    phi = np.arctan2(V[:, 1], V[:, 0])
    theta = np.where(r > 0, theta, 0.0)
    phi = np.where(r > 0, phi, 0.0)
    return r, theta, phi


def matching(Kvec, tau, R, ufun, omega: float, l_max: int):
    """A, B as (N_A N_L, N_G) complex arrays (column g = plane wave g, rows a N_L + L).

    Kvec: (N_G, 3) wave vectors k + G; tau: (N_A, 3) atom positions; R: (N_A,) sphere
    radii; ufun: (N_A, l_max + 1, 4) radial boundary values u(R), u'(R), udot(R),
    udot'(R); omega: cell volume."""
    Kvec = np.asarray(Kvec, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    ufun = np.asarray(ufun, dtype=np.float64)
    N_G, N_A = Kvec.shape[0], tau.shape[0]
    N_L = (l_max + 1) ** 2
    Kn, theta, phi = _angles(Kvec)
    Yc = np.conj(ylm(l_max, theta, phi))          # (N_L, N_G)
    lm = lm_of_L(N_L)
    il = np.array([1j ** l for l, _ in lm])       # i^l per row
    A = np.zeros((N_A * N_L, N_G), dtype=np.complex128)
    B = np.zeros_like(A)
    for a in range(N_A):
        phase = np.exp(1j * (Kvec @ tau[a]))      # e^{i K.tau_a}, (N_G,)
        x = Kn * R[a]
        for L, (l, m) in enumerate(lm):
            u, du, ud, dud = ufun[a, l]
            W = u * dud - du * ud
            j = spherical_jn(l, x)
            dj = spherical_jn(l, x, derivative=True)
            c = (4.0 * math.pi / math.sqrt(omega)) * phase * il[L] * Yc[L]
            A[a * N_L + L] = c * (j * dud - Kn * dj * ud) / W
            B[a * N_L + L] = c * (Kn * dj * u - j * du) / W
    return A, B
