"""Exact brute force of the index forms of S and H, for tiny sizes.

TEST INFRASTRUCTURE ONLY (see ``oracle/hs_oracle.py``).

Sec. 1.1 gives H and S element by element:

    S_{G',G} = sum_a sum_{L} conj(A^{a,G'}_L) A^{a,G}_L
                           + conj(B^{a,G'}_L) B^{a,G}_L ||udot^a_l||^2
    H_{G',G} = sum_a sum_{L',L} sum_{X,Y in {A,B}}
                     conj(X^{a,G'}_{L'}) T^{[XY]}_{L',L;a} Y^{a,G}_L

with T^{[BA]}_{L',L;a} = conj(T^{[AB]}_{L,L';a}) (Sec. 2: T^BA is the
Hermitian transpose of T^AB) and ||udot^a_l||^2 read as U[a, L]^2.

Every double input is an exact binary rational, so the sums are evaluated in
``fractions.Fraction`` arithmetic without any rounding; the result is the
exact value of the definition for the given floating-point inputs.  Pure
Python loops: only for N_A <= 3, N_L <= 4, N_G <= 8.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _q(z):
    z = complex(z)
    return (Fraction(z.real), Fraction(z.imag))


def _mul(x, y):
    return (x[0] * y[0] - x[1] * y[1], x[0] * y[1] + x[1] * y[0])


def _conj(x):
    return (x[0], -x[1])


def _add(x, y):
    return (x[0] + y[0], x[1] + y[1])


def exact_hs(A, B, T_AA, T_AB, T_BB, U, N_A: int, N_L: int):
    """Exact (H, S) as nested lists of (Fraction re, Fraction im)."""
    A = np.asarray(A)
    B = np.asarray(B)
    N_G = A.shape[1]
    qA = [[_q(A[k, g]) for g in range(N_G)] for k in range(N_A * N_L)]
    qB = [[_q(B[k, g]) for g in range(N_G)] for k in range(N_A * N_L)]
    zero = (Fraction(0), Fraction(0))
    H = [[zero for _ in range(N_G)] for _ in range(N_G)]
    S = [[zero for _ in range(N_G)] for _ in range(N_G)]
    for a in range(N_A):
        base = a * N_L
        T = {
            ("A", "A"): [[_q(T_AA[a][i, j]) for j in range(N_L)] for i in range(N_L)],
            ("A", "B"): [[_q(T_AB[a][i, j]) for j in range(N_L)] for i in range(N_L)],
            # T^BA_{L',L} = conj(T^AB_{L,L'})
            ("B", "A"): [[_conj(_q(T_AB[a][j, i])) for j in range(N_L)] for i in range(N_L)],
            ("B", "B"): [[_q(T_BB[a][i, j]) for j in range(N_L)] for i in range(N_L)],
        }
        coef = {"A": qA, "B": qB}
        u2 = [Fraction(float(U[a][L])) ** 2 for L in range(N_L)]
        for gp in range(N_G):
            for g in range(N_G):
                s = S[gp][g]
                for L in range(N_L):
                    s = _add(s, _mul(_conj(qA[base + L][gp]), qA[base + L][g]))
                    bb = _mul(_conj(qB[base + L][gp]), qB[base + L][g])
                    s = _add(s, (bb[0] * u2[L], bb[1] * u2[L]))
                S[gp][g] = s
                h = H[gp][g]
                for X in ("A", "B"):
                    for Y in ("A", "B"):
                        TXY = T[(X, Y)]
                        cX = coef[X]
                        cY = coef[Y]
                        for Lp in range(N_L):
                            xc = _conj(cX[base + Lp][gp])
                            for L in range(N_L):
                                h = _add(h, _mul(_mul(xc, TXY[Lp][L]), cY[base + L][g]))
                H[gp][g] = h
    return H, S


def to_complex(M):
    """Round an exact (Fraction, Fraction) matrix to complex128."""
    return np.array([[complex(float(x[0]), float(x[1])) for x in row] for row in M])


def abs_sum_bound(A, B, T_AA, T_AB, T_BB, U, N_A: int, N_L: int):
    """Elementwise sum of |terms| of Eqs. (h), (s) (scale for rounding bounds)."""
    A = np.abs(np.asarray(A))
    B = np.abs(np.asarray(B))
    N_G = A.shape[1]
    Hb = np.zeros((N_G, N_G))
    Sb = np.zeros((N_G, N_G))
    for a in range(N_A):
        r = slice(a * N_L, (a + 1) * N_L)
        Aa, Ba = A[r], B[r]
        for X, TXY, Y in ((Aa, T_AA[a], Aa), (Aa, T_AB[a], Ba),
                          (Ba, np.conj(T_AB[a]).T, Aa), (Ba, T_BB[a], Ba)):
            Hb += X.T @ (np.abs(TXY) @ Y)
        Sb += Aa.T @ Aa + (U[a][:, None] ** 2 * Ba).T @ Ba
    return Hb, Sb
