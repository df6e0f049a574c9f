"""Textbook FP64 Cholesky of each T^AA_a, with LAPACK-style failure test.

TEST INFRASTRUCTURE ONLY (see ``oracle/hs_oracle.py``).

Sec. 2 tries a Cholesky factorisation of every T^AA_a and falls back to a
plain Hermitian product for atoms whose factorisation fails (Algorithm 1,
second part of H).  The paper does not define "fails"; the reading taken is
the usual one (zpotrf): the factorisation of the lower triangle proceeds
column by column and fails at the first pivot

    d_j = Re(T_jj) - sum_{k<j} |L_jk|^2

that is not strictly positive (zero, negative or NaN).  On success
T = L L^H with L lower triangular and real positive diagonal.

Algorithm: column-oriented ("gaxpy") Cholesky, Golub & Van Loan, Matrix
Computations, Sec. 4.2, restated for complex Hermitian matrices.  Only the
lower triangle of T is read.
"""
from __future__ import annotations

import numpy as np


def cholesky_lower(T):
    """Return (L, ok).  L is lower triangular with T = L L^H when ok."""
    T = np.asarray(T, dtype=np.complex128)
    n = T.shape[0]
    L = np.zeros_like(T)
    for j in range(n):
        # v = T[j:, j] - L[j:, :j] conj(L[j, :j])
        v = T[j:, j] - L[j:, :j] @ np.conj(L[j, :j])
        d = v[0].real
        if not d > 0.0:  # also catches NaN
            return L, False
        ljj = np.sqrt(d)
        L[j, j] = ljj
        L[j + 1:, j] = v[1:] / ljj
    return L, True


def fail_flags(T_AA):
    """fail[a] = 1 where the Cholesky of T_AA[a] fails, else 0."""
    return np.array([0 if cholesky_lower(T)[1] else 1 for T in T_AA], dtype=np.int32)
