"""FP64 reduction of the generalized eigenproblem of one k-point to standard form.

TEST INFRASTRUCTURE ONLY (see ``oracle/hs_oracle.py``): only tests, the smoke
check and the CPU legs of the benchmark call it; it shares no code with the
CUDA library.

Sec. 1.1: the H and S of one k-point define the generalized eigenvalue problem
sum_G' [H_GG' - lambda S_GG'] c_G' = 0, the consumer of the assembly.  S is an
overlap matrix, Hermitian positive definite, so the problem has the textbook
reduction to a standard Hermitian one (Golub & Van Loan, Matrix Computations,
Sec. 8.7.2):

    S = L L^H              (Cholesky, L lower triangular, real positive diagonal)
    C = L^{-1} H L^{-H}    (Hermitian; same eigenvalues; c = L^{-H} y)

This module writes that definition out: the Cholesky factor from the library
(numpy), with the column-oriented textbook routine of ``cholesky.py`` locating
the failing column when the library reports that S is not positive definite;
C from two triangular solves (scipy ``solve_triangular`` as a step):
X = L^{-1} H, then C = (L^{-1} X^H)^H.

Failure reading (the paper is silent; the zpotrf convention): the factorisation
proceeds column by column and fails at the first pivot that is not strictly
positive (zero, negative or NaN); ``fail_col`` is that column, 1-based, and
0 on success.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from .cholesky import cholesky_lower


def reduce_standard(H, S):
    """Return (L, C, fail_col) with S = L L^H and C = L^{-1} H L^{-H}.

    On failure (S not positive definite) L and C are None and fail_col > 0.
    """
    H = np.asarray(H, dtype=np.complex128)
    S = np.asarray(S, dtype=np.complex128)
    n = S.shape[0]
    if n == 0:
        return np.zeros((0, 0), np.complex128), np.zeros((0, 0), np.complex128), 0
    try:
        L = np.linalg.cholesky(S)
        ok = bool(np.all(np.isfinite(L)))
    except np.linalg.LinAlgError:
        ok = False
    if not ok:
        Lt, ok_t = cholesky_lower(S)
        if ok_t:  # the library refused a matrix the textbook test accepts
            raise RuntimeError("Cholesky failure tests disagree")
        d = np.array([np.nan])
        # the failing column: the first j whose pivot is not strictly positive
        for j in range(n):
            v = S[j, j] - Lt[j, :j] @ np.conj(Lt[j, :j])
            d = v.real
            if not d > 0.0:
                return None, None, j + 1
        raise RuntimeError("no failing pivot found")
    X = solve_triangular(L, H, lower=True)
    C = solve_triangular(L, X.conj().T, lower=True).conj().T
    return L, C, 0


def standard_eigenvalues(H, S):
    """Eigenvalues (ascending) of the generalized problem via the reduction."""
    L, C, fail = reduce_standard(H, S)
    if fail:
        raise ValueError(f"S is not positive definite (column {fail})")
    return np.linalg.eigvalsh(C)
