"""CPU FP64 oracle for the FLAPW Hamiltonian / overlap assembly.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library.

What it computes is the plain definition, not Algorithm 1:

* Eq. (h):  H = sum_a A_a^H T^AA_a A_a + A_a^H T^AB_a B_a
                      + B_a^H T^BA_a A_a + B_a^H T^BB_a B_a
* Eq. (s):  S = sum_a A_a^H A_a + B_a^H U_a^H U_a B_a

with A_a, B_a in C^{N_L x N_G} (rows a*N_L .. (a+1)*N_L-1 of the stacked
K x N_G arrays), T in C^{N_L x N_L} and U_a diagonal (sizes after Eq. (s)).
T^BA is not an input: Sec. 2 states it is the Hermitian transpose of T^AB, so
it is formed explicitly here.  U_a is the real diagonal of the norms
||udot_l^a||^2 appearing in the index form of S (Sec. 1.1, Eq. for S_{G',G});
the oracle takes U as given per (a, L).

Every product is evaluated atom by atom, unstacked, with both triangles of
H and S computed independently (no symmetry used).  A library matrix product
(numpy ``@``) serves as each step.

Readings of the paper taken here:
* T_AA, T_AB, T_BB are used as full matrices exactly as given.
* U is real, U_a = diag(U[a, :]), so U_a^H U_a = diag(U[a, :]^2).
"""
from __future__ import annotations

import numpy as np


def _atom_rows(a: int, N_L: int) -> slice:
    return slice(a * N_L, (a + 1) * N_L)


def assemble(A, B, T_AA, T_AB, T_BB, U, N_A: int, N_L: int, cols=None):
    """H and S by Eqs. (h) and (s).

    A, B: (K, N_G) complex128.  T_*: (N_A, N_L, N_L) complex128 (natural
    orientation, T[a][r, c]).  U: (N_A, N_L) float64.
    ``cols``: optional index array/slice of output columns G; returns the
    column panel H[:, cols], S[:, cols] (same arithmetic restricted to those
    columns), else the full N_G x N_G matrices.
    """
    A = np.asarray(A)
    B = np.asarray(B)
    N_G = A.shape[1]
    if cols is None:
        cols = slice(None)
    nc = np.arange(N_G)[cols].size
    H = np.zeros((N_G, nc), dtype=np.complex128)
    S = np.zeros((N_G, nc), dtype=np.complex128)
    for a in range(N_A):
        r = _atom_rows(a, N_L)
        Aa = A[r, :]
        Ba = B[r, :]
        Aa_c = Aa[:, cols]
        Ba_c = Ba[:, cols]
        T_BA = np.conj(T_AB[a]).T  # T^BA = (T^AB)^H, Sec. 2
        # Eq. (h), the four terms of atom a
        H += np.conj(Aa).T @ (T_AA[a] @ Aa_c)
        H += np.conj(Aa).T @ (T_AB[a] @ Ba_c)
        H += np.conj(Ba).T @ (T_BA @ Aa_c)
        H += np.conj(Ba).T @ (T_BB[a] @ Ba_c)
        # Eq. (s): A_a^H A_a + (U_a B_a)^H (U_a B_a)
        UBa = U[a][:, None] * Ba
        UBa_c = U[a][:, None] * Ba_c
        S += np.conj(Aa).T @ Aa_c
        S += np.conj(UBa).T @ UBa_c
    return H, S


def h_aa(A, T_AA, N_A: int, N_L: int):
    """H_AA = sum_a A_a^H T^AA_a A_a alone (the first under-brace of Eq. (h))."""
    A = np.asarray(A)
    N_G = A.shape[1]
    H = np.zeros((N_G, N_G), dtype=np.complex128)
    for a in range(N_A):
        Aa = A[_atom_rows(a, N_L), :]
        H += np.conj(Aa).T @ (T_AA[a] @ Aa)
    return H


def rel_frobenius(X, X_ref) -> float:
    """||X - X_ref||_F / ||X_ref||_F (the error measure used for parity)."""
    num = np.linalg.norm(np.asarray(X) - np.asarray(X_ref))
    den = np.linalg.norm(np.asarray(X_ref))
    return float(num / den) if den > 0 else float(num)
