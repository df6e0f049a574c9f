"""Seeded synthetic inputs for FLAPW H/S assembly (shared by the oracle tests,
the GPU tests, ``smoke()`` and ``bench.py``).

This module holds no arithmetic of the method itself: it only draws the
coefficient blocks A, B, the per-atom T matrices and the U norms with the
shapes and structure of Sec. 2 (matrix sizes after Eq. (s); N_L = (l_max+1)^2
and N_G ranges of Tab. 1) and of the Hermitian / positive-definite facts stated
for S, H and T in Sec. 1.1.  The physical inputs (NaCl, AuAg from FLEUR) are
not available, so these draws stand in for them.

Recipe (one tensor id per array, ``numpy.random.Philox(key=(seed, id))``):

* complex normal ``z = (x + i y)`` with ``x, y ~ N(0, 1/2)`` (so E|z|^2 = 1);
* ``A_a``, ``B_a``: complex normal, row ``L`` (0-based inside the atom)
  scaled by ``1 / (1 + floor(sqrt(L)))`` -- the angular-momentum ``l`` of
  the compound index ``L = (l, m)``;
* ``T_AA[a] = M M^H + N_L I`` (HPD, smallest eigenvalue >= N_L), except the
  "indefinite" atoms where the diagonal is shifted by ``-2 N_L``;
* ``T_AB[a]``: complex normal; ``T_BB[a] = (N + N^H) / 2``;
* every Hermitian draw is symmetrised exactly, ``T <- (T + T^H) / 2``;
* ``U[a, L]``: uniform in [0.5, 2].

Real-symmetric variant (``make_inputs_real``; Sec. 1.1: real H and S for systems
with inversion symmetry): the same recipe with real normal draws ``N(0, 1)``,
``T_AA = M M^T + N_L I`` (or shifted), ``T_BB = (N + N^T) / 2``, from streams of
their own (tensor id + 100).

Generalized-eigenproblem reduction inputs (``reduce_inputs``; Sec. 1.1: H is
Hermitian, S Hermitian positive definite): ``S = Q diag(s) Q^H`` with ``Q`` the
unitary factor of the QR of an ``n x n`` complex normal draw and ``s`` log-spaced
from ``1/cond`` to 1, ``H = (N + N^H) / 2`` with ``N`` complex normal (tensor ids
20, 21), both symmetrised exactly.

Device draws (``make_inputs_device``, for the benchmark's large shapes, where
drawing 14 GB of coefficients on the host would take a minute): A and B with the
same distribution (``torch.randn`` complex128 gives re, im ~ N(0, 1/2); rows scaled
by ``1 / (1 + l)``) from torch's counter-based (Philox) CUDA generator seeded with
``seed * 1000003 + tensor id``; T and U from the host recipe above.  A different
stream from the host draws, so the values differ; the shapes, distributions and
structure are the same.

Matching-coefficient inputs (``matching_inputs``; Sec. 1.1: the basis functions are
plane waves e^{i(k+G).r} outside the muffin-tin spheres and radial functions times
spherical harmonics inside): a cubic cell of side ``a`` with volume ``Omega = a^3``
sized so that N_G plane waves reach |k+G| <= K_max = (l_max + 1) / 2.2 (the usual
R K_max ~ l_max balance); a k-point uniform in the Brillouin zone; the N_G vectors
k + G (G on the reciprocal lattice of spacing 2 pi / a) of smallest length; atom
positions uniform in the cell; sphere radii R uniform in [1.6, 2.2]; per (atom, l)
radial boundary values u(R) ~ U[0.5, 1.5], u'(R) ~ U[-1, 1], udot(R) ~ U[-0.5, 0.5]
and udot'(R) chosen so that the Wronskian u udot' - u' udot equals 1 / R^2 (the
normalisation of a radial function and its energy derivative), tensor ids 30-33.

Indefinite atoms: ``n_f = round(frac * N_A)`` atoms at
``(3 + floor(i * N_A / n_f)) mod N_A`` for ``i < n_f``.

Memory layout (identical to the C ABI, BLAS column-major):

* ``A``, ``B``: numpy arrays of shape ``(K, N_G)``, ``K = N_A * N_L``,
  Fortran order (each column of length K is contiguous; atom ``a`` owns
  rows ``[a*N_L, (a+1)*N_L)``);
* ``T_AA``, ``T_AB``, ``T_BB``: shape ``(N_A, N_L, N_L)`` in natural math
  orientation (``T[a][r, c]``); ``as_colmajor_T`` gives the ABI order;
* ``U``: shape ``(N_A, N_L)`` float64, C order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# tensor ids of the counter-based streams
_ID_A, _ID_B, _ID_TAA, _ID_TAB, _ID_TBB, _ID_U = 1, 2, 3, 4, 5, 6
_ID_RH, _ID_RS = 20, 21


@dataclasses.dataclass(frozen=True)
class Workload:
    """One k-point assembly problem: sizes plus the indefinite-atom fraction."""
    name: str
    N_A: int
    N_L: int
    N_G: int
    indefinite: tuple  # 0-based atom indices whose T_AA is indefinite
    seed: int = 0

    @property
    def K(self) -> int:
        return self.N_A * self.N_L


def indefinite_atoms(N_A: int, frac: float) -> tuple:
    """Atoms given an indefinite T_AA: n_f = round(frac*N_A), spread from atom 3."""
    n_f = int(round(frac * N_A))
    if n_f <= 0:
        return ()
    return tuple(sorted({(3 + (i * N_A) // n_f) % N_A for i in range(n_f)}))


# The five problem shapes.  "tiny" is small enough for the oracle in a second;
# the paper-scale shapes follow Tab. 1 (N_L = 121 = (10+1)^2 as AuAg,
# N_G in the K_max range) and the sizes stated after Eq. (s).
WORKLOADS = {
    "tiny": Workload("tiny", 4, 16, 256, (3,)),
    "auag_like_4000": Workload("auag_like_4000", 100, 121, 4000, indefinite_atoms(100, 0.05)),
    "large_12000": Workload("large_12000", 256, 144, 12000, indefinite_atoms(256, 0.02)),
    "split_8000": Workload("split_8000", 100, 121, 8000, indefinite_atoms(100, 0.05)),
    # half the atoms of auag_like at N_G = 2048: every input still larger than
    # L2, a few GB on the device in split mode (kernel profiling case)
    "profile_2048": Workload("profile_2048", 50, 121, 2048, indefinite_atoms(50, 0.05)),
}


def _rng(seed: int, tid: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed, tid * 1_000_003 + sub]))


def _cnormal(rng: np.random.Generator, shape) -> np.ndarray:
    x = rng.standard_normal(size=(2,) + tuple(shape))
    s = math.sqrt(0.5)
    return (x[0] * s) + 1j * (x[1] * s)


def _herm(T: np.ndarray) -> np.ndarray:
    """Exact Hermitian symmetrisation (T + T^H)/2 on the last two axes."""
    return 0.5 * (T + np.conj(np.swapaxes(T, -1, -2)))


def l_of_L(N_L: int) -> np.ndarray:
    """Angular momentum l of each compound row index L = l^2 + l + m (0-based)."""
    return np.floor(np.sqrt(np.arange(N_L))).astype(np.int64)


def coefficients(N_A: int, N_L: int, N_G: int, seed: int = 0, tid: int = _ID_A,
                 col0: int = 0, chunk: int = 512) -> np.ndarray:
    """A complex (K, N_G) Fortran-order coefficient matrix (A or B).

    Columns are drawn in independent chunks of ``chunk`` columns (one Philox
    stream per chunk) so any column range can be regenerated on its own;
    ``col0`` is the global index of the first returned column.
    """
    K = N_A * N_L
    scale = 1.0 / (1.0 + l_of_L(N_L).astype(np.float64))
    rowscale = np.tile(scale, N_A)  # (K,)
    out = np.empty((N_G, K), dtype=np.complex128)  # C order: row g = column g
    g = 0
    while g < N_G:
        gg = col0 + g
        c = gg // chunk
        lo = gg - c * chunk
        n = min(chunk - lo, N_G - g)
        blk = _cnormal(_rng(seed, tid, c), (chunk, K))[lo:lo + n]
        out[g:g + n] = blk * rowscale[None, :]
        g += n
    return out.T  # (K, N_G), Fortran order


def t_matrices(N_A: int, N_L: int, indefinite=(), seed: int = 0):
    """(T_AA, T_AB, T_BB), each (N_A, N_L, N_L) complex128, natural orientation."""
    M = _cnormal(_rng(seed, _ID_TAA), (N_A, N_L, N_L))
    T_AA = M @ np.conj(np.swapaxes(M, -1, -2))
    eye = np.eye(N_L)
    T_AA = T_AA + N_L * eye[None]
    for a in indefinite:
        T_AA[a] -= 2 * N_L * eye
    T_AA = _herm(T_AA)
    T_AB = _cnormal(_rng(seed, _ID_TAB), (N_A, N_L, N_L))
    N = _cnormal(_rng(seed, _ID_TBB), (N_A, N_L, N_L))
    T_BB = _herm(N)
    return T_AA, T_AB, T_BB


def u_norms(N_A: int, N_L: int, seed: int = 0) -> np.ndarray:
    return _rng(seed, _ID_U).uniform(0.5, 2.0, size=(N_A, N_L))


def make_inputs(w: Workload, cols: slice | None = None):
    """Draw every input of workload ``w``.

    Returns dict with A, B (K, N_G or the requested column range), T_AA, T_AB,
    T_BB (N_A, N_L, N_L) and U (N_A, N_L).
    """
    if cols is None:
        c0, n = 0, w.N_G
    else:
        c0, c1, _ = cols.indices(w.N_G)
        n = c1 - c0
    A = coefficients(w.N_A, w.N_L, n, w.seed, _ID_A, col0=c0)
    B = coefficients(w.N_A, w.N_L, n, w.seed, _ID_B, col0=c0)
    T_AA, T_AB, T_BB = t_matrices(w.N_A, w.N_L, w.indefinite, w.seed)
    U = u_norms(w.N_A, w.N_L, w.seed)
    return dict(A=A, B=B, T_AA=T_AA, T_AB=T_AB, T_BB=T_BB, U=U)


_REAL = 100  # tensor-id offset of the real-variant streams


def coefficients_real(N_A: int, N_L: int, N_G: int, seed: int = 0, tid: int = _ID_A,
                      col0: int = 0, chunk: int = 512) -> np.ndarray:
    """A real (K, N_G) Fortran-order coefficient matrix, rows scaled as the complex one."""
    K = N_A * N_L
    rowscale = np.tile(1.0 / (1.0 + l_of_L(N_L).astype(np.float64)), N_A)
    out = np.empty((N_G, K), dtype=np.float64)
    g = 0
    while g < N_G:
        gg = col0 + g
        c = gg // chunk
        lo = gg - c * chunk
        n = min(chunk - lo, N_G - g)
        blk = _rng(seed, tid + _REAL, c).standard_normal(size=(chunk, K))[lo:lo + n]
        out[g:g + n] = blk * rowscale[None, :]
        g += n
    return out.T


def t_matrices_real(N_A: int, N_L: int, indefinite=(), seed: int = 0):
    """Real (T_AA, T_AB, T_BB), each (N_A, N_L, N_L), natural orientation; T_AA, T_BB
    exactly symmetric."""
    M = _rng(seed, _ID_TAA + _REAL).standard_normal(size=(N_A, N_L, N_L))
    T_AA = M @ np.swapaxes(M, -1, -2)
    eye = np.eye(N_L)
    T_AA = T_AA + N_L * eye[None]
    for a in indefinite:
        T_AA[a] -= 2 * N_L * eye
    T_AA = 0.5 * (T_AA + np.swapaxes(T_AA, -1, -2))
    T_AB = _rng(seed, _ID_TAB + _REAL).standard_normal(size=(N_A, N_L, N_L))
    N = _rng(seed, _ID_TBB + _REAL).standard_normal(size=(N_A, N_L, N_L))
    T_BB = 0.5 * (N + np.swapaxes(N, -1, -2))
    return T_AA, T_AB, T_BB


def make_inputs_real(w: Workload, cols: slice | None = None):
    """Real-variant inputs of workload ``w`` (same keys and shapes as make_inputs)."""
    if cols is None:
        c0, n = 0, w.N_G
    else:
        c0, c1, _ = cols.indices(w.N_G)
        n = c1 - c0
    A = coefficients_real(w.N_A, w.N_L, n, w.seed, _ID_A, col0=c0)
    B = coefficients_real(w.N_A, w.N_L, n, w.seed, _ID_B, col0=c0)
    T_AA, T_AB, T_BB = t_matrices_real(w.N_A, w.N_L, w.indefinite, w.seed)
    U = u_norms(w.N_A, w.N_L, w.seed)
    return dict(A=A, B=B, T_AA=T_AA, T_AB=T_AB, T_BB=T_BB, U=U)


def reduce_inputs(n: int, seed: int = 0, cond: float = 1e3):
    """(H, S): n x n complex, Fortran order; S Hermitian positive definite with
    2-norm condition number ``cond`` (up to rounding), H Hermitian."""
    G = _cnormal(_rng(seed, _ID_RS), (n, n))
    Q, R = np.linalg.qr(G)
    Q = Q * (np.diag(R) / np.abs(np.where(np.diag(R) == 0, 1, np.diag(R))))  # unique phase
    s = np.logspace(-math.log10(cond), 0.0, n) if n > 1 else np.ones(1)
    S = _herm((Q * s) @ Q.conj().T)
    H = _herm(_cnormal(_rng(seed, _ID_RH), (n, n)))
    return np.asfortranarray(H), np.asfortranarray(S)


def coefficients_device(N_A: int, N_L: int, N_G: int, device, seed: int = 0,
                        tid: int = _ID_A):
    """A complex (K, N_G) column-major CUDA tensor (strides (1, K)) drawn on the device
    with the coefficient recipe (complex normal, rows scaled by 1 / (1 + l))."""
    import torch
    K = N_A * N_L
    g = torch.Generator(device=device)
    g.manual_seed(seed * 1_000_003 + tid)
    x = torch.randn((N_G, K), generator=g, device=device, dtype=torch.complex128)
    rowscale = torch.from_numpy(np.tile(1.0 / (1.0 + l_of_L(N_L).astype(np.float64)), N_A))
    x.mul_(rowscale.to(device)[None, :])
    return x.T


def make_inputs_device(w: Workload, device):
    """Inputs of workload ``w`` with A, B drawn on ``device`` (see the module notes);
    T_AA, T_AB, T_BB (N_A, N_L, N_L) and U (N_A, N_L) as numpy arrays (host recipe)."""
    A = coefficients_device(w.N_A, w.N_L, w.N_G, device, w.seed, _ID_A)
    B = coefficients_device(w.N_A, w.N_L, w.N_G, device, w.seed, _ID_B)
    T_AA, T_AB, T_BB = t_matrices(w.N_A, w.N_L, w.indefinite, w.seed)
    U = u_norms(w.N_A, w.N_L, w.seed)
    return dict(A=A, B=B, T_AA=T_AA, T_AB=T_AB, T_BB=T_BB, U=U)


_ID_KPT, _ID_TAU, _ID_RMT, _ID_UFUN = 30, 31, 32, 33


def matching_inputs(N_A: int, l_max: int, N_G: int, seed: int = 0):
    """Inputs of the matching step: dict with Kvec (N_G, 3) wave vectors k + G, tau
    (N_A, 3) atom positions, R (N_A,) sphere radii, ufun (N_A, l_max + 1, 4) radial
    boundary values u, u', udot, udot' at R, omega (cell volume), a (cell side)."""
    K_max = (l_max + 1) / 2.2
    omega = 6.0 * math.pi ** 2 * N_G / K_max ** 3  # N_G ~ Omega K_max^3 / (6 pi^2)
    a = omega ** (1.0 / 3.0)
    b = 2.0 * math.pi / a
    k = (_rng(seed, _ID_KPT).uniform(-0.5, 0.5, size=3)) * b
    nmax = int(math.ceil(K_max / b)) + 3
    while True:
        r = np.arange(-nmax, nmax + 1)
        n = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
        K = k[None, :] + b * n
        if len(K) >= 2 * N_G:
            break
        nmax += 2
    order = np.argsort(np.linalg.norm(K, axis=1), kind="stable")
    Kvec = K[order[:N_G]]
    tau = _rng(seed, _ID_TAU).uniform(0.0, 1.0, size=(N_A, 3)) * a
    R = _rng(seed, _ID_RMT).uniform(1.6, 2.2, size=N_A)
    g = _rng(seed, _ID_UFUN)
    u = g.uniform(0.5, 1.5, size=(N_A, l_max + 1))
    du = g.uniform(-1.0, 1.0, size=(N_A, l_max + 1))
    ud = g.uniform(-0.5, 0.5, size=(N_A, l_max + 1))
    dud = (1.0 / R[:, None] ** 2 + du * ud) / u  # Wronskian u udot' - u' udot = 1 / R^2
    ufun = np.stack([u, du, ud, dud], axis=-1)
    return dict(Kvec=Kvec, tau=tau, R=R, ufun=ufun, omega=omega, a=a)


def as_colmajor_T(T: np.ndarray) -> np.ndarray:
    """(N_A, N_L, N_L) natural -> C-contiguous buffer holding each T_a column-major."""
    return np.ascontiguousarray(np.swapaxes(T, -1, -2))
