"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

No GPU.  Each test is chosen so that a plausible slip in the oracle (a dropped
term of Eq. (h)/(s), T^BA not conjugate-transposed, U applied once instead of
squared, a wrong atom-row offset, a transposed operand) fails at least one:

* exact rational brute force of the index forms (Sec. 1.1) on tiny inputs;
* closed forms: T = I gives H = (A+B)^H (A+B); S = C^H C with C the
  row-stacked [A; U B] (Sec. 2's stacking argument);
* invariants: H and S Hermitian (Sec. 1.1); rank(S) = min(N_G, 2 N_A N_L)
  and S positive definite when 2 N_A N_L >= N_G; atom-permutation
  invariance; column-permutation equivariance; linearity in T;
* the textbook Cholesky against LAPACK (numpy) and its failure semantics.
"""
import numpy as np
import pytest

from oracle import assemble, h_aa, rel_frobenius, cholesky_lower, fail_flags
from oracle import brute
from paper_1611_00606_gb300 import synth

EPS = np.finfo(np.float64).eps


def _inputs(N_A, N_L, N_G, indefinite=(), seed=0):
    w = synth.Workload("t", N_A, N_L, N_G, tuple(indefinite), seed)
    return synth.make_inputs(w)


def _run(d, N_A, N_L, **kw):
    return assemble(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L, **kw)


@pytest.mark.parametrize("N_A,N_L,N_G,indef", [(1, 1, 1, ()), (2, 4, 5, (1,)), (3, 4, 8, (0,))])
def test_exact_brute_force(N_A, N_L, N_G, indef):
    d = _inputs(N_A, N_L, N_G, indef, seed=7)
    H, S = _run(d, N_A, N_L)
    He, Se = brute.exact_hs(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    He, Se = brute.to_complex(He), brute.to_complex(Se)
    Hb, Sb = brute.abs_sum_bound(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    # standard dot-product rounding bound, n = number of summed products
    n = 4 * N_A * N_L * N_L + 8
    assert np.all(np.abs(H - He) <= n * EPS * Hb + 1e-300)
    assert np.all(np.abs(S - Se) <= n * EPS * Sb + 1e-300)


def test_brute_force_detects_transposed_tba():
    """A reading that forgets the conjugate transpose of T^AB is far from exact."""
    N_A, N_L, N_G = 2, 4, 5
    d = _inputs(N_A, N_L, N_G, seed=3)
    He, _ = brute.exact_hs(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    He = brute.to_complex(He)
    wrong = np.zeros_like(He)
    for a in range(N_A):
        r = slice(a * N_L, (a + 1) * N_L)
        Aa, Ba = d["A"][r], d["B"][r]
        wrong += Aa.conj().T @ d["T_AA"][a] @ Aa + Aa.conj().T @ d["T_AB"][a] @ Ba
        wrong += Ba.conj().T @ d["T_AB"][a] @ Aa + Ba.conj().T @ d["T_BB"][a] @ Ba
    assert rel_frobenius(wrong, He) > 1e-3


def test_identity_T_closed_form():
    N_A, N_L, N_G = 3, 9, 40
    d = _inputs(N_A, N_L, N_G, seed=1)
    I = np.broadcast_to(np.eye(N_L, dtype=np.complex128), (N_A, N_L, N_L)).copy()
    ones = np.ones((N_A, N_L))
    H, S = assemble(d["A"], d["B"], I, I, I, ones, N_A, N_L)
    C = d["A"] + d["B"]
    assert rel_frobenius(H, C.conj().T @ C) < 1e-14
    St = np.vstack([d["A"], d["B"]])
    assert rel_frobenius(S, St.conj().T @ St) < 1e-14


def test_overlap_stacked_closed_form():
    N_A, N_L, N_G = 4, 16, 64
    d = _inputs(N_A, N_L, N_G, seed=2)
    _, S = _run(d, N_A, N_L)
    C = np.vstack([d["A"], d["U"].reshape(-1)[:, None] * d["B"]])
    assert rel_frobenius(S, C.conj().T @ C) < 1e-14


def test_haa_identity_equals_overlap_of_A():
    """B = 0, T^AA = I: H = A^H A = S."""
    N_A, N_L, N_G = 3, 16, 50
    d = _inputs(N_A, N_L, N_G, seed=4)
    Z = np.zeros_like(d["B"])
    I = np.broadcast_to(np.eye(N_L, dtype=np.complex128), (N_A, N_L, N_L)).copy()
    H, S = assemble(d["A"], Z, I, d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    assert rel_frobenius(H, S) < 1e-14
    assert rel_frobenius(h_aa(d["A"], I, N_A, N_L), S) < 1e-14


@pytest.mark.parametrize("N_A,N_L,N_G,indef", [(2, 4, 5, ()), (3, 4, 6, (1,))])
def test_haa_general_hermitian_T_exact(N_A, N_L, N_G, indef):
    """H_AA at a general Hermitian T^AA (complex off-diagonal entries) against the exact
    index form with B = 0, where Eq. (h) reduces to its first under-brace.  A slip that
    applies T^T (= conj(T) for Hermitian T) or conj(A) on the wrong side is caught."""
    d = _inputs(N_A, N_L, N_G, indef, seed=13)
    T = d["T_AA"]
    assert np.abs(T - np.conj(np.swapaxes(T, -1, -2))).max() == 0      # Hermitian
    assert np.abs(np.imag(T[:, 0, 1])).min() > 0                        # not real
    Z = np.zeros_like(d["B"])
    He, _ = brute.exact_hs(d["A"], Z, T, d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    He = brute.to_complex(He)
    Hb, _ = brute.abs_sum_bound(d["A"], Z, T, d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    n = N_L * N_L + 4
    H = h_aa(d["A"], T, N_A, N_L)
    assert np.all(np.abs(H - He) <= n * EPS * Hb + 1e-300)
    # the same H_AA is the whole H of Eq. (h) when B = 0
    Hf, _ = assemble(d["A"], Z, T, d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    assert rel_frobenius(Hf, He) < 1e-14
    # negative controls: transposed T, conjugate on the right-hand factor
    wrong_t = np.zeros_like(He)
    wrong_c = np.zeros_like(He)
    for a in range(N_A):
        Aa = d["A"][a * N_L:(a + 1) * N_L]
        wrong_t += Aa.conj().T @ T[a].T @ Aa
        wrong_c += Aa.T @ T[a] @ Aa.conj()
    assert rel_frobenius(wrong_t, He) > 1e-3
    assert rel_frobenius(wrong_c, He) > 1e-3


def test_haa_matches_assemble_with_zero_b_at_scale():
    """B = 0 at a paper-like shape with indefinite atoms: h_aa equals the full
    definition (both pinned by the exact index form at tiny sizes)."""
    N_A, N_L, N_G = 5, 49, 300
    d = _inputs(N_A, N_L, N_G, (1, 3), seed=14)
    Z = np.zeros_like(d["B"])
    Hf, _ = assemble(d["A"], Z, d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    assert rel_frobenius(h_aa(d["A"], d["T_AA"], N_A, N_L), Hf) < 1e-14


def test_hermitian():
    N_A, N_L, N_G = 4, 16, 256
    d = _inputs(N_A, N_L, N_G, (3,), seed=0)
    H, S = _run(d, N_A, N_L)
    assert rel_frobenius(H, H.conj().T) < 1e-14
    assert rel_frobenius(S, S.conj().T) < 1e-14


def test_overlap_rank_deficient_tiny():
    """tiny shape: 2 N_A N_L = 128 < N_G = 256, so S is PSD with rank 128."""
    w = synth.WORKLOADS["tiny"]
    d = synth.make_inputs(w)
    _, S = _run(d, w.N_A, w.N_L)
    ev = np.linalg.eigvalsh(0.5 * (S + S.conj().T))
    top = ev.max()
    r = 2 * w.N_A * w.N_L
    assert np.all(np.abs(ev[: w.N_G - r]) < 1e-12 * top)
    assert ev[w.N_G - r] > 1e-6 * top


def test_overlap_positive_definite_when_full_rank():
    N_A, N_L, N_G = 4, 16, 100  # 2 N_A N_L = 128 >= 100
    d = _inputs(N_A, N_L, N_G, seed=5)
    _, S = _run(d, N_A, N_L)
    np.linalg.cholesky(0.5 * (S + S.conj().T))  # raises if not PD
    assert np.linalg.eigvalsh(0.5 * (S + S.conj().T)).min() > 0


def test_atom_permutation_invariance():
    N_A, N_L, N_G = 4, 9, 30
    d = _inputs(N_A, N_L, N_G, (2,), seed=6)
    H, S = _run(d, N_A, N_L)
    perm = np.array([2, 0, 3, 1])
    rows = np.concatenate([np.arange(a * N_L, (a + 1) * N_L) for a in perm])
    dp = dict(A=d["A"][rows], B=d["B"][rows], T_AA=d["T_AA"][perm], T_AB=d["T_AB"][perm],
              T_BB=d["T_BB"][perm], U=d["U"][perm])
    Hp, Sp = _run(dp, N_A, N_L)
    assert rel_frobenius(Hp, H) < 1e-14 and rel_frobenius(Sp, S) < 1e-14


def test_column_permutation_equivariance():
    N_A, N_L, N_G = 3, 9, 30
    d = _inputs(N_A, N_L, N_G, seed=8)
    H, S = _run(d, N_A, N_L)
    p = np.random.default_rng(0).permutation(N_G)
    dp = dict(d, A=d["A"][:, p], B=d["B"][:, p])
    Hp, Sp = _run(dp, N_A, N_L)
    assert rel_frobenius(Hp, H[np.ix_(p, p)]) < 1e-14
    assert rel_frobenius(Sp, S[np.ix_(p, p)]) < 1e-14


def test_linearity_in_T():
    N_A, N_L, N_G = 2, 9, 20
    d1 = _inputs(N_A, N_L, N_G, seed=9)
    d2 = _inputs(N_A, N_L, N_G, seed=10)
    dsum = dict(d1, T_AA=d1["T_AA"] + d2["T_AA"], T_AB=d1["T_AB"] + d2["T_AB"],
                T_BB=d1["T_BB"] + d2["T_BB"])
    d2b = dict(d1, T_AA=d2["T_AA"], T_AB=d2["T_AB"], T_BB=d2["T_BB"])
    H1, _ = _run(d1, N_A, N_L)
    H2, _ = _run(d2b, N_A, N_L)
    Hs, _ = _run(dsum, N_A, N_L)
    assert rel_frobenius(Hs, H1 + H2) < 1e-14


def test_single_column_is_real():
    N_A, N_L = 3, 16
    d = _inputs(N_A, N_L, 1, seed=11)
    H, S = _run(d, N_A, N_L)
    assert abs(H[0, 0].imag) <= 1e-14 * abs(H[0, 0])
    assert abs(S[0, 0].imag) <= 1e-14 * abs(S[0, 0]) and S[0, 0].real > 0


def test_column_panel_matches_full():
    N_A, N_L, N_G = 3, 9, 40
    d = _inputs(N_A, N_L, N_G, (1,), seed=12)
    H, S = _run(d, N_A, N_L)
    cols = np.array([0, 7, 39])
    Hp, Sp = _run(d, N_A, N_L, cols=cols)
    assert np.array_equal(Hp.shape, (N_G, 3))
    assert rel_frobenius(Hp, H[:, cols]) < 1e-15 and rel_frobenius(Sp, S[:, cols]) < 1e-15


def test_cholesky_matches_lapack_and_flags():
    w = synth.WORKLOADS["tiny"]
    d = synth.make_inputs(w)
    for a in range(w.N_A):
        L, ok = cholesky_lower(d["T_AA"][a])
        if a in w.indefinite:
            assert not ok
            with pytest.raises(np.linalg.LinAlgError):
                np.linalg.cholesky(d["T_AA"][a])
        else:
            assert ok
            assert rel_frobenius(L @ L.conj().T, d["T_AA"][a]) < 1e-14
            assert rel_frobenius(L, np.linalg.cholesky(d["T_AA"][a])) < 1e-13
    assert list(np.nonzero(fail_flags(d["T_AA"]))[0]) == list(w.indefinite)


def test_cholesky_reads_lower_triangle_only_and_nan_fails():
    T = synth.t_matrices(1, 8, ())[0][0]
    Tl = np.tril(T) + np.triu(np.full_like(T, 1e300), 1)
    L, ok = cholesky_lower(Tl)
    assert ok and rel_frobenius(L @ L.conj().T, T) < 1e-14
    Tn = T.copy()
    Tn[3, 3] = np.nan
    assert not cholesky_lower(Tn)[1]
    Tz = np.zeros((4, 4), dtype=np.complex128)
    assert not cholesky_lower(Tz)[1]


def test_indefinite_recipe_spreads_atoms():
    assert synth.indefinite_atoms(100, 0.05) == (3, 23, 43, 63, 83)
    assert synth.indefinite_atoms(256, 0.02) == (3, 54, 105, 156, 207)
    assert synth.WORKLOADS["tiny"].indefinite == (3,)


# ---- real-symmetric variant (Sec. 1.1: real H, S with inversion symmetry)

def _inputs_real(N_A, N_L, N_G, indefinite=(), seed=0):
    return synth.make_inputs_real(synth.Workload("r", N_A, N_L, N_G, tuple(indefinite), seed))


def test_real_inputs_give_real_symmetric_outputs():
    N_A, N_L, N_G = 3, 9, 40
    d = _inputs_real(N_A, N_L, N_G, (1,), seed=21)
    assert d["A"].dtype == np.float64 and np.array_equal(d["T_AA"], np.swapaxes(d["T_AA"], 1, 2))
    H, S = _run(d, N_A, N_L)
    assert np.max(np.abs(H.imag)) == 0.0 and np.max(np.abs(S.imag)) == 0.0
    for X in (H.real, S.real):
        assert np.linalg.norm(X - X.T) <= 8 * EPS * np.linalg.norm(X)


@pytest.mark.parametrize("N_A,N_L,N_G,indef", [(2, 4, 5, (1,)), (3, 4, 8, (0,))])
def test_real_exact_brute_force(N_A, N_L, N_G, indef):
    d = _inputs_real(N_A, N_L, N_G, indef, seed=9)
    H, S = _run(d, N_A, N_L)
    He, Se = brute.exact_hs(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    He, Se = brute.to_complex(He), brute.to_complex(Se)
    assert np.max(np.abs(He.imag)) == 0.0  # the definition itself is real here
    Hb, Sb = brute.abs_sum_bound(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    n = 4 * N_A * N_L * N_L + 8  # dot-product rounding bound, as for the complex case
    assert np.all(np.abs(H - He) <= n * EPS * Hb + 1e-300)
    assert np.all(np.abs(S - Se) <= n * EPS * Sb + 1e-300)


def test_real_transposed_tab_enters_as_tba():
    """With real T, T^BA = (T^AB)^T: H is invariant under swapping (A, B) together with
    (T^AA, T^BB) and transposing T^AB (the two cross terms trade places)."""
    N_A, N_L, N_G = 2, 5, 12
    d = _inputs_real(N_A, N_L, N_G, (), seed=4)
    H, _ = _run(d, N_A, N_L)
    H2, _ = assemble(d["B"], d["A"], d["T_BB"], np.swapaxes(d["T_AB"], 1, 2), d["T_AA"], d["U"],
                     N_A, N_L)
    assert rel_frobenius(H2, H) <= 16 * EPS


# ---------------------------------------------------------------------------
# Generalized-eigenproblem reduction (Sec. 1.1: H c = lambda S c), oracle/reduce.py

from oracle.reduce import reduce_standard, standard_eigenvalues  # noqa: E402


def test_reduce_identity_overlap_is_exact():
    # S = I: L = I and C = H, exactly
    H, _ = synth.reduce_inputs(9, seed=3)
    L, C, fail = reduce_standard(H, np.eye(9, dtype=np.complex128))
    assert fail == 0
    assert np.array_equal(L, np.eye(9))
    assert np.array_equal(C, H)


def test_reduce_diagonal_overlap_closed_form():
    # S = diag(d): L = diag(sqrt d), C_ij = H_ij / sqrt(d_i d_j)
    d = np.array([1.0, 4.0, 9.0, 0.25, 16.0, 2.25])
    H, _ = synth.reduce_inputs(6, seed=4)
    L, C, fail = reduce_standard(H, np.diag(d).astype(np.complex128))
    assert fail == 0
    assert np.allclose(L, np.diag(np.sqrt(d)), rtol=0, atol=1e-15)
    r = np.sqrt(d)
    assert np.allclose(C, H / np.outer(r, r), rtol=1e-15, atol=1e-15)


def test_reduce_2x2_eigenvalues_closed_form():
    # det(H - lam S) = 0 for 2 x 2: a lam^2 + b lam + c = 0 with a = det S,
    # b = -(h11 s22 + h22 s11 - 2 Re(h12 conj(s12))), c = det H
    H = np.array([[2.0, 1.0 - 2.0j], [1.0 + 2.0j, -3.0]])
    S = np.array([[4.0, 1.0 + 1.0j], [1.0 - 1.0j, 3.0]])
    a = (S[0, 0] * S[1, 1] - abs(S[0, 1]) ** 2).real
    b = -(H[0, 0] * S[1, 1] + H[1, 1] * S[0, 0] - 2 * (H[0, 1] * np.conj(S[0, 1])).real).real
    c = (H[0, 0] * H[1, 1] - abs(H[0, 1]) ** 2).real
    disc = np.sqrt(b * b - 4 * a * c)
    lam = np.sort([(-b - disc) / (2 * a), (-b + disc) / (2 * a)])
    assert np.allclose(standard_eigenvalues(H, S), lam, rtol=1e-14, atol=1e-14)


def test_reduce_invariants_fix_l_and_c():
    # L lower with real positive diagonal and L L^H = S fix L uniquely; L C L^H = H
    # then fixes C.  A transposed factor, a dropped conjugate or a one-sided
    # transform breaks one of them.
    H, S = synth.reduce_inputs(40, seed=5, cond=1e3)
    L, C, fail = reduce_standard(H, S)
    assert fail == 0
    assert np.array_equal(L, np.tril(L))
    assert np.all(np.diag(L).imag == 0) and np.all(np.diag(L).real > 0)
    assert rel_frobenius(L @ L.conj().T, S) < 1e-14
    assert rel_frobenius(L @ C @ L.conj().T, H) < 1e-13
    assert rel_frobenius(C, C.conj().T) < 1e-14


def test_reduce_eigenvalues_match_unsymmetric_route():
    # eigenvalues of C = those of S^{-1} H, computed by a general (non-Hermitian)
    # eigensolver that shares no step with the reduction
    H, S = synth.reduce_inputs(30, seed=6, cond=50.0)
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(S, H)).real)
    assert np.allclose(standard_eigenvalues(H, S), ev, rtol=1e-11, atol=1e-11)


def test_reduce_factor_matches_textbook_cholesky():
    H, S = synth.reduce_inputs(25, seed=7)
    L, _, _ = reduce_standard(H, S)
    Lt, ok = cholesky_lower(S)
    assert ok and np.allclose(L, Lt, rtol=0, atol=1e-13)


def test_reduce_not_positive_definite_reports_column():
    # S = L0 L0^H with small integers and L0[2, 2] = 0: the third pivot is exactly 0
    L0 = np.array([[2, 0, 0, 0], [1, 1, 0, 0], [1, 2, 0, 0], [0, 1, 3, 1]], dtype=np.complex128)
    S = L0 @ L0.conj().T
    H = np.eye(4, dtype=np.complex128)
    assert reduce_standard(H, S)[2] == 3
    # a negative pivot at column 5, and a NaN at column 2
    S = np.diag([1.0, 2.0, 3.0, 4.0, -1.0, 6.0]).astype(np.complex128)
    assert reduce_standard(np.eye(6), S)[2] == 5
    S = np.eye(3, dtype=np.complex128)
    S[1, 1] = np.nan
    assert reduce_standard(np.eye(3), S)[2] == 2


def test_reduce_real_symmetric_pair_stays_real():
    # Sec. 1.1: with inversion symmetry H and S are real symmetric; then L and C are
    # real (zero imaginary parts exactly) and equal the real-arithmetic reduction
    H, S = synth.reduce_inputs(30, seed=8, cond=1e2)
    Hr, Sr = H.real.copy(), (S.real + S.real.T) / 2 + 30 * np.eye(30)
    L, C, fail = reduce_standard(Hr.astype(np.complex128), Sr.astype(np.complex128))
    assert fail == 0
    assert np.all(L.imag == 0) and np.all(C.imag == 0)
    Lx = np.linalg.cholesky(Sr)
    Cx = np.linalg.solve(Lx, np.linalg.solve(Lx, Hr).T).T
    assert np.allclose(L.real, Lx, rtol=0, atol=1e-13)
    assert np.allclose(C.real, Cx, rtol=0, atol=1e-12)
