"""Parity of hs_reduce (generalized-eigenproblem reduction, Sec. 1.1: S = L L^H,
C = L^{-1} H L^{-H}) with the CPU FP64 oracle.

Tolerance, FP64 form: to first order the forward error of a backward-stable
Cholesky and of triangular solves is bounded by n u kappa(S) relative to the
result (u = 2^-53), so every comparison uses max(1e-13, n u kappa(S)) with kappa
the 2-norm condition number of the case's S.

Split form (plans of precision split_bf16): the Cholesky and the inverse factor
128-wide panels in FP64 (up to N_G = 128 L is bitwise equal to the FP64 form's)
and run their trailing updates, and the two products H L^{-H} and Z^H B + B^H Z,
on the BF16 slice path, whose results carry a relative error of at most the split
assembly's 1e-10 of their operands' scale; ||B||^2 = 1/lambda_min(S) and
||C|| >= ||H|| / lambda_max(S) turn that into 1e-10 kappa(S) relative to C, and
the Schur complements' errors into no more than that relative to L.

Both forms: L's strict upper triangle is exactly zero, and C exactly Hermitian
with an exactly real diagonal.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import rel_frobenius  # noqa: E402
from oracle.reduce import reduce_standard  # noqa: E402
from paper_1611_00606_gb300 import synth  # noqa: E402

U_ROUND = 2.0 ** -53


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_00606_gb300 import hs as _hs
    return _hs


def _dev(X):
    """numpy (n, n) -> column-major complex128 CUDA tensor."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X, np.complex128).T)).cuda().T


TOL_SPLIT = 1e-10


def _kappa(S):
    w = np.linalg.eigvalsh(S)  # kappa_2 of a Hermitian positive definite S
    return w[-1] / w[0] if w[0] > 0 else np.inf


def _tol(S, precision="fp64"):
    if precision == "split_bf16":
        return TOL_SPLIT * max(1.0, _kappa(S))
    return max(1e-13, S.shape[0] * U_ROUND * _kappa(S))


def _reduce(hs, H, S, precision="fp64"):
    n = H.shape[0]
    with hs.Plan(1, 1, max(n, 1), precision) as p:
        Hd, Sd = _dev(H), _dev(S)
        info = p.reduce(Hd, Sd)
    torch.cuda.synchronize()
    return Hd.cpu().numpy(), Sd.cpu().numpy(), info


def _check(C, L, H, S, precision="fp64"):
    Lr, Cr, fail = reduce_standard(H, S)
    assert fail == 0
    tol = _tol(S, precision)
    assert np.all(np.triu(L, 1) == 0)
    assert rel_frobenius(L, Lr) <= tol, (rel_frobenius(L, Lr), tol)
    assert rel_frobenius(C, Cr) <= tol, (rel_frobenius(C, Cr), tol)
    assert np.array_equal(C, C.conj().T)
    assert np.all(np.diag(C).imag == 0)
    return rel_frobenius(L, Lr), rel_frobenius(C, Cr)


@pytest.mark.parametrize("n,cond", [
    (1, 1.0),        # one element: L = sqrt(s), C = h / s
    (37, 1e3),       # inside one 64-tile
    (64, 1e3),       # exactly one tile
    (65, 1e3),       # one tile plus a 1-wide tail
    (130, 1e4),      # three tiles, ragged
    (257, 1e3),      # five tiles, 1-wide tail; several Cholesky panels
    (520, 1e6),      # nine panels, ragged, ill-conditioned
    (1000, 1e4),     # 32-wide tiles of the FP64 products (fewer than 2 x 152 64-wide)
    (1300, 1e3),     # 64-wide tiles for the two-sided products, 32-wide late in the Cholesky
])
def test_reduce_parity(hs, n, cond):
    H, S = synth.reduce_inputs(n, seed=n + 7, cond=cond)
    C, L, info = _reduce(hs, H, S)
    eL, eC = _check(C, L, H, S)
    print(f"n={n} cond={cond:g}: L {eL:.2e} C {eC:.2e} ms {info['ms_total']:.3f}")
    assert info["fail_col"] == 0


@pytest.mark.parametrize("n,cond", [
    (1, 1.0),
    (65, 1e3),
    (130, 1e4),
    (128, 1e3),      # one FP64 panel exactly
    (129, 1e3),      # a 1-wide second panel
    (257, 1e3),      # three panels, the last 1 wide; several row blocks of the stacked operand
    (520, 1e6),      # three panels, ragged, ill-conditioned
    (777, 1e2),      # four panels: trailing updates of several sizes
])
def test_reduce_split_parity(hs, n, cond):
    H, S = synth.reduce_inputs(n, seed=n + 7, cond=cond)
    C, L, info = _reduce(hs, H, S, "split_bf16")
    C64, L64, _ = _reduce(hs, H, S, "fp64")
    if n <= 128:
        assert np.array_equal(L, L64)  # one panel: the factor is all FP64
    eL, eC = _check(C, L, H, S, "split_bf16")
    print(f"split n={n} cond={cond:g}: L {eL:.2e} C {eC:.2e} (fp64 form {rel_frobenius(C64, C):.2e} "
          f"apart) ms {info['ms_total']:.3f}")


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_reduce_reads_lower_triangles_only(hs, precision):
    n = 150
    H, S = synth.reduce_inputs(n, seed=3)
    C1, L1, _ = _reduce(hs, H, S, precision)
    Hp, Sp = H.copy(), S.copy()
    iu = np.triu_indices(n, 1)
    Hp[iu] = np.nan
    Sp[iu] = 1e300
    Hp[np.diag_indices(n)] += 5j  # the diagonal enters as its real part
    C2, L2, _ = _reduce(hs, Hp, Sp, precision)
    assert np.array_equal(C1, C2) and np.array_equal(L1, L2)


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
@pytest.mark.parametrize("n,col,val", [(100, 71, -1.0), (200, 130, np.nan), (70, 1, 0.0)])
def test_reduce_not_positive_definite(hs, n, col, val, precision):
    H, _ = synth.reduce_inputs(n, seed=5)
    S = np.eye(n, dtype=np.complex128)
    S[col - 1, col - 1] = val
    assert reduce_standard(H, S)[2] == col
    Hd, Sd = _dev(H), _dev(S)
    with hs.Plan(1, 1, n, precision) as p:
        with pytest.raises(hs.HSError) as e:
            p.reduce(Hd, Sd)
    assert e.value.code == hs.HS_ENOTPD and e.value.fail_col == col
    assert np.array_equal(Hd.cpu().numpy(), H)  # H untouched


def test_reduce_of_assembled_overlap(hs):
    """The consumer path: H, S from hs_assemble (FP64), then hs_reduce."""
    w = synth.Workload("r", 4, 36, 200, (1,), seed=19)  # 2K = 288 >= N_G: S definite
    d = synth.make_inputs(w)
    A, B = hs.to_device_coef(d["A"]), hs.to_device_coef(d["B"])
    T = [hs.to_device_T(d[k]) for k in ("T_AA", "T_AB", "T_BB")]
    U = hs.to_device_U(d["U"])
    with hs.Plan(w.N_A, w.N_L, w.N_G, "fp64") as p:
        Hd, Sd, _ = p.assemble(A, B, *T, U)
        H0, S0 = Hd.cpu().numpy(), Sd.cpu().numpy()
        p.reduce(Hd, Sd)
    C, L = Hd.cpu().numpy(), Sd.cpu().numpy()
    eL, eC = _check(C, L, H0, S0)
    print(f"assembled N_G=200: L {eL:.2e} C {eC:.2e}")


def test_reduce_paper_scale(hs):
    """auag_like_4000 (N_G = 4000) from the split assembly in the benchmark's launch
    configuration, then the reduction in both forms; the whole results against the
    oracle."""
    w = synth.WORKLOADS["auag_like_4000"]
    d = synth.make_inputs(w)
    A, B = hs.to_device_coef(d["A"]), hs.to_device_coef(d["B"])
    T = [hs.to_device_T(d[k]) for k in ("T_AA", "T_AB", "T_BB")]
    U = hs.to_device_U(d["U"])
    with hs.Plan(w.N_A, w.N_L, w.N_G, "split_bf16") as p:
        H0d, S0d, _ = p.assemble(A, B, *T, U)
        H0, S0 = H0d.cpu().numpy(), S0d.cpu().numpy()
        Hd, Sd = H0d.clone(), S0d.clone()
        info = p.reduce(Hd, Sd)
    C, L = Hd.cpu().numpy(), Sd.cpu().numpy()
    eL, eC = _check(C, L, H0, S0, "split_bf16")
    with hs.Plan(1, 1, w.N_G, "fp64") as p:
        info64 = p.reduce(H0d, S0d)
    C64, L64 = H0d.cpu().numpy(), S0d.cpu().numpy()
    eL64, eC64 = _check(C64, L64, H0, S0)
    print(f"auag_like_4000: split L {eL:.2e} C {eC:.2e} ms {info['ms_total']:.1f}; "
          f"fp64 L {eL64:.2e} C {eC64:.2e} ms {info64['ms_total']:.1f}")


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_reduce_deterministic(hs, precision):
    H, S = synth.reduce_inputs(300, seed=9)
    C1, L1, _ = _reduce(hs, H, S, precision)
    C2, L2, _ = _reduce(hs, H, S, precision)
    assert np.array_equal(C1, C2) and np.array_equal(L1, L2)


def test_reduce_misuse(hs):
    H, S = synth.reduce_inputs(20, seed=2)
    Hd, Sd = _dev(H), _dev(S)
    with hs.Plan(1, 1, 10) as p:  # N_G above N_G_max
        with pytest.raises(hs.HSError) as e:
            hs.hs_reduce(p.h, Hd, Sd, 20)
        assert e.value.code == hs.HS_EINVAL
    with hs.Plan(1, 1, 20) as p:
        with pytest.raises(hs.HSError) as e:  # H and S the same buffer
            hs.hs_reduce(p.h, Hd, Hd, 20)
        assert e.value.code == hs.HS_EINVAL
        assert hs._lib.hs_reduce(p.h, Hd.data_ptr(), Sd.data_ptr(), 0, None) == hs.HS_OK
    with hs.Plan(1, 1, 20, "fp64_real") as p:  # real plans: not supported
        with pytest.raises(hs.HSError) as e:
            hs.hs_reduce(p.h, Hd, Sd, 20)
        assert e.value.code == hs.HS_EINVAL
    assert np.array_equal(Hd.cpu().numpy(), H) and np.array_equal(Sd.cpu().numpy(), S)


def test_reduce_real_fp64(hs):
    """hs_reduce_real (real symmetric pairs, Sec. 1.1) on an FP64 real plan."""
    n = 200
    H, S = synth.reduce_inputs(n, seed=21, cond=1e3)
    Hr, Sr = np.asfortranarray(H.real), np.asfortranarray(S.real)  # S.real is SPD
    Hd, Sd = hs.to_device_real(Hr), hs.to_device_real(Sr)
    with hs.Plan(1, 1, n, "fp64_real") as p:
        info = hs.hs_reduce_real(p.h, Hd, Sd)
    C, L = Hd.cpu().numpy(), Sd.cpu().numpy()
    Lr, Cr, fail = reduce_standard(Hr, Sr)
    assert fail == 0 and info["fail_col"] == 0
    tol = _tol(Sr)
    assert np.all(np.triu(L, 1) == 0)
    assert rel_frobenius(L, Lr.real) <= tol and rel_frobenius(C, Cr.real) <= tol
    assert np.array_equal(C, C.T)
    # a failing pivot leaves both matrices unchanged
    Sbad = Sr.copy()
    Sbad[40, 40] = -1.0
    Hd, Sd = hs.to_device_real(Hr), hs.to_device_real(Sbad)
    with hs.Plan(1, 1, n, "fp64_real") as p:
        with pytest.raises(hs.HSError) as e:
            hs.hs_reduce_real(p.h, Hd, Sd)
    assert e.value.code == hs.HS_ENOTPD and e.value.fail_col == reduce_standard(Hr, Sbad)[2]
    assert np.array_equal(Hd.cpu().numpy(), Hr) and np.array_equal(Sd.cpu().numpy(), Sbad)
    # complex plans take hs_reduce
    with hs.Plan(1, 1, n, "fp64") as p:
        with pytest.raises(hs.HSError) as e:
            hs.hs_reduce_real(p.h, Hd, Sd)
        assert e.value.code == hs.HS_EINVAL


@pytest.mark.parametrize("n", [200, 777])
def test_reduce_real_split(hs, n):
    """hs_reduce_real on a split real plan (the pair embedded as complex, the split
    form's kernels): L and C within the split form's bound of the oracle, L lower with a
    zero upper triangle, C exactly symmetric; a failing pivot leaves both unchanged."""
    H, S = synth.reduce_inputs(n, seed=22 + n, cond=1e3)
    Hr, Sr = np.asfortranarray(H.real), np.asfortranarray(S.real)
    Hd, Sd = hs.to_device_real(Hr), hs.to_device_real(Sr)
    with hs.Plan(1, 1, n, "split_bf16_real") as p:
        info = hs.hs_reduce_real(p.h, Hd, Sd)
    C, L = Hd.cpu().numpy(), Sd.cpu().numpy()
    Lr, Cr, fail = reduce_standard(Hr, Sr)
    assert fail == 0 and info["fail_col"] == 0
    tol = _tol(Sr, "split_bf16")
    assert np.all(np.triu(L, 1) == 0)
    assert rel_frobenius(L, Lr.real) <= tol and rel_frobenius(C, Cr.real) <= tol
    assert np.array_equal(C, C.T)
    Sbad = Sr.copy()
    Sbad[40, 40] = -1.0
    Hd, Sd = hs.to_device_real(Hr), hs.to_device_real(Sbad)
    with hs.Plan(1, 1, n, "split_bf16_real") as p:
        with pytest.raises(hs.HSError) as e:
            hs.hs_reduce_real(p.h, Hd, Sd)
    assert e.value.code == hs.HS_ENOTPD and e.value.fail_col == reduce_standard(Hr, Sbad)[2]
    assert np.array_equal(Hd.cpu().numpy(), Hr) and np.array_equal(Sd.cpu().numpy(), Sbad)
