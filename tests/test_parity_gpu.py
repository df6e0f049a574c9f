"""Parity of the CUDA path (through the C-ABI) with the CPU FP64 oracle.

FP64 form: relative Frobenius error <= 1e-12 against the oracle (full
matrices at small sizes; sampled column panels at the paper-scale shape).
Cholesky failure flags must equal the oracle Cholesky's flags exactly.  The
outputs must be exactly Hermitian with exactly real diagonals.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import assemble, fail_flags, h_aa, rel_frobenius  # noqa: E402
from paper_1611_00606_gb300 import synth  # noqa: E402

TOL_FP64 = 1e-12


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_00606_gb300 import hs as _hs
    return _hs


def _dev(hs, d):
    return dict(A=hs.to_device_coef(d["A"]), B=hs.to_device_coef(d["B"]),
                T_AA=hs.to_device_T(d["T_AA"]), T_AB=hs.to_device_T(d["T_AB"]),
                T_BB=hs.to_device_T(d["T_BB"]), U=hs.to_device_U(d["U"]))


def _gpu_run(hs, d, N_A, N_L, precision="fp64", slices=0):
    N_G = d["A"].shape[1]
    g = _dev(hs, d)
    with hs.Plan(N_A, N_L, N_G, precision, slices) as p:
        H, S, info = p.assemble(g["A"], g["B"], g["T_AA"], g["T_AB"], g["T_BB"], g["U"])
        flags = hs.hs_fallback_flags(p.h, N_A)
    torch.cuda.synchronize()
    return H.cpu().numpy(), S.cpu().numpy(), info, flags


def _check_structure(H, S):
    assert np.array_equal(H, H.conj().T)
    assert np.array_equal(S, S.conj().T)
    assert np.all(np.diag(H).imag == 0) and np.all(np.diag(S).imag == 0)


@pytest.mark.parametrize("N_A,N_L,N_G,indef", [
    (4, 16, 256, (3,)),      # the tiny workload
    (1, 1, 1, ()),           # degenerate: one atom, one L, one G
    (3, 9, 7, (1,)),
    (2, 5, 65, ()),          # ragged: one full 64-tile plus a 1-wide tail
    (5, 16, 257, (0, 4)),    # several tiles and a ragged tail, two failing atoms
    (3, 33, 130, (0, 1, 2)), # every atom fails (no HPD segment)
])
def test_fp64_full_parity(hs, N_A, N_L, N_G, indef):
    d = synth.make_inputs(synth.Workload("p", N_A, N_L, N_G, indef, seed=N_G))
    H, S, info, flags = _gpu_run(hs, d, N_A, N_L)
    Hr, Sr = assemble(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    assert rel_frobenius(H, Hr) <= TOL_FP64
    assert rel_frobenius(S, Sr) <= TOL_FP64
    assert np.array_equal(flags, fail_flags(d["T_AA"]))
    assert info["n_fallback"] == len(indef)
    _check_structure(H, S)


def test_cholesky_path_equals_fallback_path(hs):
    """B = 0: H = H_AA.  -T^AA (negative definite) sends every atom to the
    fallback product; H_AA(-T) must equal -H_AA(T) from the Cholesky path."""
    N_A, N_L, N_G = 6, 25, 200
    d = synth.make_inputs(synth.Workload("x", N_A, N_L, N_G, (), seed=3))
    d["B"] = np.zeros_like(d["B"])
    H1, _, i1, f1 = _gpu_run(hs, d, N_A, N_L)
    d2 = dict(d, T_AA=-d["T_AA"])
    H2, _, i2, f2 = _gpu_run(hs, d2, N_A, N_L)
    assert i1["n_fallback"] == 0 and f1.sum() == 0
    assert i2["n_fallback"] == N_A and f2.sum() == N_A
    assert rel_frobenius(-H2, H1) <= TOL_FP64
    assert rel_frobenius(H1, h_aa(d["A"], d["T_AA"], N_A, N_L)) <= TOL_FP64


def test_identity_T_closed_form_on_gpu(hs):
    N_A, N_L, N_G = 3, 16, 100
    d = synth.make_inputs(synth.Workload("i", N_A, N_L, N_G, (), seed=5))
    I = np.broadcast_to(np.eye(N_L, dtype=np.complex128), (N_A, N_L, N_L)).copy()
    d.update(T_AA=I, T_AB=I, T_BB=I, U=np.ones((N_A, N_L)))
    H, S, _, _ = _gpu_run(hs, d, N_A, N_L)
    C = d["A"] + d["B"]
    assert rel_frobenius(H, C.conj().T @ C) <= TOL_FP64
    St = np.vstack([d["A"], d["B"]])
    assert rel_frobenius(S, St.conj().T @ St) <= TOL_FP64


def test_nan_propagates(hs):
    N_A, N_L, N_G = 2, 4, 10
    d = synth.make_inputs(synth.Workload("n", N_A, N_L, N_G, (), seed=6))
    d["A"] = d["A"].copy(order="F")
    d["A"][2, 3] = np.nan
    H, S, _, _ = _gpu_run(hs, d, N_A, N_L)
    assert np.isnan(H[:, 3]).any() and np.isnan(S[:, 3]).any()


def _panel_cols(N_G, width=16):
    mid = N_G // 2
    return np.concatenate([np.arange(0, width), np.arange(mid - width // 2, mid + width // 2),
                           np.arange(N_G - width, N_G)])


def test_fp64_paper_scale_panels(hs):
    """auag_like_4000 (N_A=100, N_L=121, N_G=4000, 5 indefinite atoms), the
    benchmark's launch configuration; oracle on three column panels."""
    w = synth.WORKLOADS["auag_like_4000"]
    d = synth.make_inputs(w)
    H, S, info, flags = _gpu_run(hs, d, w.N_A, w.N_L)
    cols = _panel_cols(w.N_G)
    Hr, Sr = assemble(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], w.N_A, w.N_L,
                      cols=cols)
    assert rel_frobenius(H[:, cols], Hr) <= TOL_FP64
    assert rel_frobenius(S[:, cols], Sr) <= TOL_FP64
    assert info["n_fallback"] == len(w.indefinite)
    assert list(np.nonzero(flags)[0]) == list(w.indefinite)
    _check_structure(H, S)
