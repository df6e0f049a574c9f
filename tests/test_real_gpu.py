"""Real-symmetric variant (Sec. 1.1: H and S real symmetric for systems with inversion
symmetry): parity of hs_assemble_real with the CPU FP64 oracle.

The split form slices every operand as a real array (one K position per row); the
FP64 form runs the complex kernels on embedded inputs.  Tolerances as for the complex
forms: 1e-10 relative Frobenius for the split form at 5 slices, 1e-12 for FP64.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import assemble, fail_flags, rel_frobenius  # noqa: E402
from paper_1611_00606_gb300 import synth  # noqa: E402

TOL_SPLIT = 1e-10
TOL_FP64 = 1e-12


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_00606_gb300 import hs as _hs
    return _hs


def _dev(hs, d):
    A, B = hs.to_device_real(d["A"]), hs.to_device_real(d["B"])
    T = [hs.to_device_T_real(d[k]) for k in ("T_AA", "T_AB", "T_BB")]
    return A, B, T, hs.to_device_U(d["U"])


def _run(hs, d, N_A, N_L, precision="split_bf16_real", slices=0):
    N_G = d["A"].shape[1]
    A, B, T, U = _dev(hs, d)
    with hs.Plan(N_A, N_L, N_G, precision, slices) as p:
        H, S, info = p.assemble_real(A, B, *T, U)
        flags = hs.hs_fallback_flags(p.h, N_A)
    torch.cuda.synchronize()
    return H.cpu().numpy(), S.cpu().numpy(), info, flags


def _oracle(d, N_A, N_L, cols=None):
    Hr, Sr = assemble(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L,
                      cols=cols)
    assert np.max(np.abs(Hr.imag)) == 0.0 and np.max(np.abs(Sr.imag)) == 0.0
    return Hr.real, Sr.real


@pytest.mark.parametrize("N_A,N_L,N_G,indef", [
    (4, 16, 256, (3,)),        # tiny workload shape
    (1, 1, 1, ()),             # one atom, one L, one G
    (3, 9, 7, (1,)),           # 27 real K: ragged 16-wide blocks, atoms straddling them
    (2, 5, 129, ()),           # one 128-column tile plus a 1-wide tail
    (5, 16, 300, (0, 4)),      # several row blocks, a half-empty last column pair
    (3, 33, 130, (0, 1, 2)),   # every atom fails: no Y segment
    (2, 121, 520, (1,)),       # N_L = 121: per-atom K ranges at odd offsets
])
def test_real_split_parity(hs, N_A, N_L, N_G, indef):
    d = synth.make_inputs_real(synth.Workload("r", N_A, N_L, N_G, indef, seed=N_G + 3))
    H, S, info, flags = _run(hs, d, N_A, N_L)
    Hr, Sr = _oracle(d, N_A, N_L)
    assert rel_frobenius(H, Hr) <= TOL_SPLIT and rel_frobenius(S, Sr) <= TOL_SPLIT
    assert np.array_equal(H, H.T) and np.array_equal(S, S.T)
    assert np.array_equal(flags, fail_flags(d["T_AA"]))
    assert info["slices"] == 5 and info["n_fallback"] == len(indef)


@pytest.mark.parametrize("N_A,N_L,N_G,indef", [(4, 16, 256, (3,)), (3, 9, 70, (0, 2))])
def test_real_fp64_parity(hs, N_A, N_L, N_G, indef):
    d = synth.make_inputs_real(synth.Workload("r", N_A, N_L, N_G, indef, seed=5))
    H, S, info, _ = _run(hs, d, N_A, N_L, precision="fp64_real")
    Hr, Sr = _oracle(d, N_A, N_L)
    assert rel_frobenius(H, Hr) <= TOL_FP64 and rel_frobenius(S, Sr) <= TOL_FP64
    assert np.array_equal(H, H.T) and np.array_equal(S, S.T)


def test_real_error_decreases_with_slices(hs):
    N_A, N_L, N_G = 4, 16, 256
    d = synth.make_inputs_real(synth.Workload("e", N_A, N_L, N_G, (3,), seed=13))
    Hr, Sr = _oracle(d, N_A, N_L)
    errs = []
    for s in range(2, 6):
        H, S, info, _ = _run(hs, d, N_A, N_L, slices=s)
        errs.append(max(rel_frobenius(H, Hr), rel_frobenius(S, Sr)))
    for a, b in zip(errs, errs[1:]):
        assert b < a / 16
    assert errs[-1] <= TOL_SPLIT


def test_real_split_deterministic_and_matches_fp64_form(hs):
    N_A, N_L, N_G = 6, 25, 400
    d = synth.make_inputs_real(synth.Workload("d", N_A, N_L, N_G, (2,), seed=14))
    H1, S1, _, _ = _run(hs, d, N_A, N_L)
    H2, S2, _, _ = _run(hs, d, N_A, N_L)
    assert np.array_equal(H1, H2) and np.array_equal(S1, S2)
    Hf, Sf, _, _ = _run(hs, d, N_A, N_L, precision="fp64_real")
    assert rel_frobenius(H1, Hf) <= TOL_SPLIT and rel_frobenius(S1, Sf) <= TOL_SPLIT


def test_real_plan_rejects_complex_calls(hs):
    N_A, N_L, N_G = 2, 4, 10
    d = synth.make_inputs(synth.Workload("c", N_A, N_L, N_G, (), seed=1))
    A, B = hs.to_device_coef(d["A"]), hs.to_device_coef(d["B"])
    T = [hs.to_device_T(d[k]) for k in ("T_AA", "T_AB", "T_BB")]
    U = hs.to_device_U(d["U"])
    with hs.Plan(N_A, N_L, N_G, "split_bf16_real") as p:
        with pytest.raises(hs.HSError) as e:
            p.assemble(A, B, *T, U)
        assert e.value.code == hs.HS_EINVAL
    dr = synth.make_inputs_real(synth.Workload("c", N_A, N_L, N_G, (), seed=1))
    Ar, Br, Tr, Ur = _dev(hs, dr)
    with hs.Plan(N_A, N_L, N_G, "split_bf16") as p:
        with pytest.raises(hs.HSError) as e:
            p.assemble_real(Ar, Br, *Tr, Ur)
        assert e.value.code == hs.HS_EINVAL


def _panel_cols(N_G, width=16):
    mid = N_G // 2
    return np.concatenate([np.arange(0, width), np.arange(mid - width // 2, mid + width // 2),
                           np.arange(N_G - width, N_G)])


def test_real_split_paper_scale_panels(hs):
    """auag_like_4000 shape, real inputs; oracle column panels."""
    w = synth.WORKLOADS["auag_like_4000"]
    d = synth.make_inputs_real(w)
    H, S, info, flags = _run(hs, d, w.N_A, w.N_L)
    cols = _panel_cols(w.N_G)
    Hr, Sr = _oracle(d, w.N_A, w.N_L, cols=cols)
    eh, es = rel_frobenius(H[:, cols], Hr), rel_frobenius(S[:, cols], Sr)
    print(f"auag_like_4000 real split s=5: H {eh:.3e} S {es:.3e}")
    assert eh <= TOL_SPLIT and es <= TOL_SPLIT
    assert list(np.nonzero(flags)[0]) == list(w.indefinite)
