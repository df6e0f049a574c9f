"""The largest shape, large_12000 (N_A=256, N_L=144 = (11+1)^2, N_G=12000, 5 atoms
with indefinite T^AA), in both forms against the CPU FP64 oracle on column panels
at the start, middle and end of H and S.

The inputs (A, B 7.1 GB each) and the oracle panels are made once per module and
shared by the two forms.  Bars: relative Frobenius error <= 1e-12 for the plain
FP64 form and <= 1e-10 for the split form (5 BF16 slices), the Cholesky failure
flags equal to the indefinite atoms, and the panels consistent with an exactly
Hermitian result.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import assemble, rel_frobenius  # noqa: E402
from paper_1611_00606_gb300 import synth  # noqa: E402

TOL = {"fp64": 1e-12, "split_bf16": 1e-10}


def _panel_cols(N_G, width=16):
    mid = N_G // 2
    return np.concatenate([np.arange(0, width), np.arange(mid - width // 2, mid + width // 2),
                           np.arange(N_G - width, N_G)])


@pytest.fixture(scope="module")
def large():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_00606_gb300 import hs
    w = synth.WORKLOADS["large_12000"]
    d = synth.make_inputs(w)
    cols = _panel_cols(w.N_G)
    Hr, Sr = assemble(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], w.N_A, w.N_L,
                      cols=cols)
    dev = dict(A=hs.to_device_coef(d["A"]), B=hs.to_device_coef(d["B"]),
               T=[hs.to_device_T(d[k]) for k in ("T_AA", "T_AB", "T_BB")],
               U=hs.to_device_U(d["U"]))
    del d
    yield hs, w, cols, Hr, Sr, dev
    del dev
    torch.cuda.empty_cache()


@pytest.mark.parametrize("precision", ["split_bf16", "fp64"])
def test_large_12000_panels(large, precision):
    hs, w, cols, Hr, Sr, g = large
    with hs.Plan(w.N_A, w.N_L, w.N_G, precision) as p:
        H, S, info = p.assemble(g["A"], g["B"], *g["T"], g["U"])
        flags = hs.hs_fallback_flags(p.h, w.N_A)
    torch.cuda.synchronize()
    Hc, Sc = H[:, cols].cpu().numpy(), S[:, cols].cpu().numpy()
    Hcc = H[cols][:, cols].cpu().numpy()
    del H, S
    torch.cuda.empty_cache()
    eh, es = rel_frobenius(Hc, Hr), rel_frobenius(Sc, Sr)
    print(f"large_12000 {precision}: H {eh:.3e} S {es:.3e}  {info['ms_total']:.1f} ms")
    assert eh <= TOL[precision] and es <= TOL[precision]
    assert info["n_fallback"] == len(w.indefinite)
    assert list(np.nonzero(flags)[0]) == list(w.indefinite)
    assert np.array_equal(Hcc.conj().T, Hcc)
    assert np.all(np.diag(Hcc).imag == 0)
