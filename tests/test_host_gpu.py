"""hs_assemble_host (host buffers; copies of A and B in column chunks overlapped with
the slicing, S copied back while H is computed) returns exactly what hs_assemble
returns on the same inputs: same kernels, same reduction order."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import assemble, rel_frobenius  # noqa: E402
from paper_1611_00606_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_00606_gb300 import hs as _hs
    return _hs


def _pin(t):
    h = torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, pin_memory=True)
    h.copy_(t)
    return h


@pytest.mark.parametrize("precision", ["split_bf16", "fp64"])
@pytest.mark.parametrize("N_A,N_L,N_G,indef", [
    (4, 16, 256, (3,)),   # N_G = padded rows: the last chunk has no zero rows
    (3, 9, 7, (1,)),      # fewer columns than chunks
    (5, 16, 300, (0,)),   # ragged chunks and zero rows past N_G
])
def test_host_call_matches_device_call(hs, precision, N_A, N_L, N_G, indef):
    d = synth.make_inputs(synth.Workload("h", N_A, N_L, N_G, indef, seed=N_G + 11))
    A, B = hs.to_device_coef(d["A"]), hs.to_device_coef(d["B"])
    T = [hs.to_device_T(d[k]) for k in ("T_AA", "T_AB", "T_BB")]
    U = hs.to_device_U(d["U"])
    with hs.Plan(N_A, N_L, N_G, precision) as p:
        Hd, Sd, _ = p.assemble(A, B, *T, U)
        torch.cuda.synchronize()
        hA, hB, hU = _pin(A.cpu()), _pin(B.cpu()), _pin(U.cpu())
        hT = [_pin(t.cpu()) for t in T]
        hH = torch.empty((N_G, N_G), dtype=torch.complex128, pin_memory=True).T
        hS = torch.empty((N_G, N_G), dtype=torch.complex128, pin_memory=True).T
        for _ in range(2):  # second call: factor served from the cache
            hs.hs_assemble_host(p.h, hA, hB, *hT, hU, N_A, N_L, N_G, hH, hS)
            assert np.array_equal(hH.numpy(), Hd.cpu().numpy())
            assert np.array_equal(hS.numpy(), Sd.cpu().numpy())
        # new T contents at new host addresses: refactored, still equal to the oracle
        hT2 = [_pin(t.cpu()) for t in T]
        hs.hs_assemble_host(p.h, hA, hB, *hT2, hU, N_A, N_L, N_G, hH, hS)
    Hr, Sr = assemble(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    tol = 1e-10 if precision == "split_bf16" else 1e-12
    assert rel_frobenius(hH.numpy(), Hr) <= tol and rel_frobenius(hS.numpy(), Sr) <= tol
