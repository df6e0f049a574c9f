"""The bounded device waits of the split kernels run out and report instead of hanging.

With the test-only stall injection (HS_TEST_STALL=1) the slice-GEMM producers arm no
pipeline stage and issue no copy, so no MMA is ever issued and the MMA thread's and
the drain warps' waits on their barriers expire (2 s).  The kernel then sets the device
error word, frees its tensor memory and returns: hs_assemble returns HS_EDEVICE after a
few seconds (three slice-GEMM launches, each giving up after its 2 s wait), the context
stays usable, and the next assembly on the same plan, without the injection, matches
the oracle.
"""
import time

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


def test_expired_wait_reports_edevice_and_plan_recovers(hs, monkeypatch):
    N_A, N_L, N_G = 3, 9, 130
    d = synth.make_inputs(synth.Workload("w", N_A, N_L, N_G, (1,), seed=77))
    A, B = hs.to_device_coef(d["A"]), hs.to_device_coef(d["B"])
    T = [hs.to_device_T(d[k]) for k in ("T_AA", "T_AB", "T_BB")]
    U = hs.to_device_U(d["U"])
    with hs.Plan(N_A, N_L, N_G, "split_bf16") as p:
        monkeypatch.setenv("HS_TEST_STALL", "1")
        t0 = time.perf_counter()
        with pytest.raises(hs.HSError) as e:
            p.assemble(A, B, *T, U)
        dt = time.perf_counter() - t0
        assert e.value.code == hs.HS_EDEVICE
        assert dt < 60.0
        monkeypatch.delenv("HS_TEST_STALL")
        H, S, info = p.assemble(A, B, *T, U)
        torch.cuda.synchronize()
    Hr, Sr = assemble(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    assert rel_frobenius(H.cpu().numpy(), Hr) <= 1e-10
    assert rel_frobenius(S.cpu().numpy(), Sr) <= 1e-10
    assert info["n_fallback"] == 1
