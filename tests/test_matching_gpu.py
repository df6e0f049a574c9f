"""GPU parity of the matching coefficients A, B (``hs_matching``, Sec. 1.1) against the
FP64 oracle (``oracle/matching.py``), called through the C ABI.

Tolerance: both sides compute in FP64.  The kernel's Y_lm come from the l recurrence
of the normalised Legendre functions, its j_l from Miller's downward recurrence
normalised to j_0 or j_1; the oracle's from P_l differentiated in the Legendre basis,
and scipy.  Each product of the matching formula adds a few ulps, so an element may
differ by a small multiple of 1e-16 relative to itself plus the cancellation of the
recurrences (bounded by the largest element of its column times ~1e-15); the test
allows 1e-12 relative plus 1e-13 of the matrix's largest element, a margin of ~100x.
"""
import math

import numpy as np
import pytest

import oracle.matching as om
from paper_1611_00606_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL, ATOL_REL = 1e-12, 1e-13


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1611_00606_gb300 import hs as _hs
    return _hs


def _dev(d):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(d[k], dtype=np.float64)).cuda()
            for k in ("Kvec", "tau", "R", "ufun")}


def _gpu(hs, d, l_max, **kw):
    t = _dev(d)
    A, B = hs.hs_matching(t["Kvec"], t["tau"], t["R"], t["ufun"], d["omega"], l_max, **kw)
    return A.cpu().numpy(), B.cpu().numpy()


def _compare(X, X_ref, what):
    scale = np.abs(X_ref).max()
    err = np.abs(X - X_ref)
    bound = RTOL * np.abs(X_ref) + ATOL_REL * scale
    bad = err > bound
    assert not bad.any(), (what, int(bad.sum()), float((err / scale).max()))


def _check(hs, d, l_max):
    A, B = _gpu(hs, d, l_max)
    A_ref, B_ref = om.matching(d["Kvec"], d["tau"], d["R"], d["ufun"], d["omega"], l_max)
    _compare(A, A_ref, "A")
    _compare(B, B_ref, "B")
    return A, B


@pytest.mark.parametrize("N_A,l_max,N_G,seed", [
    (3, 8, 300, 1),      # several chunks of threads per column, N_L = 81
    (70, 3, 97, 2),      # two atom chunks, the second ragged (64 + 6)
    (1, 0, 5, 3),        # l_max = 0: one row per atom
    (2, 11, 150, 4),     # l_max = 11, the largest accepted (N_L = 144)
])
def test_matching_parity(hs, N_A, l_max, N_G, seed):
    d = synth.matching_inputs(N_A, l_max, N_G, seed=seed)
    _check(hs, d, l_max)


def test_matching_special_directions(hs):
    """K = 0 (Y_00 only), K along +z and -z (sin theta = 0, phi undefined: 0), K in
    the xy plane, one wave vector long enough that x = |K| R exceeds l_max + 8 (the
    Bessel recurrence runs upwards there) and one just below that switch (Miller's
    recurrence started above x)."""
    d = synth.matching_inputs(4, 6, 40, seed=7)
    K = d["Kvec"].copy()
    K[0] = 0.0
    K[1] = (0.0, 0.0, 1.3)
    K[2] = (0.0, 0.0, -0.7)
    K[3] = (0.9, -0.4, 0.0)
    K[4] = (7.0, -11.0, 5.0)     # |K| R ~ 30
    K[5] = (1e-3, 0.0, 0.0)      # small x: j_l ~ x^l / (2l + 1)!!
    K[6] = (0.0, 13.0 / d["R"][0], 0.0)  # x = 13 for atom 0 (<= l_max + 8 = 14), 9.5-18 for the others
    d = dict(d, Kvec=K)
    A, B = _check(hs, d, 6)
    N_L = 49
    assert np.all(A[1:N_L, 0] == 0) and np.all(B[1:N_L, 0] == 0)


def test_matching_leading_dimension(hs):
    """A, B written into wider buffers (ld > N_A N_L): the padding rows stay as they were."""
    import torch
    d = synth.matching_inputs(3, 4, 64, seed=8)
    N_L, K, ld = 25, 75, 96
    bufA = torch.full((64, ld), 7 + 7j, dtype=torch.complex128, device="cuda")
    bufB = torch.full((64, ld), -3 + 1j, dtype=torch.complex128, device="cuda")
    A, B = _gpu(hs, d, 4, A=bufA.T[:K], B=bufB.T[:K])
    A_ref, B_ref = om.matching(d["Kvec"], d["tau"], d["R"], d["ufun"], d["omega"], 4)
    _compare(A, A_ref, "A")
    _compare(B, B_ref, "B")
    assert torch.all(bufA.T[K:] == 7 + 7j) and torch.all(bufB.T[K:] == -3 + 1j)


def test_matching_argument_errors(hs):
    import ctypes as C
    import torch
    d = synth.matching_inputs(2, 3, 8, seed=9)
    t = _dev(d)
    A = torch.zeros((8, 32), dtype=torch.complex128, device="cuda").T
    B = torch.zeros((8, 32), dtype=torch.complex128, device="cuda").T
    lib = hs._lib
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = [t[k].data_ptr() for k in ("Kvec", "tau", "R", "ufun")]

    def call(omega=d["omega"], N_A=2, l_max=3, N_G=8, a=A, b=B, ld=32):
        return lib.hs_matching(*p, omega, N_A, l_max, N_G, a.data_ptr(), b.data_ptr(), ld, s)

    assert call() == 0
    assert call(l_max=12) == -1            # above the largest l_max
    assert call(omega=0.0) == -1
    assert call(omega=float("nan")) == -1
    assert call(ld=31) == -1               # ld below N_A N_L
    assert call(b=A) == -1                 # A and B the same buffer
    assert call(N_A=0) == -1
    assert call(N_G=0) == 0                # nothing to do
    assert lib.hs_matching(None, *p[1:], d["omega"], 2, 3, 8, A.data_ptr(), B.data_ptr(),
                           32, s) == -1


def test_matching_feeds_assembly(hs):
    """A, B from the kernel assemble (FP64 plan) to the oracle's H, S of the oracle's
    A, B: the matching step and the assembly chained on the device."""
    import torch
    from oracle import hs_oracle
    N_A, l_max, N_G = 3, 4, 90
    N_L = (l_max + 1) ** 2
    d = synth.matching_inputs(N_A, l_max, N_G, seed=11)
    t = _dev(d)
    A, B = hs.hs_matching(t["Kvec"], t["tau"], t["R"], t["ufun"], d["omega"], l_max)
    p = synth.make_inputs(synth.Workload("matching_chain", N_A, N_L, N_G, (1,), seed=11))
    T_AA, T_AB, T_BB, U = (p[k] for k in ("T_AA", "T_AB", "T_BB", "U"))
    A_ref, B_ref = om.matching(d["Kvec"], d["tau"], d["R"], d["ufun"], d["omega"], l_max)
    H_ref, S_ref = hs_oracle.assemble(A_ref, B_ref, T_AA, T_AB, T_BB, U, N_A, N_L)
    plan = hs.hs_plan(N_A, N_L, N_G, "fp64")
    try:
        H, S = hs.empty_hs(N_G), hs.empty_hs(N_G)
        hs.hs_assemble(plan, A, B, hs.to_device_T(T_AA), hs.to_device_T(T_AB),
                       hs.to_device_T(T_BB), hs.to_device_U(U), N_A, N_L, N_G, H, S)
        torch.cuda.synchronize()
    finally:
        hs.hs_destroy(plan)
    assert hs_oracle.rel_frobenius(H.cpu().numpy(), H_ref) < 1e-12
    assert hs_oracle.rel_frobenius(S.cpu().numpy(), S_ref) < 1e-12


def test_matching_full_size_sampled(hs):
    """N_A = 256, l_max = 11, N_G = 12000 (the assembly's large workload, 7.1 GB per
    output): sampled columns, first and last atom blocks included, against the oracle
    run on those columns' wave vectors alone."""
    import torch
    N_A, l_max, N_G = 256, 11, 12000
    d = synth.matching_inputs(N_A, l_max, N_G, seed=12)
    t = _dev(d)
    A, B = hs.hs_matching(t["Kvec"], t["tau"], t["R"], t["ufun"], d["omega"], l_max)
    torch.cuda.synchronize()
    cols = np.unique(np.r_[0, 1, N_G - 1, np.random.default_rng(0).integers(0, N_G, 13)])
    A_s = A[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    B_s = B[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    del A, B
    A_ref, B_ref = om.matching(d["Kvec"][cols], d["tau"], d["R"], d["ufun"], d["omega"],
                               l_max)
    _compare(A_s, A_ref, "A")
    _compare(B_s, B_ref, "B")
    assert math.isfinite(float(np.abs(A_s).max()))
