"""Pins of the matching-coefficient oracle (``oracle/matching.py``), no GPU.

The coefficients are fixed by the matching conditions of Sec. 1.1 (value and radial
derivative of the basis function continuous on each muffin-tin sphere), so the
strongest pin is the conditions themselves: the sphere-side expansion built from A, B
must reproduce the plane wave e^{i K.r} / sqrt(Omega) and its radial derivative at
points of the sphere, evaluated directly, up to the truncation of the l sum.  The
spherical harmonics are pinned to their closed forms and orthonormality (which the
reconstruction alone would not fix: any orthonormal set obeying the addition theorem
reconstructs the plane wave), the Bessel functions to theirs.  Negative controls plant
a dropped conjugate, a flipped phase and swapped radial functions in the oracle and
check that the reconstruction catches each.
"""
import math

import numpy as np
import pytest

import oracle.matching as om
from paper_1611_00606_gb300 import synth
from scipy.special import spherical_jn


def _sphere_points(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    theta = np.arccos(np.clip(v[:, 2], -1, 1))
    phi = np.arctan2(v[:, 1], v[:, 0])
    return v, theta, phi


def test_ylm_closed_forms():
    _, th, ph = _sphere_points(50, 1)
    Y = om.ylm(2, th, ph)
    c, s = np.cos(th), np.sin(th)
    pi = math.pi
    ref = {
        (0, 0): np.full_like(th, 1 / math.sqrt(4 * pi)) + 0j,
        (1, -1): math.sqrt(3 / (8 * pi)) * s * np.exp(-1j * ph),
        (1, 0): math.sqrt(3 / (4 * pi)) * c + 0j,
        (1, 1): -math.sqrt(3 / (8 * pi)) * s * np.exp(1j * ph),
        (2, -2): math.sqrt(15 / (32 * pi)) * s ** 2 * np.exp(-2j * ph),
        (2, -1): math.sqrt(15 / (8 * pi)) * s * c * np.exp(-1j * ph),
        (2, 0): math.sqrt(5 / (16 * pi)) * (3 * c ** 2 - 1) + 0j,
        (2, 1): -math.sqrt(15 / (8 * pi)) * s * c * np.exp(1j * ph),
        (2, 2): math.sqrt(15 / (32 * pi)) * s ** 2 * np.exp(2j * ph),
    }
    for (l, m), y in ref.items():
        assert np.allclose(Y[l * l + l + m], y, rtol=0, atol=1e-14), (l, m)


def test_ylm_orthonormal_on_exact_quadrature():
    l_max = 8
    x, w = np.polynomial.legendre.leggauss(l_max + 2)      # exact in cos(theta)
    nphi = 2 * l_max + 3                                   # exact in phi
    phi = 2 * math.pi * np.arange(nphi) / nphi
    TH, PH = np.meshgrid(np.arccos(x), phi, indexing="ij")
    W = np.outer(w, np.full(nphi, 2 * math.pi / nphi))
    Y = om.ylm(l_max, TH, PH).reshape((l_max + 1) ** 2, -1)
    G = (np.conj(Y) * W.reshape(-1)) @ Y.T
    assert np.allclose(G, np.eye(G.shape[0]), atol=1e-13)


def test_ylm_matches_scipy_when_available():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    _, th, ph = _sphere_points(40, 2)
    Y = om.ylm(7, th, ph)
    for l, m in om.lm_of_L(64):
        assert np.allclose(Y[l * l + l + m], sp.sph_harm_y(l, m, th, ph), atol=1e-13)


def test_ylm_and_bessel_against_40_digit_values():
    """Y_lm up to l = 11 (the largest l the assembly takes) and j_l, j_l' at the x range
    of the workloads, against mpmath at 40 digits: pins the accuracy the parity tests
    rely on (1e-14 absolute on Y, 1e-14 relative on j_l, 5e-14 on j_l')."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    _, th, ph = _sphere_points(12, 3)
    Y = om.ylm(11, th, ph)
    for L, (l, m) in enumerate(om.lm_of_L(144)):
        for k in range(0, 12, 3):
            t = complex(mpmath.spherharm(l, m, mpmath.mpf(float(th[k])),
                                         mpmath.mpf(float(ph[k]))))
            assert abs(Y[L, k] - t) < 1e-14, (l, m, k)
    for x in (0.37, 2.9, 7.3, 12.0):
        X = mpmath.mpf(x)
        for l in range(12):
            jl = mpmath.sqrt(mpmath.pi / (2 * X)) * mpmath.besselj(l + mpmath.mpf(1) / 2, X)
            jn = mpmath.sqrt(mpmath.pi / (2 * X)) * mpmath.besselj(l + mpmath.mpf(3) / 2, X)
            assert abs(spherical_jn(l, x) - float(jl)) <= 1e-14 * abs(float(jl))
            djl = float(l / X * jl - jn)
            # scipy's j_l' = j_{l-1} - (l + 1) / x j_l cancels at small x: ~1.5e-14 at l = 11
            assert abs(spherical_jn(l, x, derivative=True) - djl) <= 5e-14 * abs(djl)


def test_spherical_bessel_closed_forms():
    x = np.linspace(0.1, 12.0, 37)
    j0 = np.sin(x) / x
    j1 = np.sin(x) / x ** 2 - np.cos(x) / x
    j2 = (3 / x ** 2 - 1) * np.sin(x) / x - 3 * np.cos(x) / x ** 2
    assert np.allclose(spherical_jn(0, x), j0, atol=1e-15)
    assert np.allclose(spherical_jn(1, x), j1, atol=1e-15)
    assert np.allclose(spherical_jn(2, x), j2, atol=1e-14)
    assert np.allclose(spherical_jn(0, x, derivative=True), -j1, atol=1e-15)
    assert np.allclose(spherical_jn(1, x, derivative=True), j0 - 2 * j1 / x, atol=1e-15)


def _reconstruct(A, B, d, l_max, a, rhat, theta, phi):
    """Sphere-side function and radial derivative at R_a rhat for every plane wave."""
    N_L = (l_max + 1) ** 2
    Y = om.ylm(l_max, theta, phi)                          # (N_L, n)
    l = np.array([ll for ll, _ in om.lm_of_L(N_L)])
    u, du, ud, dud = (d["ufun"][a][l, i][:, None] for i in range(4))
    rows = slice(a * N_L, (a + 1) * N_L)
    val = ((A[rows] * u + B[rows] * ud).T) @ Y             # (N_G, n)
    der = ((A[rows] * du + B[rows] * dud).T) @ Y
    return val, der


def _plane_wave(d, a, rhat):
    pts = d["tau"][a][None, :] + d["R"][a] * rhat          # (n, 3)
    ph = np.exp(1j * d["Kvec"] @ pts.T) / math.sqrt(d["omega"])   # (N_G, n)
    return ph, 1j * (d["Kvec"] @ rhat.T) * ph


@pytest.fixture(scope="module")
def small():
    # l_max 16 against |K| R <= ~3: the neglected l > 16 terms are below ~1e-12 of the
    # plane wave (j_17(3) ~ 3^17 / 35!!)
    l_max = 16
    d = synth.matching_inputs(2, 2, 60, seed=5)
    d = dict(d, ufun=np.pad(d["ufun"], ((0, 0), (0, l_max - 2), (0, 0)), mode="edge"))
    A, B = om.matching(d["Kvec"], d["tau"], d["R"], d["ufun"], d["omega"], l_max)
    return d, A, B, l_max


@pytest.mark.parametrize("a", [0, 1])
def test_matching_conditions_reconstruct_the_plane_wave(small, a):
    d, A, B, l_max = small
    assert (np.linalg.norm(d["Kvec"], axis=1) * d["R"][a]).max() < 3.2
    rhat, th, ph = _sphere_points(30, 10 + a)
    val, der = _reconstruct(A, B, d, l_max, a, rhat, th, ph)
    pw, dpw = _plane_wave(d, a, rhat)
    scale = 1 / math.sqrt(d["omega"])
    assert np.abs(val - pw).max() < 1e-11 * scale
    assert np.abs(der - dpw).max() < 1e-10 * scale


def test_zero_wave_vector_closed_form():
    d = synth.matching_inputs(2, 3, 30, seed=6)
    d["Kvec"] = d["Kvec"].copy()
    d["Kvec"][0] = 0.0
    A, B = om.matching(d["Kvec"], d["tau"], d["R"], d["ufun"], d["omega"], 3)
    N_L = 16
    c00 = math.sqrt(4 * math.pi) / math.sqrt(d["omega"])   # 4 pi Y_00 / sqrt(Omega)
    for a in range(2):
        u, du, ud, dud = d["ufun"][a, 0]
        W = u * dud - du * ud
        assert abs(W - 1 / d["R"][a] ** 2) < 1e-14
        assert np.isclose(A[a * N_L, 0], c00 * dud / W, rtol=1e-14)
        assert np.isclose(B[a * N_L, 0], -c00 * du / W, rtol=1e-14)
        assert np.all(A[a * N_L + 1:(a + 1) * N_L, 0] == 0)
        assert np.all(B[a * N_L + 1:(a + 1) * N_L, 0] == 0)


def test_negative_controls(small, monkeypatch):
    d, A, B, l_max = small
    rhat, th, ph = _sphere_points(20, 12)
    pw, _ = _plane_wave(d, 0, rhat)
    scale = 1 / math.sqrt(d["omega"])

    def err(A2, B2, d2=d):
        val, _ = _reconstruct(A2, B2, d2, l_max, 0, rhat, th, ph)
        return np.abs(val - pw).max() / scale

    args = (d["Kvec"], d["tau"], d["R"], d["ufun"], d["omega"], l_max)
    # phase e^{-i K.tau} instead of e^{+i K.tau}
    A2, B2 = om.matching(d["Kvec"], -d["tau"], d["R"], d["ufun"], d["omega"], l_max)
    assert err(A2, B2) > 1e-2
    # u and udot swapped in the 2 x 2 solve
    sw = d["ufun"][..., [2, 3, 0, 1]]
    A3, B3 = om.matching(d["Kvec"], d["tau"], d["R"], sw, d["omega"], l_max)
    assert err(A3, B3) > 1e-2
    # conjugate dropped from Y_lm(K^)
    real_ylm = om.ylm
    monkeypatch.setattr(om, "ylm", lambda *a: np.conj(real_ylm(*a)))
    A4, B4 = om.matching(*args)
    monkeypatch.setattr(om, "ylm", real_ylm)
    assert err(A4, B4) > 1e-2
    assert err(A, B) < 1e-11
