"""Pins of the oracle's AdS4 eigenbasis, mode-energy spectrum and initial-data synthesis.

The eigenfunctions are checked against the Gauss hypergeometric closed form evaluated at
high precision (mpmath), Gauss-Legendre orthonormality, the eigen-equation and e_0 in closed
form; the spectrum against Parseval identities; the synthesis + projection chain against the
temperatures printed in arXiv:1706.07413 Sec. II (tests/golden/qp_temperatures.json)."""
import json
import math
import os

import mpmath
import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hyp_e(j, x):
    """e_j(x) = d_j cos^3 x (3/2)_j / j! 2F1(-j, j+3; 3/2; sin^2 x) (working precision set by
    the caller)."""
    x = mpmath.mpf(x)
    dj = 2 * mpmath.sqrt(mpmath.factorial(j) * mpmath.factorial(j + 2)) / mpmath.gamma(j + mpmath.mpf(3) / 2)
    pref = mpmath.rf(mpmath.mpf(3) / 2, j) / mpmath.factorial(j)
    return dj * mpmath.cos(x) ** 3 * pref * mpmath.hyp2f1(-j, j + 3, mpmath.mpf(3) / 2, mpmath.sin(x) ** 2)


@pytest.mark.parametrize("j", [0, 1, 2, 7, 31, 63])
def test_eigenfunctions_match_hypergeometric_closed_form(orc, j):
    xs = np.array([0.0, 0.013, 0.3, 0.777, 1.2, 1.5, 1.5707])
    e, de = orc.eigen_at(j + 1, xs)
    mpmath.mp.dps = 40
    for k, x in enumerate(xs):
        ref = float(_hyp_e(j, float(x)))
        dref = float(mpmath.diff(lambda t: _hyp_e(j, t), mpmath.mpf(float(x))))
        scale = 1.0 + math.sqrt(j + 1.0)
        assert abs(e[j, k] - ref) < 1e-12 * scale * (1 + abs(ref)), (j, x, e[j, k], ref)
        assert abs(de[j, k] - dref) < 1e-11 * scale * (1 + abs(dref)) * (2 * j + 3), (j, x, de[j, k], dref)


def test_e0_closed_form(orc):
    x = np.linspace(0, math.pi / 2, 101)
    e, _ = orc.eigen_at(1, x)
    assert np.allclose(e[0], 4 * math.sqrt(2) / math.sqrt(math.pi) * np.cos(x) ** 3, rtol=1e-14, atol=1e-15)


def test_orthonormality_gauss_legendre(orc):
    """int_0^{pi/2} e_i e_j tan^2 x dx = delta_ij, by 400-point Gauss-Legendre quadrature."""
    J = 64
    t, w = np.polynomial.legendre.leggauss(400)
    x = 0.25 * math.pi * (t + 1)
    w = 0.25 * math.pi * w
    e, de = orc.eigen_at(J, x)
    wt = w * np.tan(x) ** 2
    G = (e * wt) @ e.T
    assert np.abs(G - np.eye(J)).max() < 1e-12
    # the derivatives are orthogonal too, with norms omega_j^2 (integration by parts)
    Gd = (de * wt) @ de.T
    om = orc.omega(np.arange(J))
    assert np.abs(Gd / np.outer(om, om) - np.eye(J)).max() < 1e-11


@pytest.mark.parametrize("j", [0, 5, 40])
def test_eigen_equation(orc, j):
    """-tan^{-2} x (tan^2 x e_j')' = omega_j^2 e_j, i.e. e'' + 2 e'/(sin x cos x) + omega^2 e = 0,
    with e'' from a central difference of the oracle's e'."""
    x = np.linspace(0.05, 1.52, 40)
    hh = 1e-5
    e, de = orc.eigen_at(j + 1, x)
    _, dep = orc.eigen_at(j + 1, x + hh)
    _, dem = orc.eigen_at(j + 1, x - hh)
    d2 = (dep[j] - dem[j]) / (2 * hh)
    w = orc.omega(j)
    res = d2 + 2 * de[j] / (np.sin(x) * np.cos(x)) + w * w * e[j]
    assert np.abs(res).max() < 1e-6 * w * w * (1 + np.abs(e[j]).max())


def test_spectrum_parseval_single_modes(orc):
    """Pi = eps e_k gives E_j = eps^2 delta_jk; Phi = eps e_k'/omega_k gives the same (A = 1 to
    O(eps^2)); the sum of E_j over a complete set equals the mass M."""
    N, J, eps = 1025, 16, 1e-5
    e, de = orc.eigen(N, J)
    for k in (0, 3, 9):
        Pi = eps * e[k].copy(); Pi[-1] = 0.0
        Phi = np.zeros(N)
        A, _, _, M = orc.constraints(Phi, Pi)
        E, _, _ = orc.spectrum(Phi, Pi, A, J)
        ref = np.zeros(J); ref[k] = eps * eps
        assert np.abs(E - ref).max() < 1e-9 * eps * eps
        assert abs(E.sum() / M - 1) < 1e-7
        Phi = eps * de[k] / orc.omega(k); Phi[0] = Phi[-1] = 0.0
        A, _, _, M = orc.constraints(Phi, np.zeros(N))
        E, _, _ = orc.spectrum(Phi, np.zeros(N), A, J)
        assert np.abs(E - ref).max() < 1e-8 * eps * eps


def test_synthesis_then_projection_recovers_coefficients(orc):
    N, eps = 2049, 1e-4
    a = eps * np.exp(-np.arange(12) / 3.0) * np.cos(np.arange(12))
    Phi, Pi = orc.synthesize(N, a)
    A, _, _, _ = orc.constraints(Phi, Pi)
    E, pj, _ = orc.spectrum(Phi, Pi, A, 16)
    assert np.allclose(pj[:12], a, rtol=0, atol=1e-8 * eps)
    assert np.abs(pj[12:]).max() < 1e-8 * eps


def test_paper_temperatures(orc):
    """Synthesize the approximate QP data (Eq. (eq:approxQP)) with the oracle's eigenbasis,
    project it back with the oracle's spectrum and form T = sum E_j / sum (E_j / omega_j):
    the paper's printed temperatures must come out (Sec. II)."""
    gold = json.load(open(os.path.join(GOLDEN, "qp_temperatures.json")))
    N = 2049
    for case in gold["cases"]:
        a = W.approx_qp_coefficients(case["kd"], case["mu"], eps=1e-4, K=32)
        Phi, Pi = orc.synthesize(N, a)
        A, _, _, _ = orc.constraints(Phi, Pi)
        E, _, _ = orc.spectrum(Phi, Pi, A, 40)
        T = orc.temperature_from_energies(E)
        tol = 0.5 * 10 ** (math.floor(math.log10(case["T"])) - case["digits"] + 1)
        assert abs(T - case["T"]) <= tol, (case, T)
