"""Pins of the oracle's evolved-A scheme (the paper's production variant, Sec. II: A evolved by
Eq. (eq:adot), re-integrated from Eq. (eq:aprime) only periodically, delta integrated every
stage, third-order Runge-Kutta) against facts that do not come from the oracle itself:
convergence orders (the paper reports third order), the momentum constraint, exact special
cases, and the mass integral's quadrature order."""
import math

import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

T = 0.5


def _run(orc, N, order, reint=0, amp=2.0):
    Phi, Pi = W.smooth_random(N, 7, amp=amp)
    A, _, _, M0 = orc.constraints(Phi, Pi)
    n = 160 * (N - 1) // 256          # dt = T / n halves exactly with h
    r = orc.ea_evolve(Phi, Pi, A, T / n, n, order=order, reint=reint)
    Ac = orc.constraints(r.Phi, r.Pi)[0]
    return r, Ac, M0


@pytest.fixture(scope="module")
def runs(orc):
    return {order: {N: _run(orc, N, order) for N in (257, 513, 1025)} for order in (2, 3)}


def _q(u1, u2, u3):
    return math.log2(np.abs(u1 - u2[::2]).max() / np.abs(u2[::2] - u3[::4]).max())


@pytest.mark.parametrize("order,lo,hi", [(3, 2.7, 3.7), (2, 1.8, 2.2)])
def test_self_convergence_order(runs, order, lo, hi):
    r = runs[order]
    assert lo < _q(r[257][0].Pi, r[513][0].Pi, r[1025][0].Pi) < hi
    assert lo < _q(r[257][0].Phi, r[513][0].Phi, r[1025][0].Phi) < hi + 0.3
    assert lo < _q(r[257][0].A, r[513][0].A, r[1025][0].A) < hi


@pytest.mark.parametrize("order", [2, 3])
def test_evolved_A_converges_to_the_hamiltonian_constraint(runs, order):
    """Eq. (eq:adot) is consistent with Eq. (eq:aprime): the evolved A departs from the
    constraint solution only by the truncation error, which falls at the scheme's order."""
    r = runs[order]
    d = [np.abs(r[N][0].A - r[N][1]).max() for N in (257, 513, 1025)]
    m = [abs(r[N][0].mass - r[N][2]) for N in (257, 513, 1025)]
    for k in range(2):
        assert d[k] / d[k + 1] > 2.0 ** (order - 0.4)
        assert m[k] / m[k + 1] > 2.0 ** (order - 0.4)


def test_adot_matches_time_derivative_of_constraint_A(orc):
    """A-dot of Eq. (eq:adot) against a centred time difference of the constraint A along the
    (independent) RK4 evolution: agreement to O(dt^2) -- a wrong factor or sign fails."""
    N = 513
    Phi, Pi = W.smooth_random(N, 11, amp=2.0)
    dt = 1e-4
    P1, Q1 = orc.rk4_step(Phi, Pi, dt, sigma=0.0)
    P0, Q0 = orc.rk4_step(Phi, Pi, -dt, sigma=0.0)
    A1 = orc.constraints(P1, Q1)[0]
    A0 = orc.constraints(P0, Q0)[0]
    A, dl, _, _ = orc.constraints(Phi, Pi)
    dA = orc.adot(Phi, Pi, A, dl)
    fd = (A1 - A0) / (2 * dt)
    assert np.abs(dA - fd).max() < 1e-4 * np.abs(dA).max()
    assert dA[0] == 0.0 and dA[-1] == 0.0


def test_simpson_mass_converges_to_the_mass_function(orc):
    """The composite-Simpson mass and m(pi/2) from the RK4-in-x mass function are two
    4th-order quadratures of the same integral (Sec. II)."""
    d = []
    for N in (129, 257, 513):
        Phi, Pi = W.smooth_random(N, 3, amp=2.0)
        A, _, _, M = orc.constraints(Phi, Pi)
        d.append(abs(orc.mass_simpson(Phi, Pi, A) - M))
    assert d[0] / d[1] > 12 and d[1] / d[2] > 12


def test_reintegration_every_step_gives_the_constraint_A(orc):
    N = 257
    Phi, Pi = W.smooth_random(N, 5, amp=2.0)
    A = orc.constraints(Phi, Pi)[0]
    r = orc.ea_evolve(Phi, Pi, A + 0.01, orc.dt_for(N), 7, order=3, reint=1)
    assert np.array_equal(r.A, orc.constraints(r.Phi, r.Pi)[0])


def test_static_ads_is_exact(orc):
    N = 129
    z = np.zeros(N)
    r = orc.ea_evolve(z, z, np.ones(N), orc.dt_for(N), 20, order=3, reint=0)
    assert np.array_equal(r.Phi, z) and np.array_equal(r.Pi, z) and np.array_equal(r.A, np.ones(N))
    assert r.mass == 0.0 and r.status == orc.DONE


def test_evolved_scheme_collapses_like_the_constraint_scheme(orc):
    """A strong pulse collapses at nearly the same time under both schemes (both converge to
    the same continuum solution)."""
    N = 513
    Pi0 = W.gaussian_pi(N, 20.0, sigma=1.0 / 8)
    z = np.zeros(N)
    dt = orc.dt_for(N)
    A = orc.constraints(z, Pi0)[0]
    r3 = orc.ea_evolve(z, Pi0, A, dt, 4000, order=3, reint=16, theta=0.05)
    r4 = orc.evolve(z, Pi0, dt, 4000, theta=0.05)
    assert r3.status == orc.COLLAPSED and r4.status == orc.COLLAPSED
    assert abs(r3.t_collapse / r4.t_collapse - 1) < 1.5e-3


@pytest.mark.parametrize("j", [0, 3])
def test_fixed_metric_normal_mode_is_exact(orc, j):
    """Fixed metric (A = 1, delta = 0; the paper's Table II case): Eqs. (eq:phi), (eq:pi) are
    linear and Pi = cos(w t) e_j, Phi = sin(w t) e_j' / w, w = 3 + 2j, solves them exactly.  The
    SSP-RK3 solution converges to it at third order (time error dominant)."""
    errs = []
    T = 1.0
    for N in (129, 257, 513):
        e, de = orc.eigen(N, j + 1)
        w = 3.0 + 2.0 * j
        n = 160 * (N - 1) // 128
        P, Q = orc.fixed_evolve(np.zeros(N), e[j], T / n, n, order=3, sigma=0.5)
        errs.append(max(np.abs(P - np.sin(w * T) * de[j] / w).max(),
                        np.abs(Q - np.cos(w * T) * e[j]).max()))
    for k in range(2):
        assert 2.8 < math.log2(errs[k] / errs[k + 1]) < 3.6
    assert errs[-1] < (1e-7 if j == 0 else 3e-5)
