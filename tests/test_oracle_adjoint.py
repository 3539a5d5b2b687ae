"""Pins of the oracle's discrete adjoint: each transposed routine against central finite
differences of the corresponding forward routine (a dot-product test <J v, w> = <v, J^T w>
with J v taken by differencing the forward code), and the full gradient dJ/da of the
mode-energy drift functional J = sum_j (E_j(T) - E_j(0))^2 against central differences in a
(step 1e-6, as in the solver's adjoint workload)."""
import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W


def _fd(f, x, d, eps):
    return (f(x + eps * d) - f(x - eps * d)) / (2 * eps)


def _slice(N, seed, amp=1.5):
    return W.smooth_random(N, seed=seed, amp=amp)


def test_constraints_vjp_dot_product(orc):
    N = 65
    rng = np.random.default_rng(1)
    Phi, Pi = _slice(N, 3)
    Ab, db = rng.standard_normal(N), rng.standard_normal(N)
    dP, dQ = rng.standard_normal(N), rng.standard_normal(N)

    def fwd(z):
        A, dl, _, _ = orc.constraints(z[:N], z[N:])
        return float(np.dot(Ab, A) + np.dot(db, dl))
    z = np.concatenate([Phi, Pi])
    d = np.concatenate([dP, dQ])
    lhs = _fd(fwd, z, d, 1e-6)
    gP, gQ = orc.constraints_vjp(Phi, Pi, Ab, db)
    rhs = float(np.dot(gP, dP) + np.dot(gQ, dQ))
    assert abs(lhs - rhs) <= 1e-7 * max(1.0, abs(rhs)), (lhs, rhs)


def test_rhs_vjp_dot_product(orc):
    N = 65
    rng = np.random.default_rng(2)
    Phi, Pi = _slice(N, 4)
    A, dl, _, _ = orc.constraints(Phi, Pi)
    vP, vQ = rng.standard_normal(N), rng.standard_normal(N)
    d = [rng.standard_normal(N) for _ in range(4)]

    def fwd(z):
        p, q, a, de = z[:N], z[N:2 * N], z[2 * N:3 * N], z[3 * N:]
        dp, dq = orc.rhs(p, q, a, de, sigma=0.5)
        return float(np.dot(vP, dp) + np.dot(vQ, dq))
    z = np.concatenate([Phi, Pi, A, dl])
    dz = np.concatenate(d)
    lhs = _fd(fwd, z, dz, 1e-6)
    g = orc.rhs_vjp(Phi, Pi, A, dl, vP, vQ, sigma=0.5)
    rhs = sum(float(np.dot(gi, di)) for gi, di in zip(g, d))
    assert abs(lhs - rhs) <= 1e-7 * max(1.0, abs(rhs)), (lhs, rhs)


def test_rk4_step_vjp_dot_product(orc):
    N = 65
    rng = np.random.default_rng(3)
    Phi, Pi = _slice(N, 5)
    dt = orc.dt_for(N)
    lP, lQ = rng.standard_normal(N), rng.standard_normal(N)
    dP, dQ = rng.standard_normal(N), rng.standard_normal(N)
    dP[0] = dP[-1] = dQ[-1] = 0.0   # boundary values are held by the scheme

    def fwd(z):
        p, q = orc.rk4_step(z[:N], z[N:], dt, sigma=0.5)
        return float(np.dot(lP, p) + np.dot(lQ, q))
    z = np.concatenate([Phi, Pi])
    lhs = _fd(fwd, z, np.concatenate([dP, dQ]), 1e-6)
    gP, gQ = orc.rk4_step_vjp(Phi, Pi, lP, lQ, dt, sigma=0.5)
    rhs = float(np.dot(gP, dP) + np.dot(gQ, dQ))
    assert abs(lhs - rhs) <= 1e-7 * max(1.0, abs(rhs)), (lhs, rhs)


def test_spectrum_vjp_dot_product(orc):
    N = 129
    rng = np.random.default_rng(4)
    Phi, Pi = _slice(N, 6)
    Eb = rng.standard_normal(16)
    dP, dQ = rng.standard_normal(N), rng.standard_normal(N)

    def fwd(z):
        A, _, _, _ = orc.constraints(z[:N], z[N:])
        E, _, _ = orc.spectrum(z[:N], z[N:], A, 16)
        return float(np.dot(Eb, E))
    z = np.concatenate([Phi, Pi])
    lhs = _fd(fwd, z, np.concatenate([dP, dQ]), 1e-6)
    gP, gQ = orc.spectrum_vjp(Phi, Pi, Eb)
    rhs = float(np.dot(gP, dP) + np.dot(gQ, dQ))
    assert abs(lhs - rhs) <= 1e-7 * max(1.0, abs(rhs)), (lhs, rhs)


def test_full_gradient_against_central_differences(orc):
    """dJ/da of the drift functional over 40 RK4 steps at N = 65 (nonlinear amplitudes):
    every component with |g| > 1e-3 max|g| within 1e-5 relative of the central difference."""
    N, nsteps, K, Jm = 65, 40, 6, 8
    dt = orc.dt_for(N)
    rng = np.random.default_rng(5)
    a = rng.uniform(0.0, 0.8, K) * np.exp(-np.arange(K) / 2.0)
    J, g = orc.grad(a, N, nsteps, dt, sigma=0.5, Jm=Jm)
    assert J == pytest.approx(orc.functional(a, N, nsteps, dt, 0.5, Jm), rel=1e-13)
    for k in range(K):
        e = np.zeros(K)
        e[k] = 1.0
        fd = _fd(lambda x: orc.functional(x, N, nsteps, dt, 0.5, Jm), a, e, 1e-6)
        if abs(g[k]) > 1e-3 * np.abs(g).max():
            assert abs(fd - g[k]) <= 1e-5 * abs(g[k]), (k, fd, g[k])
