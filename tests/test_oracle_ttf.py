"""Pins of the oracle's TTF quantities (oracle.ttf: total energy E = sum_j E_j, particle number
N = sum_j E_j / omega_j, temperature T = E / N; arXiv:1706.07413 Sec. II, the normal-mode
decomposition and its conserved quantities, and the temperatures printed after
Eq. (eq:approxQP)).

What fixes them independently of the oracle's own code:
- single-mode data Pi = c e_j has all its energy in mode j, so T = omega_j = 3 + 2j exactly
  and E = c^2 (orthonormality);
- the paper's four printed temperatures, reached through synthesis, the constraint solve and
  the spectrum (tests/golden/qp_temperatures.json);
- completeness of {e_j} and {e_j'/omega_j} in L^2(tan^2 x dx): the total energy equals the mass
  M = int tan^2 x A (Phi^2 + Pi^2) dx of the same slice;
- the linear evolution (A = 1, delta = 0) conserves every mode energy exactly, so the fixed-metric
  scheme changes them only by its truncation error, which must fall with the scheme's order;
- under the full scheme the particle number is conserved only at leading order: its drift falls
  as eps^2 for small data.
A wrong weight (omega_j^2 for omega_j, a missing sqrt(A) or 1/omega_j^2), a dropped mode or an
index shift fails at least one of these."""
import json
import math
import os

import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("j", [0, 1, 4, 17])
def test_single_mode_temperature_is_its_frequency(orc, j):
    N, c = 1025, 0.3
    a = np.zeros(j + 1)
    a[j] = c
    Phi, Pi = orc.synthesize(N, a)
    E, _, _ = orc.spectrum(Phi, Pi, np.ones(N), 64)     # A = 1: the linear (fixed-metric) slice
    Et, Nt, T = orc.ttf(E)
    assert abs(Et - c * c) <= 1e-10 * c * c
    assert abs(Nt - c * c / (3 + 2 * j)) <= 1e-10 * c * c
    assert abs(T - (3 + 2 * j)) <= 1e-9 * (3 + 2 * j)


def test_two_mode_closed_form(orc):
    """Pi = a e_0 + b e_3: E = a^2 + b^2, N = a^2/3 + b^2/9."""
    N, a0, b3 = 1025, 0.2, -0.5
    Phi, Pi = orc.synthesize(N, np.array([a0, 0.0, 0.0, b3]))
    E, _, _ = orc.spectrum(Phi, Pi, np.ones(N), 64)
    Et, Nt, T = orc.ttf(E)
    assert abs(Et - (a0 ** 2 + b3 ** 2)) <= 1e-10
    assert abs(Nt - (a0 ** 2 / 3 + b3 ** 2 / 9)) <= 1e-10
    assert abs(T - (a0 ** 2 + b3 ** 2) / (a0 ** 2 / 3 + b3 ** 2 / 9)) <= 1e-9


def test_printed_temperatures_through_the_spectrum(orc):
    gold = json.load(open(os.path.join(GOLDEN, "qp_temperatures.json")))
    N = 1025
    for case in gold["cases"]:
        a = W.approx_qp_coefficients(case["kd"], case["mu"], eps=1e-5, K=32)
        Phi, Pi = orc.synthesize(N, a)
        A, _, _, _ = orc.constraints(Phi, Pi)
        E, _, _ = orc.spectrum(Phi, Pi, A, 64)
        T = orc.ttf(E)[2]
        tol = 0.5 * 10 ** (math.floor(math.log10(case["T"])) - case["digits"] + 1)
        assert abs(T - case["T"]) <= tol, (case, T)


def test_total_energy_equals_mass(orc):
    """sum_j E_j = int tan^2 x A (Phi^2 + Pi^2) dx = m(pi/2) on a nonlinear slice (A != 1)."""
    N = 1025
    for seed, amp in ((3, 0.5), (4, 2.0)):
        Phi, Pi = W.smooth_random(N, seed=seed, amp=amp)
        A, _, _, M = orc.constraints(Phi, Pi)
        assert A.min() < 0.99 or amp < 1.0
        E, _, _ = orc.spectrum(Phi, Pi, A, 64)
        Et = orc.ttf(E)[0]
        assert abs(Et / M - 1.0) <= 1e-8, (seed, Et, M)


def test_fixed_metric_conserves_mode_energies_to_truncation_error(orc):
    """A = 1, delta = 0, no dissipation: E_j(t) = E_j(0) for the exact solution.  The change over
    t = 1 of the fixed-metric SSP-RK3 scheme falls by about 2^3 per grid doubling."""
    a = np.array([0.6, -0.3, 0.2, 0.1])
    errs = []
    for N in (129, 257, 513):
        Phi, Pi = orc.synthesize(N, a)
        E0, _, _ = orc.spectrum(Phi, Pi, np.ones(N), 16)
        dt = orc.dt_for(N)
        P1, Q1 = orc.fixed_evolve(Phi, Pi, dt, int(round(1.0 / dt)), order=3, sigma=0.0)
        E1, _, _ = orc.spectrum(P1, Q1, np.ones(N), 16)
        t0, t1 = orc.ttf(E0), orc.ttf(E1)
        errs.append(max(np.abs(E1 - E0).max(), abs(t1[0] - t0[0]), abs(t1[1] - t0[1])))
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert errs[-1] < 1e-6, errs
    assert min(orders) > 2.5, (errs, orders)


@pytest.mark.slow
def test_particle_number_drift_is_second_order_in_amplitude(orc):
    """Full scheme (constraint A, delta every stage): the particle number of two-mode data
    e_0 + e_1 drifts by O(eps^2) relative, the total energy follows the mass."""
    N = 257
    dt = orc.dt_for(N)
    steps = int(round(2.0 / dt))
    drifts = []
    for eps in (0.01, 0.02):
        Phi, Pi = orc.synthesize(N, eps * np.array([1.0, 1.0]) / math.sqrt(2.0))
        A, _, _, M0 = orc.constraints(Phi, Pi)
        n0 = orc.ttf(orc.spectrum(Phi, Pi, A, 64)[0])
        worst = 0.0
        for _ in range(10):
            r = orc.evolve(Phi, Pi, dt, steps // 10, sigma=0.0, theta=-1.0)
            Phi, Pi = r.Phi, r.Pi
            q = orc.ttf(orc.spectrum(Phi, Pi, r.A, 64)[0])
            worst = max(worst, abs(q[1] / n0[1] - 1.0))
            assert abs(q[0] / r.mass - 1.0) <= 1e-8
        drifts.append(worst)
    ratio = drifts[1] / drifts[0]
    assert 3.0 < ratio < 5.0, (drifts, ratio)
