"""Grids beyond 32769 points, up to the paper's Table II grid N = 65537 (Sec. IV: the fixed-metric
runs used 64K points): each instance on a 16-CTA thread-block cluster (a non-portable cluster
size) with 8 nodes per thread, against the oracle.  Classic RK4 with the constraints every stage,
the paper's evolved-A SSP-RK3 scheme and the fixed metric (A = 1, delta = 0)."""
import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def test_max_points_is_65537(ad):
    assert ad.load().adscl_max_points() == 65537


# 32777: the smallest grid on 16 CTAs (uneven node blocks over the ranks); 65537: the largest
@pytest.mark.parametrize("n", [32777, 65537])
def test_sixteen_cta_constraints_and_step(ad, orc, n):
    Phi, Pi = W.smooth_random(n, seed=n % 101, amp=3.0)
    s = ad.Solver([n])
    assert s.shape(0) == (8, 512, 16)
    s.set_initial(Phi, Pi)
    _, _, A, dl = s.get_state(0)
    Ao, dlo, _, _ = orc.constraints(Phi, Pi)
    assert np.abs(A - Ao).max() < 1e-12 * max(1.0, np.abs(Ao).max())
    assert np.abs(dl - dlo).max() < 1e-12 * max(1.0, np.abs(dlo).max())
    dt, _ = s.clock()
    s.evolve(dt[0])
    gP, gQ, _, _ = s.get_state(0)
    oP, oQ = orc.rk4_step(Phi, Pi, dt[0], sigma=0.5)
    scale = max(np.abs(oP).max(), np.abs(oQ).max())
    assert np.abs(gP - oP).max() < 1e-13 * scale and np.abs(gQ - oQ).max() < 1e-13 * scale


def test_table1_grid_on_sixteen_ctas_matches_oracle(ad, orc):
    """N = 32769 (the paper's Table I grid) on the 16-CTA cluster the autotuner picks for a single
    instance instead of its default 8-CTA cluster: constraint solve and two RK4 steps."""
    n = 32769
    Phi, Pi = W.smooth_random(n, seed=77, amp=3.0)
    s = ad.Solver([n])
    assert s.shape(0) == (8, 512, 8)
    s.set_shape(n, 8, 512, 16)
    assert s.shape(0) == (8, 512, 16)
    s.set_initial(Phi, Pi)
    _, _, A, dl = s.get_state(0)
    Ao, dlo, _, _ = orc.constraints(Phi, Pi)
    assert np.abs(A - Ao).max() < 1e-12 * max(1.0, np.abs(Ao).max())
    assert np.abs(dl - dlo).max() < 1e-12 * max(1.0, np.abs(dlo).max())
    dt, _ = s.clock()
    s.evolve(2 * dt[0])
    gP, gQ, _, _ = s.get_state(0)
    oP, oQ = orc.rk4_step(*orc.rk4_step(Phi, Pi, dt[0], sigma=0.5), dt[0], sigma=0.5)
    scale = max(np.abs(oP).max(), np.abs(oQ).max())
    assert np.abs(gP - oP).max() < 1e-13 * scale and np.abs(gQ - oQ).max() < 1e-13 * scale


def test_sixteen_cta_pulse_evolution_matches_oracle(ad, orc):
    n = 65537
    Pi0 = W.gaussian_pi(n, 30.0, sigma=1.0 / 16)
    s = ad.Solver([n], collapse_threshold=2.0 ** -7, chunk_steps=7)
    s.set_initial(np.zeros(n), Pi0)
    dt, _ = s.clock()
    tr, tc, m, st = s.evolve(20 * dt[0])
    r = orc.evolve(np.zeros(n), Pi0, dt[0], 20, sigma=0.5, theta=2.0 ** -7)
    gP, gQ, gA, gd = s.get_state(0)
    scale = max(1.0, np.abs(r.Pi).max())
    assert np.abs(gP - r.Phi).max() <= 1e-11 * scale and np.abs(gQ - r.Pi).max() <= 1e-11 * scale
    assert np.abs(gA - r.A).max() <= 1e-11 and np.abs(gd - r.delta).max() <= 1e-11 * max(1.0, r.delta0)
    assert abs(m[0] / r.mass - 1) < 1e-11


def test_sixteen_cta_evolved_a_scheme_matches_oracle(ad, orc):
    n = 65537
    Phi, Pi = W.smooth_random(n, seed=5, amp=2.0)
    s = ad.Solver([n], scheme=ad.SCHEME_EVOLVED_A_RK3, a_reint_every=3)
    s.set_initial(Phi, Pi)
    dt, _ = s.clock()
    s.evolve(5 * dt[0])
    A0, _, _, _ = orc.constraints(Phi, Pi)
    r = orc.ea_evolve(Phi, Pi, A0, dt[0], 5, order=3, reint=3, sigma=0.5)
    gP, gQ, gA, _ = s.get_state(0)
    scale = max(1.0, np.abs(r.Pi).max())
    assert np.abs(gP - r.Phi).max() <= 1e-11 * scale and np.abs(gQ - r.Pi).max() <= 1e-11 * scale
    assert np.abs(gA - r.A).max() <= 1e-11


def test_fixed_metric_at_the_papers_table2_grid(ad, orc):
    """A normal mode on the fixed metric (the paper's Table II case) at N = 65537 for 60 SSP-RK3
    steps: the oracle's discrete map to 1e-11, the exact solution Pi = cos(omega t) e_j to the
    scheme's truncation error."""
    n, j = 65537, 2
    a = np.zeros(j + 1)
    a[j] = 1.0
    Phi, Pi = orc.synthesize(n, a)
    s = ad.Solver([n], scheme=ad.SCHEME_FIXED_METRIC_RK3, ko_sigma=0.5)
    s.set_initial(Phi, Pi)
    dt, _ = s.clock()
    nst = 60
    s.evolve(nst * dt[0])
    gP, gQ, _, _ = s.get_state(0)
    oP, oQ = orc.fixed_evolve(Phi, Pi, dt[0], nst, order=3, sigma=0.5)
    scale = max(1.0, np.abs(oQ).max())
    assert np.abs(gP - oP).max() <= 1e-11 * scale and np.abs(gQ - oQ).max() <= 1e-11 * scale
    w = 3.0 + 2.0 * j
    exact = np.cos(w * nst * dt[0]) * Pi
    assert np.abs(gQ - exact).max() <= 1e-6 * np.abs(Pi).max()


def test_sixteen_cta_instances_in_a_mixed_batch_equal_single_runs(ad):
    Ns = [65537, 129, 32777, 8193]
    fields = [W.smooth_random(n, seed=300 + i, amp=2.0) for i, n in enumerate(Ns)]
    s = ad.Solver(Ns, chunk_steps=3)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    t_end = 0.0004
    tb = s.evolve(t_end)
    for i, n in enumerate(Ns):
        one = ad.Solver([n], chunk_steps=3)
        one.set_initial(fields[i][0], fields[i][1])
        t1 = one.evolve(t_end)
        for x, y in zip(s.get_state(i), one.get_state(0)):
            assert np.array_equal(x, y)
        assert tb[2][i] == t1[2][0]

