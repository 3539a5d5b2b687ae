"""adscl_evolve_wide: one fixed-metric instance (the paper's Table II case, Sec. IV: A = 1,
delta = 0, SSP-RK3) spread over the whole GPU, one cooperative launch of 500-node blocks with a
grid-wide barrier per step.  Against the oracle's discrete map, against the cluster path of adscl_evolve, and the
state protocol shared with it (step counter, slice mass, statuses)."""
import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def _solver(ad, n, Phi, Pi):
    s = ad.Solver([n], scheme=ad.SCHEME_FIXED_METRIC_RK3, ko_sigma=0.5)
    s.set_initial(Phi, Pi)
    return s


# 65537: the paper's Table II grid (132 CTAs, the last with 37 nodes); 4105: a ragged last CTA
# (105 nodes); 129: a single CTA holding both ends of the grid
@pytest.mark.parametrize("n,nst", [(65537, 6), (4105, 40), (129, 40)])
def test_wide_matches_oracle(ad, orc, n, nst):
    Phi, Pi = W.smooth_random(n, seed=n % 97, amp=2.0)
    s = _solver(ad, n, Phi, Pi)
    dt, _ = s.clock()
    tr, tc, m, st = s.evolve_wide(nst * dt[0])
    assert st[0] == ad.DONE and s.clock()[1][0] == nst and tr[0] == nst * dt[0] and np.isinf(tc[0])
    gP, gQ, gA, gd = s.get_state(0)
    oP, oQ = orc.fixed_evolve(Phi, Pi, dt[0], nst, order=3, sigma=0.5)
    scale = max(1.0, np.abs(oP).max(), np.abs(oQ).max())
    assert np.abs(gP - oP).max() <= 1e-11 * scale and np.abs(gQ - oQ).max() <= 1e-11 * scale
    assert np.all(gA == 1.0) and np.all(gd == 0.0)


def test_wide_normal_mode_at_the_table2_grid(ad, orc):
    """A normal mode at N = 65537 for 60 steps: the oracle to 1e-11 and the exact solution
    Pi = cos(omega t) e_j to the scheme's truncation error."""
    n, j, nst = 65537, 2, 60
    a = np.zeros(j + 1)
    a[j] = 1.0
    Phi, Pi = orc.synthesize(n, a)
    s = _solver(ad, n, Phi, Pi)
    dt, _ = s.clock()
    s.evolve_wide(nst * dt[0])
    gP, gQ, _, _ = s.get_state(0)
    oP, oQ = orc.fixed_evolve(Phi, Pi, dt[0], nst, order=3, sigma=0.5)
    scale = max(1.0, np.abs(oQ).max())
    assert np.abs(gP - oP).max() <= 1e-11 * scale and np.abs(gQ - oQ).max() <= 1e-11 * scale
    w = 3.0 + 2.0 * j
    assert np.abs(gQ - np.cos(w * nst * dt[0]) * Pi).max() <= 1e-6 * np.abs(Pi).max()


def test_wide_and_cluster_paths_agree_and_alternate(ad):
    """The same slices (to rounding) and the same outputs as adscl_evolve on the 16-CTA cluster;
    calls of the two continue each other's step counter."""
    n = 65537
    Phi, Pi = W.smooth_random(n, seed=5, amp=2.0)
    a, b = _solver(ad, n, Phi, Pi), _solver(ad, n, Phi, Pi)
    dt, _ = a.clock()
    ra = a.evolve_wide(10 * dt[0])
    rb = b.evolve(10 * dt[0])
    aP, aQ, _, _ = a.get_state(0)
    bP, bQ, _, _ = b.get_state(0)
    scale = max(np.abs(bP).max(), np.abs(bQ).max())
    assert np.abs(aP - bP).max() <= 1e-12 * scale and np.abs(aQ - bQ).max() <= 1e-12 * scale
    assert ra[0][0] == rb[0][0] and ra[3][0] == rb[3][0] == ad.DONE
    assert abs(ra[2][0] - rb[2][0]) <= 1e-12 * abs(rb[2][0])
    # alternate: cluster path then wide, against wide then cluster
    a.evolve(16 * dt[0])
    a.evolve_wide(25 * dt[0])
    b.evolve_wide(17 * dt[0])
    b.evolve(25 * dt[0])
    assert a.clock()[1][0] == b.clock()[1][0] == 25
    aP, aQ, _, _ = a.get_state(0)
    bP, bQ, _, _ = b.get_state(0)
    assert np.abs(aP - bP).max() <= 1e-12 * scale and np.abs(aQ - bQ).max() <= 1e-12 * scale
    # a t_end already reached takes no step
    a.evolve_wide(20 * dt[0])
    assert a.clock()[1][0] == 25


def test_wide_refuses_what_it_does_not_run(ad):
    Phi, Pi = W.smooth_random(129, seed=1, amp=1.0)
    two = ad.Solver([129, 129], scheme=ad.SCHEME_FIXED_METRIC_RK3)
    two.set_initial(W.packed([Phi, Phi]), W.packed([Pi, Pi]))
    with pytest.raises(ad.AdsclError) as e:
        two.evolve_wide(0.01)
    assert e.value.status == ad.ADSCL_EUNSUPPORTED
    rk4 = ad.Solver([129])
    rk4.set_initial(Phi, Pi)
    with pytest.raises(ad.AdsclError) as e:
        rk4.evolve_wide(0.01)
    assert e.value.status == ad.ADSCL_EUNSUPPORTED
    assert rk4.clock()[1][0] == 0
