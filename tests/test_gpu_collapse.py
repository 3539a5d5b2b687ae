"""Collapse-time parity at the headline workload: the 8 earliest-collapsing pulses of the
256-instance, N = 4097 amplitude scan, evolved inside the full batch to their collapse (min A < 2^-7, the
criterion of Sec. II with the scan's threshold) on each kernel shape the bench runs, against
the CPU oracle run to the same slices on host threads.

Bars (the solver's stated tolerances): collapse time within 0.1 %; the same final slice; mass
within 1e-10 relative on the last slice before the earliest collapse and on each collapse slice;
Phi, Pi, A, delta within 1e-9 max-abs on a slice just before the earliest collapse.

Oracle cost: about 6,000-6,600 RK4 steps at N = 4097 per pulse, ~18 s each on one host core;
the 8 pulses run on up to 8 host threads (ctypes releases the GIL)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu

THETA = 2.0 ** -7
SHAPES = [(8, 256, 2), (8, 128, 4), (8, 512, 1)]


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def _batch(ad, insts, shape=None):
    N = insts[0].N
    s = ad.Solver([N] * len(insts), ko_sigma=0.5, collapse_threshold=THETA)
    Pi = W.packed([W.gaussian_pi(N, it.eps, it.sigma) for it in insts])
    s.set_initial(np.zeros_like(Pi), Pi)
    if shape is not None:
        s.set_shape(N, *shape)
    return s


@pytest.fixture(scope="module")
def reference(ad, orc):
    """A run of the batch on the default shape picks the 8 pulses that collapse first and the
    comparison slice n_pre (95 % of the earliest collapse, before any instance of the batch has
    collapsed); the oracle then runs those pulses to n_pre and on to their collapse."""
    insts = W.amp_scan()
    N = insts[0].N
    s = _batch(ad, insts)
    dt = s.clock()[0][0]
    _, tc, _, st = s.evolve(2.0)
    strongest = [int(b) for b in np.argsort(tc)[:8]]
    assert all(st[b] == ad.COLLAPSED for b in strongest)
    n_pre = int(0.95 * tc.min() / dt)
    s.close()

    def run(b):
        Pi0 = W.gaussian_pi(N, insts[b].eps, insts[b].sigma)
        r1 = orc.evolve(np.zeros(N), Pi0, dt, n_pre, sigma=0.5, theta=THETA)
        assert r1.status == orc.RUNNING or r1.status == orc.DONE
        r2 = orc.evolve(r1.Phi, r1.Pi, dt, int(2.0 / dt) - n_pre, sigma=0.5, theta=THETA, n0=n_pre,
                        minA_in=r1.minA)
        return b, r1, r2

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        res = {b: (r1, r2) for b, r1, r2 in ex.map(run, strongest)}
    return insts, strongest, dt, n_pre, res


@pytest.mark.parametrize("shape", SHAPES)
def test_strongest_pulses_collapse_like_the_oracle(ad, orc, reference, shape):
    insts, strongest, dt, n_pre, res = reference
    s = _batch(ad, insts, shape)
    assert s.shape(strongest[0]) == shape
    tr, tc, m, st = s.evolve(n_pre * dt)
    assert np.all(st == ad.DONE) and np.all(tr == n_pre * dt)
    worst = 0.0
    for b in strongest:
        r1, _ = res[b]
        gPhi, gPi, gA, gd = s.get_state(b)
        for g, o in ((gPhi, r1.Phi), (gPi, r1.Pi), (gA, r1.A), (gd, r1.delta)):
            worst = max(worst, np.abs(g - o).max())
        assert abs(m[b] / r1.mass - 1.0) <= 1e-10, (b, m[b], r1.mass)
    assert worst <= 1e-9, worst
    tr, tc, m, st = s.evolve(2.0)
    for b in strongest:
        _, r2 = res[b]
        assert r2.status == orc.COLLAPSED and st[b] == ad.COLLAPSED
        assert abs(tc[b] / r2.t_collapse - 1.0) <= 1e-3, (b, tc[b], r2.t_collapse)
        assert tr[b] == r2.t_reached                    # the same collapse slice
        assert abs(m[b] / r2.mass - 1.0) <= 1e-10, (b, m[b], r2.mass)
    s.close()
