"""Edge cases of the evolution through the C ABI: a t_end in the past, an instance collapsed at
t = 0, the smallest grid, and a batch of many tiny instances (far more work items than CTAs)."""
import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def test_t_end_in_the_past_takes_no_step(ad):
    N = 257
    Phi, Pi = W.smooth_random(N, seed=1, amp=1.0)
    s = ad.Solver([N, N])
    s.set_initial(W.packed([Phi, Phi]), W.packed([Pi, Pi]))
    tr1, _, m1, st1 = s.evolve(0.05)
    state = [s.get_state(b) for b in range(2)]
    steps = s.clock()[1].copy()
    tr2, _, m2, st2 = s.evolve(0.01)          # earlier than the current slice
    assert np.array_equal(s.clock()[1], steps)
    assert np.array_equal(tr1, tr2) and np.array_equal(m1, m2)
    assert np.all(st2 == ad.DONE)
    for b in range(2):
        for x, y in zip(state[b], s.get_state(b)):
            assert np.array_equal(x, y)


def test_instance_collapsed_at_start_never_steps(ad):
    N = 513
    strong = W.gaussian_pi(N, 400.0, sigma=1.0 / 16)     # min A < theta already at t = 0
    weak = W.gaussian_pi(N, 1.0, sigma=1.0 / 16)
    s = ad.Solver([N, N], collapse_threshold=0.2)
    s.set_initial(np.zeros(2 * N), W.packed([strong, weak]))
    _, _, A, _ = s.get_state(0)
    assert A.min() < 0.2
    tr, tc, m, st = s.evolve(0.2)
    assert st[0] == ad.COLLAPSED and tc[0] == 0.0 and tr[0] == 0.0
    assert s.clock()[1][0] == 0
    assert st[1] == ad.DONE and tr[1] > 0.19


def test_smallest_grid_matches_oracle(ad, orc):
    N = 17
    Phi, Pi = W.smooth_random(N, seed=3, amp=1.0)
    s = ad.Solver([N])
    s.set_initial(Phi, Pi)
    dt, _ = s.clock()
    s.evolve(10 * dt[0])
    r = orc.evolve(Phi, Pi, dt[0], 10, sigma=0.5)
    gP, gQ, _, _ = s.get_state(0)
    assert np.abs(gP - r.Phi).max() < 1e-12 and np.abs(gQ - r.Pi).max() < 1e-12


def test_many_tiny_instances_equal_single_runs(ad):
    rng = np.random.default_rng(5)
    Ns = list(rng.choice([17, 33, 65, 129], size=1000))
    fields = [W.smooth_random(int(n), seed=i, amp=1.5) for i, n in enumerate(Ns)]
    s = ad.Solver(Ns, chunk_steps=1)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    tb = s.evolve(0.3)
    assert np.all(tb[3] == ad.DONE)
    for i in (0, 1, 499, 998, 999):
        one = ad.Solver([int(Ns[i])])
        one.set_initial(fields[i][0], fields[i][1])
        t1 = one.evolve(0.3)
        for x, y in zip(s.get_state(i), one.get_state(0)):
            assert np.array_equal(x, y)
        assert tb[2][i] == t1[2][0]


def test_long_run_matches_oracle(ad, orc):
    """A weak pulse (no collapse) to t = 100 at N = 257 (32,600 RK4 steps): mass within 1e-10
    relative and the fields within 1e-9 of the oracle, min A and delta(0) likewise."""
    N = 257
    Pi0 = W.gaussian_pi(N, 2.0, sigma=1.0 / 8)
    s = ad.Solver([N], collapse_threshold=0.05)
    s.set_initial(np.zeros(N), Pi0)
    dt, _ = s.clock()
    nsteps = int(round(100.0 / dt[0]))
    tr, tc, m, st = s.evolve(100.0)
    r = orc.evolve(np.zeros(N), Pi0, dt[0], nsteps, sigma=0.5, theta=0.05)
    assert st[0] == ad.DONE and r.status == orc.DONE
    assert abs(m[0] / r.mass - 1) < 1e-10
    gP, gQ, gA, gd = s.get_state(0)
    assert np.abs(gP - r.Phi).max() < 1e-9 and np.abs(gQ - r.Pi).max() < 1e-9
    assert np.abs(gA - r.A).max() < 1e-9 and np.abs(gd - r.delta).max() < 1e-9
