"""GPU parity of the 2-CTA cluster path (N = 8193: each CTA of a cluster owns half of the grid;
halos, scan carries and step-end diagnostics cross over distributed shared memory)."""
import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu
N = 8193


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def test_cluster_constraints_and_step_match_oracle(ad, orc):
    Phi, Pi = W.smooth_random(N, seed=81, amp=3.0)
    s = ad.Solver([N])
    s.set_initial(Phi, Pi)
    _, _, A, dl = s.get_state(0)
    Ao, dlo, _, Mo = orc.constraints(Phi, Pi)
    assert np.abs(A - Ao).max() < 1e-12 * max(1.0, np.abs(Ao).max())
    assert np.abs(dl - dlo).max() < 1e-12 * max(1.0, np.abs(dlo).max())
    dt, _ = s.clock()
    s.evolve(dt[0])
    gP, gQ, _, _ = s.get_state(0)
    oP, oQ = orc.rk4_step(Phi, Pi, dt[0], sigma=0.5)
    scale = max(np.abs(oP).max(), np.abs(oQ).max())
    assert np.abs(gP - oP).max() < 1e-13 * scale and np.abs(gQ - oQ).max() < 1e-13 * scale


def test_cluster_evolution_matches_oracle(ad, orc):
    Pi0 = W.gaussian_pi(N, 30.0, sigma=1.0 / 16)
    s = ad.Solver([N], collapse_threshold=2.0 ** -7)
    s.set_initial(np.zeros(N), Pi0)
    dt, _ = s.clock()
    tr, tc, m, st = s.evolve(30 * dt[0])
    r = orc.evolve(np.zeros(N), Pi0, dt[0], 30, sigma=0.5, theta=2.0 ** -7)
    gP, gQ, gA, gd = s.get_state(0)
    scale = max(1.0, np.abs(r.Pi).max())
    assert np.abs(gP - r.Phi).max() <= 1e-11 * scale and np.abs(gQ - r.Pi).max() <= 1e-11 * scale
    assert np.abs(gA - r.A).max() <= 1e-11 and np.abs(gd - r.delta).max() <= 1e-11 * max(1.0, r.delta0)
    assert abs(m[0] / r.mass - 1) < 1e-11


def test_mixed_batch_equals_single_runs_bitwise(ad):
    Ns = [8193, 4097, 8193, 129, 2049]
    fields = [W.smooth_random(n, seed=90 + i, amp=3.0) for i, n in enumerate(Ns)]
    s = ad.Solver(Ns, chunk_steps=3)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    tb = s.evolve(0.02)
    for i, n in enumerate(Ns):
        one = ad.Solver([n])
        one.set_initial(fields[i][0], fields[i][1])
        t1 = one.evolve(0.02)
        for x, y in zip(s.get_state(i), one.get_state(0)):
            assert np.array_equal(x, y)
        assert tb[2][i] == t1[2][0]


def test_cluster_chunk_invariance_and_many_instances(ad):
    """More cluster instances than SM pairs, two chunk lengths: identical bits."""
    B = 80
    Ns = [N] * B
    Pi = W.packed([W.gaussian_pi(N, 5.0 + b, sigma=0.1) for b in range(B)])
    res = []
    for chunk in (2, 64):
        s = ad.Solver(Ns, chunk_steps=chunk)
        s.set_initial(np.zeros_like(Pi), Pi)
        dt, _ = s.clock()
        out = s.evolve(6 * dt[0])
        res.append((out, [s.get_state(b) for b in (0, 41, 79)]))
    for x, y in zip(res[0][0], res[1][0]):
        assert np.array_equal(x, y)
    for a, b in zip(res[0][1], res[1][1]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_cluster_collapse_and_spectrum(ad, orc):
    """A strong pulse on the cluster path collapses at the oracle's time; the spectrum of an
    N = 8193 slice matches the oracle."""
    Pi0 = W.gaussian_pi(N, 60.0, sigma=1.0 / 16)
    s = ad.Solver([N], collapse_threshold=0.05)
    s.set_initial(np.zeros(N), Pi0)
    dt, _ = s.clock()
    tr, tc, m, st = s.evolve(3.0)
    r = orc.evolve(np.zeros(N), Pi0, dt[0], int(round(3.0 / dt[0])), sigma=0.5, theta=0.05)
    assert st[0] == r.status
    if r.status == orc.COLLAPSED:
        assert abs(tc[0] / r.t_collapse - 1) < 1e-3
    Phi, Pi = W.smooth_random(N, seed=5, amp=1.0)
    s2 = ad.Solver([N])
    s2.set_initial(Phi, Pi)
    E = s2.spectrum(64)
    A, _, _, M = orc.constraints(Phi, Pi)
    Eo, _, _ = orc.spectrum(Phi, Pi, A, 64)
    assert np.abs(E[0] - Eo).max() <= 1e-12 * M


# smallest and largest grid of each cluster size: 4105 / 8193 (2 CTAs), 8201 / 16385 (4),
# 16393 / 32769 (8); the smallest ones split their node blocks unevenly over the ranks
@pytest.mark.parametrize("n", [4105, 8201, 16385, 16393, 32769])
def test_cluster_sizes_constraints_and_step(ad, orc, n):
    Phi, Pi = W.smooth_random(n, seed=n % 97, amp=3.0)
    s = ad.Solver([n])
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


def test_eight_cta_cluster_evolution_matches_oracle(ad, orc):
    n = 32769
    Pi0 = W.gaussian_pi(n, 30.0, sigma=1.0 / 16)
    s = ad.Solver([n], collapse_threshold=2.0 ** -7, chunk_steps=7)
    s.set_initial(np.zeros(n), Pi0)
    dt, _ = s.clock()
    tr, tc, m, st = s.evolve(25 * dt[0])
    r = orc.evolve(np.zeros(n), Pi0, dt[0], 25, sigma=0.5, theta=2.0 ** -7)
    gP, gQ, gA, gd = s.get_state(0)
    scale = max(1.0, np.abs(r.Pi).max())
    assert np.abs(gP - r.Phi).max() <= 1e-11 * scale and np.abs(gQ - r.Pi).max() <= 1e-11 * scale
    assert np.abs(gA - r.A).max() <= 1e-11 and np.abs(gd - r.delta).max() <= 1e-11 * max(1.0, r.delta0)
    assert abs(m[0] / r.mass - 1) < 1e-11


def test_all_cluster_sizes_in_one_batch_equal_single_runs(ad):
    Ns = [32769, 129, 16385, 4097, 8193, 16393, 2049, 32769]
    fields = [W.smooth_random(n, seed=200 + i, amp=2.0) for i, n in enumerate(Ns)]
    s = ad.Solver(Ns, chunk_steps=4)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    t_end = 0.0015
    tb = s.evolve(t_end)
    for i, n in enumerate(Ns):
        one = ad.Solver([n], chunk_steps=4)
        one.set_initial(fields[i][0], fields[i][1])
        t1 = one.evolve(t_end)
        for x, y in zip(s.get_state(i), one.get_state(0)):
            assert np.array_equal(x, y)
        assert tb[2][i] == t1[2][0]


def test_more_clusters_than_fit_chunk_invariance(ad):
    """More 8-CTA instances than co-resident clusters, two chunk lengths: identical bits."""
    n, B = 16393, 24
    Pi = W.packed([W.gaussian_pi(n, 5.0 + b, sigma=0.1) for b in range(B)])
    res = []
    for chunk in (3, 50):
        s = ad.Solver([n] * B, chunk_steps=chunk)
        s.set_initial(np.zeros_like(Pi), Pi)
        dt, _ = s.clock()
        out = s.evolve(5 * dt[0])
        res.append((out, [s.get_state(b) for b in (0, 13, 23)]))
        s.close()
    for x, y in zip(res[0][0], res[1][0]):
        assert np.array_equal(x, y)
    for a, b in zip(res[0][1], res[1][1]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("shape", [None, (8, 512, 9)])
def test_production_batch_sampled_matches_oracle(ad, orc, shape):
    """The bench's production-resolution batch (15 pulses at N = 32769, one cluster each, the
    default chunking) after 12 RK4 steps on the default 8-CTA shape and on the 9-CTA shape the
    autotuner picks for it: sampled instances match the oracle."""
    insts = W.production()
    n = insts[0].N
    Pi0 = W.packed([W.gaussian_pi(it.N, it.eps, it.sigma) for it in insts])
    s = ad.Solver([it.N for it in insts], ko_sigma=0.5, collapse_threshold=2.0 ** -7)
    assert s.shape(0) == (8, 512, 8)
    if shape:
        s.set_shape(n, *shape)
        assert s.shape(0) == shape
    s.set_initial(np.zeros_like(Pi0), Pi0)
    dt, _ = s.clock()
    tr, tc, m, st = s.evolve(12 * dt[0])
    assert np.all(s.clock()[1] == 12)
    for b in (0, 7, len(insts) - 1):
        r = orc.evolve(np.zeros(n), W.gaussian_pi(n, insts[b].eps, insts[b].sigma), dt[0], 12,
                       sigma=0.5, theta=2.0 ** -7)
        gP, gQ, gA, gd = s.get_state(b)
        scale = max(1.0, np.abs(r.Pi).max())
        assert np.abs(gP - r.Phi).max() <= 1e-11 * scale and np.abs(gQ - r.Pi).max() <= 1e-11 * scale
        assert np.abs(gA - r.A).max() <= 1e-11 and np.abs(gd - r.delta).max() <= 1e-11 * max(1.0, r.delta0)
        assert abs(m[b] / r.mass - 1) < 1e-11
    s.close()
