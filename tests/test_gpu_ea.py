"""GPU parity of the evolved-A schemes (the paper's production variant, Sec. II: A evolved with
Eq. (eq:adot), periodically re-integrated from Eq. (eq:aprime), SSP Runge-Kutta of order 3 or
2) against the oracle's evolved-A scheme, through the C ABI."""
import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def _close(gpu, ref, rel):
    scale = max(1.0, np.abs(ref).max())
    return np.abs(gpu - ref).max() <= rel * scale


@pytest.mark.parametrize("N,scheme,reint,steps", [(1025, 1, 0, 40), (4097, 1, 7, 30),
                                                  (513, 2, 5, 40), (129, 1, 1, 25)])
def test_evolution_matches_oracle(ad, orc, N, scheme, reint, steps):
    order = 3 if scheme == 1 else 2
    Phi, Pi = W.smooth_random(N, seed=N + reint, amp=2.5)
    s = ad.Solver([N], scheme=scheme, a_reint_every=reint)
    s.set_initial(Phi, Pi)
    _, _, A0, _ = s.get_state(0)
    Ac = orc.constraints(Phi, Pi)[0]
    assert _close(A0, Ac, 1e-12)
    dt, _ = s.clock()
    tr, tc, m, st = s.evolve(steps * dt[0])
    r = orc.ea_evolve(Phi, Pi, Ac, dt[0], steps, order=order, reint=reint, sigma=0.5)
    gP, gQ, gA, gd = s.get_state(0)
    assert _close(gP, r.Phi, 1e-11) and _close(gQ, r.Pi, 1e-11)
    assert _close(gA, r.A, 1e-11) and _close(gd, r.delta, 1e-11)
    assert abs(m[0] - r.mass) <= 1e-11 * max(1.0, r.mass)
    assert st[0] == ad.DONE and tr[0] == pytest.approx(steps * dt[0], rel=0, abs=1e-12)


def test_collapse_time_matches_oracle(ad, orc):
    N = 513
    Pi0 = W.gaussian_pi(N, 20.0, sigma=1.0 / 8)
    z = np.zeros(N)
    s = ad.Solver([N], scheme=1, a_reint_every=16, collapse_threshold=0.05)
    s.set_initial(z, Pi0)
    dt, _ = s.clock()
    tr, tc, m, st = s.evolve(10.0)
    r = orc.ea_evolve(z, Pi0, orc.constraints(z, Pi0)[0], dt[0], 4000, order=3, reint=16,
                      theta=0.05)
    assert st[0] == ad.COLLAPSED and r.status == orc.COLLAPSED
    assert abs(tc[0] / r.t_collapse - 1) < 1e-9


def test_batch_chunks_and_restarts_are_bit_identical(ad):
    Ns = [4097, 1025, 129, 2049, 4097, 513]
    fields = [W.smooth_random(n, seed=300 + i, amp=2.0) for i, n in enumerate(Ns)]
    Phi, Pi = W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields])
    runs = []
    for chunk, t_ends in ((3, (0.02,)), (64, (0.005, 0.013, 0.02))):
        s = ad.Solver(Ns, scheme=1, a_reint_every=5, chunk_steps=chunk)
        s.set_initial(Phi, Pi)
        for t in t_ends:
            out = s.evolve(t)
        runs.append((out, [s.get_state(b) for b in range(len(Ns))]))
        s.close()
    for x, y in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(x, y)
    for a, b in zip(runs[0][1], runs[1][1]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    for i, n in enumerate(Ns):   # batched = single instance
        one = ad.Solver([n], scheme=1, a_reint_every=5)
        one.set_initial(fields[i][0], fields[i][1])
        one.evolve(0.02)
        for x, y in zip(one.get_state(0), runs[0][1][i]):
            assert np.array_equal(x, y)


def test_unsupported_requests_fail_cleanly(ad):
    s = ad.Solver([257] * 2, scheme=1)
    with pytest.raises(ad.AdsclError) as e:
        s.set_shape(257, 4, 256, 1)          # not among the evolved-A kernel's shapes
    assert e.value.status == ad.ADSCL_EINVAL
    s.set_initial_modes(np.full((2, 4), 0.01))
    with pytest.raises(ad.AdsclError) as e:
        s.grad(np.full((2, 4), 0.01), 0.1)
    assert e.value.status == ad.ADSCL_EUNSUPPORTED


@pytest.mark.parametrize("N,j", [(1025, 0), (2049, 5)])
def test_fixed_metric_matches_oracle_and_exact_mode(ad, orc, N, j):
    """Scheme 3 (A = 1, delta = 0; the paper's Table II case): a normal mode e_j, synthesised on
    the device, evolves as Pi = cos(w t) e_j, Phi = sin(w t) e_j' / w."""
    a = np.zeros((1, j + 1))
    a[0, j] = 1.0
    s = ad.Solver([N], scheme=ad.SCHEME_FIXED_METRIC_RK3)
    s.set_initial_modes(a)
    dt, _ = s.clock()
    n = 200
    tr, tc, m, st = s.evolve(n * dt[0])
    gP, gQ, gA, gd = s.get_state(0)
    e, de = orc.eigen(N, j + 1)
    oP, oQ = orc.fixed_evolve(np.zeros(N), e[j], dt[0], n, order=3, sigma=0.5)
    assert np.abs(gP - oP).max() < 1e-11 and np.abs(gQ - oQ).max() < 1e-11
    w, T = 3.0 + 2.0 * j, n * dt[0]
    err = max(np.abs(gP - np.sin(w * T) * de[j] / w).max(), np.abs(gQ - np.cos(w * T) * e[j]).max())
    assert err < (1e-7 if j == 0 else 1e-5)
    assert np.all(gA == 1.0) and np.all(gd == 0.0)
    assert st[0] == ad.DONE


# the paper's production configuration (Sec. II, Table I: N = 32K, A evolved, third order) on
# clusters of 2, 4 and 8 CTAs, with and without re-integration
@pytest.mark.parametrize("N,reint,steps", [(8193, 0, 6), (16385, 3, 5), (32769, 2, 4), (4105, 0, 6)])
def test_evolved_a_on_clusters_matches_oracle(ad, orc, N, reint, steps):
    Phi, Pi = W.smooth_random(N, seed=N % 101, amp=2.5)
    s = ad.Solver([N], scheme=1, a_reint_every=reint, chunk_steps=3)
    s.set_initial(Phi, Pi)
    Ac = orc.constraints(Phi, Pi)[0]
    assert _close(s.get_state(0)[2], Ac, 1e-12)
    dt, _ = s.clock()
    tr, tc, m, st = s.evolve(steps * dt[0])
    r = orc.ea_evolve(Phi, Pi, Ac, dt[0], steps, order=3, reint=reint, sigma=0.5)
    gP, gQ, gA, gd = s.get_state(0)
    assert _close(gP, r.Phi, 1e-11) and _close(gQ, r.Pi, 1e-11)
    assert _close(gA, r.A, 1e-11) and _close(gd, r.delta, 1e-11)
    assert abs(m[0] - r.mass) <= 1e-11 * max(1.0, r.mass)


def test_evolved_a_mixed_cluster_batch_equals_single_runs(ad):
    Ns = [32769, 1025, 8193, 16385, 129]
    fields = [W.smooth_random(n, seed=400 + i, amp=2.0) for i, n in enumerate(Ns)]
    s = ad.Solver(Ns, scheme=1, a_reint_every=4, chunk_steps=3)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    tb = s.evolve(0.002)
    for i, n in enumerate(Ns):
        one = ad.Solver([n], scheme=1, a_reint_every=4, chunk_steps=3)
        one.set_initial(fields[i][0], fields[i][1])
        t1 = one.evolve(0.002)
        for x, y in zip(s.get_state(i), one.get_state(0)):
            assert np.array_equal(x, y)
        assert tb[2][i] == t1[2][0]


def test_fixed_metric_on_an_eight_cta_cluster(ad, orc):
    N, j = 32769, 2
    a = np.zeros((1, j + 1))
    a[0, j] = 1.0
    s = ad.Solver([N], scheme=ad.SCHEME_FIXED_METRIC_RK3)
    s.set_initial_modes(a)
    dt, _ = s.clock()
    n = 40
    s.evolve(n * dt[0])
    gP, gQ, gA, gd = s.get_state(0)
    e, de = orc.eigen(N, j + 1)
    oP, oQ = orc.fixed_evolve(np.zeros(N), e[j], dt[0], n, order=3, sigma=0.5)
    assert np.abs(gP - oP).max() < 1e-11 and np.abs(gQ - oQ).max() < 1e-11
    w, T = 3.0 + 2.0 * j, n * dt[0]
    assert np.abs(gQ - np.cos(w * T) * e[j]).max() < 1e-9
    assert np.all(gA == 1.0) and np.all(gd == 0.0)


# (32769, (8, 512, 16)): the paper's Table I grid on the 16-CTA cluster the autotuner picks for
# a single instance
@pytest.mark.parametrize("N,shape", [(4097, (8, 256, 2)), (2049, (8, 128, 2)), (1025, (8, 256, 2)),
                                     (36865, (8, 512, 9)), (4105, (8, 512, 9)), (32769, (8, 512, 16))])
@pytest.mark.parametrize("scheme", [1, 3])
def test_evolved_a_shapes_match_oracle(ad, orc, N, shape, scheme):
    Phi, Pi = W.smooth_random(N, seed=N + scheme, amp=2.0)
    s = ad.Solver([N, N], scheme=scheme, a_reint_every=3, chunk_steps=2)
    s.set_shape(N, *shape)
    assert s.shape(0) == shape
    s.set_initial(W.packed([Phi, Phi]), W.packed([Pi, Pi]))
    dt, _ = s.clock()
    s.evolve(7 * dt[0])
    gP, gQ, gA, _ = s.get_state(1)
    if scheme == 1:
        r = orc.ea_evolve(Phi, Pi, orc.constraints(Phi, Pi)[0], dt[0], 7, order=3, reint=3, sigma=0.5)
        oP, oQ, oA = r.Phi, r.Pi, r.A
    else:
        oP, oQ = orc.fixed_evolve(Phi, Pi, dt[0], 7, order=3, sigma=0.5)
        oA = np.ones(N)
    assert _close(gP, oP, 1e-11) and _close(gQ, oQ, 1e-11) and _close(gA, oA, 1e-11)


def test_evolved_a_autotune_keeps_state(ad):
    Ns = [2049] * 3 + [4097] * 2
    fields = [W.smooth_random(n, seed=600 + i, amp=2.0) for i, n in enumerate(Ns)]
    s = ad.Solver(Ns, scheme=1, a_reint_every=8)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    s.evolve(0.005)
    before = [s.get_state(b) for b in range(len(Ns))]
    clk = s.clock()[1].copy()
    shapes = s.autotune(trial_steps=4)
    for n, shp in shapes.items():
        assert shp[0] == 8 and (shp[1] == 512 or shp[2] == 2)
    for b in range(len(Ns)):
        after = s.get_state(b)
        for x, y in zip(before[b][:3], after[:3]):   # Phi, Pi and the evolved A are state
            assert np.array_equal(x, y)
    assert np.array_equal(clk, s.clock()[1])


@pytest.mark.parametrize("scheme", [1, 3])
def test_evolved_a_and_fixed_metric_without_dissipation(ad, orc, scheme):
    """sigma = 0 in the evolved-A and fixed-metric kernels (the dissipation term is switched off,
    Pi-dot is not divided by a dissipation factor)."""
    N, steps = 1025, 20
    Phi, Pi = W.smooth_random(N, seed=77 + scheme, amp=2.0)
    s = ad.Solver([N], scheme=scheme, a_reint_every=0, ko_sigma=0.0)
    s.set_initial(Phi, Pi)
    dt, _ = s.clock()
    s.evolve(steps * dt[0])
    gP, gQ, _, _ = s.get_state(0)
    if scheme == 1:
        r = orc.ea_evolve(Phi, Pi, orc.constraints(Phi, Pi)[0], dt[0], steps, order=3, reint=0, sigma=0.0)
        oP, oQ = r.Phi, r.Pi
    else:
        oP, oQ = orc.fixed_evolve(Phi, Pi, dt[0], steps, order=3, sigma=0.0)
    assert _close(gP, oP, 1e-11) and _close(gQ, oQ, 1e-11)


def test_fixed_metric_amp_scan_full_size_sampled(ad, orc):
    """The bench's fixed-metric line in its launch configuration: the 256-pulse amplitude scan at
    N = 4097 on the (8, 256, 2) shape, 16 SSP-RK3 steps; sampled instances match the oracle."""
    insts = W.amp_scan()
    n = insts[0].N
    Pi0 = W.packed([W.gaussian_pi(it.N, it.eps, it.sigma) for it in insts])
    s = ad.Solver([n] * len(insts), scheme=ad.SCHEME_FIXED_METRIC_RK3, collapse_threshold=2.0 ** -7)
    s.set_shape(n, 8, 256, 2)
    s.set_initial(np.zeros_like(Pi0), Pi0)
    dt, _ = s.clock()
    s.evolve(16 * dt[0])
    assert np.all(s.clock()[1] == 16)
    for b in (0, 131, len(insts) - 1):
        oP, oQ = orc.fixed_evolve(np.zeros(n), W.gaussian_pi(n, insts[b].eps, insts[b].sigma), dt[0], 16,
                                  order=3, sigma=0.5)
        gP, gQ, gA, gd = s.get_state(b)
        scale = max(1.0, np.abs(oQ).max())
        assert np.abs(gP - oP).max() <= 1e-11 * scale and np.abs(gQ - oQ).max() <= 1e-11 * scale
        assert np.all(gA == 1.0) and np.all(gd == 0.0)
    s.close()
