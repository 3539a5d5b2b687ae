"""Kernel shapes (P nodes per thread, NT threads per CTA, CL CTAs per instance) and the
autotuner: every shape the library is built with matches the oracle; batches mixing shapes
equal single-instance runs bit for bit; autotuning leaves the state untouched and is cached."""
import itertools

import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def _candidates():
    out = []
    # the 16-CTA shape is tested in tests/test_gpu_grid65537.py
    for P, NT, CL in itertools.product((4, 8), (128, 256, 512), (1, 2, 4, 8, 9)):
        nmax = P * NT * CL + 1
        out.append((P, NT, CL, nmax))
        small = 8 * CL * 3 + 1          # three node blocks of 8 per CTA, several tiles short
        if small < nmax:
            out.append((P, NT, CL, small))
    return out


def test_every_built_shape_matches_oracle(ad, orc):
    built = 0
    for P, NT, CL, N in _candidates():
        s = ad.Solver([N])
        try:
            s.set_shape(N, P, NT, CL)
        except ad.AdsclError as e:
            assert e.status == ad.ADSCL_EINVAL
            continue
        built += 1
        Phi, Pi = W.smooth_random(N, seed=N % 89 + P + NT, amp=3.0)
        s.set_initial(Phi, Pi)
        _, _, A, dl = s.get_state(0)
        Ao, dlo, _, _ = orc.constraints(Phi, Pi)
        assert np.abs(A - Ao).max() < 1e-12 * max(1.0, np.abs(Ao).max()), (P, NT, CL, N)
        assert np.abs(dl - dlo).max() < 1e-12 * max(1.0, np.abs(dlo).max()), (P, NT, CL, N)
        dt, _ = s.clock()
        s.evolve(2 * dt[0])
        gP, gQ, _, _ = s.get_state(0)
        oP, oQ = orc.rk4_step(*orc.rk4_step(Phi, Pi, dt[0], sigma=0.5), dt[0], sigma=0.5)
        scale = max(np.abs(oP).max(), np.abs(oQ).max())
        assert np.abs(gP - oP).max() < 1e-13 * scale and np.abs(gQ - oQ).max() < 1e-13 * scale, \
            (P, NT, CL, N)
        s.close()
    assert built >= 17


def test_mixed_shapes_batch_equals_single_runs(ad):
    cfg = [(1025, (4, 256, 1)), (2049, (8, 256, 2)), (4097, (4, 512, 2)), (513, (8, 128, 1)),
           (8193, (8, 256, 4)), (1025, (4, 256, 1))]
    Ns = [n for n, _ in cfg]
    fields = [W.smooth_random(n, seed=500 + i, amp=2.0) for i, n in enumerate(Ns)]
    s = ad.Solver(Ns, chunk_steps=5)
    for n, shp in cfg:
        s.set_shape(n, *shp)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    tb = s.evolve(0.01)
    for i, (n, shp) in enumerate(cfg):
        assert s.shape(i) == shp
        one = ad.Solver([n], chunk_steps=5)
        one.set_shape(n, *shp)
        one.set_initial(fields[i][0], fields[i][1])
        t1 = one.evolve(0.01)
        for x, y in zip(s.get_state(i), one.get_state(0)):
            assert np.array_equal(x, y)
        assert tb[2][i] == t1[2][0]


def test_autotune_keeps_state_and_is_cached(ad, orc):
    Ns = [1025] * 3 + [4097] * 2 + [129]
    fields = [W.smooth_random(n, seed=700 + i, amp=2.0) for i, n in enumerate(Ns)]
    Phi, Pi = W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields])
    s = ad.Solver(Ns)
    s.set_initial(Phi, Pi)
    s.evolve(0.01)
    before = [s.get_state(b) for b in range(len(Ns))]
    clk = s.clock()[1].copy()
    shapes = s.autotune(trial_steps=4)
    assert set(shapes) == {129, 1025, 4097}
    for b in range(len(Ns)):   # the slice is untouched; A, delta are re-solved with the new shape
        after = s.get_state(b)
        assert np.array_equal(before[b][0], after[0]) and np.array_equal(before[b][1], after[1])
        assert np.abs(before[b][2] - after[2]).max() < 1e-13
        assert np.abs(before[b][3] - after[3]).max() < 1e-13 * max(1.0, np.abs(after[3]).max())
    assert np.array_equal(clk, s.clock()[1])
    # the evolution continues correctly with the tuned shapes
    s.evolve(0.02)
    for b in (0, 3, 5):
        dt = s.clock()[0][b]
        n_done = int(s.clock()[1][b] - clk[b])
        r = orc.evolve(before[b][0], before[b][1], dt, n_done, sigma=0.5, n0=int(clk[b]))
        gP, gQ, _, _ = s.get_state(b)
        scale = max(1.0, np.abs(r.Pi).max())
        assert np.abs(gP - r.Phi).max() < 1e-11 * scale and np.abs(gQ - r.Pi).max() < 1e-11 * scale
    # a second context of the same sizes reuses the cached choice without touching its state
    s2 = ad.Solver(Ns)
    s2.set_initial(Phi, Pi)
    s2.evolve(0.005)
    before2 = [s2.get_state(b)[:2] for b in range(len(Ns))]
    clk2 = s2.clock()[1].copy()
    assert s2.autotune(trial_steps=4) == shapes
    assert np.array_equal(clk2, s2.clock()[1])
    for b in range(len(Ns)):
        after = s2.get_state(b)
        assert np.array_equal(before2[b][0], after[0]) and np.array_equal(before2[b][1], after[1])


def test_set_shape_rejects_what_does_not_fit(ad):
    s = ad.Solver([4097, 129])
    for bad in ((4, 256, 1), (8, 512, 3), (2, 512, 1)):
        with pytest.raises(ad.AdsclError) as e:
            s.set_shape(4097, *bad)
        assert e.value.status == ad.ADSCL_EINVAL
    with pytest.raises(ad.AdsclError):
        s.set_shape(2049, 8, 512, 1)          # no instance of that size
    s.set_shape(129, 8, 512, 8)               # 16 node blocks over 8 CTAs: fits
    assert s.shape(1) == (8, 512, 8)
    s.set_shape(129, 8, 128, 1)
    assert s.shape(1) == (8, 128, 1)


def test_autotune_after_collapses_keeps_state(ad):
    """A batch thinned by collapses (some instances stopped) is tuned again for the running ones
    (the cache is keyed by their number); the call changes no slice, step or status."""
    N, B = 1025, 24
    amps = np.where(np.arange(B) % 2 == 0, 40.0, 5.0)   # the strong half collapses early
    Pi = W.packed([W.gaussian_pi(N, e, 1.0 / 16) for e in amps])
    s = ad.Solver([N] * B, collapse_threshold=2.0 ** -7)
    s.set_initial(np.zeros_like(Pi), Pi)
    s.autotune(trial_steps=4)
    tr, tc, m, st = s.evolve(6.0)
    assert np.sum(st == ad.COLLAPSED) >= B // 2 - 2 and np.sum(st == ad.DONE) >= B // 2 - 2
    before = [s.get_state(b)[:2] for b in range(B)]
    clk = s.clock()[1].copy()
    s.autotune(trial_steps=4)
    assert np.array_equal(clk, s.clock()[1])
    for b in range(B):
        x = s.get_state(b)
        assert np.array_equal(before[b][0], x[0]) and np.array_equal(before[b][1], x[1])
    tr2, tc2, m2, st2 = s.evolve(6.5)
    assert np.array_equal(st2 == ad.COLLAPSED, st == ad.COLLAPSED)
    assert np.array_equal(tc2[st == ad.COLLAPSED], tc[st == ad.COLLAPSED])
