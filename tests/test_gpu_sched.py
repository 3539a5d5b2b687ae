"""GPU tests of the solver's own exp and of the chunked persistent scheduler."""
import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def test_exp_neg_within_two_ulp_of_libm(ad):
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(0, 1, 20000), rng.uniform(0, 60, 20000), rng.uniform(0, 1e-6, 2000),
                        rng.uniform(0, 700, 2000), [0.0, 1e-300, 5e-324, np.log(2) / 512, 699.999]])
    y = ad.exp_neg(x)
    ref = np.exp(-x)
    err = np.abs(y - ref) / np.spacing(ref)
    assert err.max() <= 2.0, (err.max(), x[np.argmax(err)])
    assert y[x == 0.0][0] == 1.0
    big = ad.exp_neg(np.array([700.5, 1e4]))
    assert big[0] == 0.0 and big[1] == 0.0
    assert np.isnan(ad.exp_neg(np.array([np.nan]))[0])


def test_exp_neg_scaled_within_two_ulp(ad):
    """The kernels' exp takes its argument in units of ln2/256; the reference e^{-X ln2/256} is
    evaluated in 40-digit arithmetic (the product X ln2/256 would itself round in FP64)."""
    from mpmath import mp, mpf, exp, log
    rng = np.random.default_rng(1)
    X = np.concatenate([rng.uniform(0, 400, 3000), rng.uniform(0, 25000, 3000),
                        rng.uniform(0, 258000, 1000), rng.uniform(0, 1e-6, 200),
                        np.arange(-3, 4) * 0.5 + 1000, [0.0, 0.5, 1.0, 1.5, 5e-324, 258531.0]])
    y = ad.exp_neg_scaled(X)
    with mp.workdps(40):
        L = log(2) / 256
        ref = np.array([float(exp(-mpf(float(v)) * L)) for v in X])
    err = np.abs(y - ref) / np.spacing(ref)
    assert err.max() <= 2.0, (err.max(), X[np.argmax(err)])
    assert y[X == 0.0][0] == 1.0
    big = ad.exp_neg_scaled(np.array([258700.0, 3.7e6]))
    assert big[0] == 0.0 and big[1] == 0.0
    assert np.isnan(ad.exp_neg_scaled(np.array([np.nan]))[0])


def _batch(ad, Ns, seed, chunk, amp=3.0, t_end=0.08, **kw):
    fields = [W.smooth_random(n, seed=seed + i, amp=amp) for i, n in enumerate(Ns)]
    s = ad.Solver(Ns, ko_sigma=0.5, collapse_threshold=2.0 ** -7, chunk_steps=chunk, **kw)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    out = s.evolve(t_end)
    return s, out


def test_chunk_size_does_not_change_bits(ad):
    """Instances migrate between SMs at chunk boundaries (B > #SMs here); results are
    bit-identical for every chunk length."""
    Ns = [129] * 200 + [257] * 60
    ref_s, ref_o = _batch(ad, Ns, 11, chunk=1000)
    for chunk in (1, 3, 16):
        s, o = _batch(ad, Ns, 11, chunk=chunk)
        for x, y in zip(o, ref_o):
            assert np.array_equal(x, y)
        for b in (0, 57, 199, 200, 259):
            for x, y in zip(s.get_state(b), ref_s.get_state(b)):
                assert np.array_equal(x, y)


def test_collapsing_and_long_instances_mixed(ad):
    """Strong pulses collapse early while weak ones run on; every instance equals its own
    single-instance run (CTAs retire as instances finish)."""
    N = 257
    eps = [60.0, 2.0, 45.0, 1.0, 70.0]
    Pi = W.packed([W.gaussian_pi(N, e, sigma=0.125) for e in eps])
    s = ad.Solver([N] * len(eps), ko_sigma=0.5, collapse_threshold=0.05, chunk_steps=4)
    s.set_initial(np.zeros_like(Pi), Pi)
    tr, tc, m, st = s.evolve(6.0)
    assert (st == ad.COLLAPSED).sum() >= 1 and (st == ad.DONE).sum() >= 1
    for b, e in enumerate(eps):
        one = ad.Solver([N], ko_sigma=0.5, collapse_threshold=0.05)
        one.set_initial(np.zeros(N), W.gaussian_pi(N, e, sigma=0.125))
        t1 = one.evolve(6.0)
        assert t1[3][0] == st[b] and t1[0][0] == tr[b] and (t1[1][0] == tc[b] or np.isinf(tc[b]))
        for x, y in zip(s.get_state(b), one.get_state(0)):
            assert np.array_equal(x, y)


def test_bounded_wait_times_out_cleanly(ad):
    """With a one-iteration wait limit and one-step chunks, the CTA that finishes a chunk of the
    small instance (N = 129, ~60 us) first must wait for the large one's chunk (N = 4097,
    ~400 us) and gives up: the call returns ADSCL_ETIMEOUT and leaves nothing running; a solver
    with the default limit then completes the same request."""
    Ns = [4097, 129]
    fields = [W.smooth_random(n, seed=40 + i, amp=1.0) for i, n in enumerate(Ns)]
    s = ad.Solver(Ns, ko_sigma=0.5, chunk_steps=1, max_device_iters=1)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    dt, _ = s.clock()
    t_end = 8 * dt[1]          # 8 steps of the small instance, ~500 of the large one
    with pytest.raises(ad.AdsclError) as ei:
        s.evolve(t_end)
    assert ei.value.status == ad.ADSCL_ETIMEOUT
    s2 = ad.Solver(Ns, ko_sigma=0.5, chunk_steps=1)
    s2.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    tr, tc, m, st = s2.evolve(t_end)
    assert np.all(st == ad.DONE)
