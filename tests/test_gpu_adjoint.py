"""GPU discrete adjoint (adscl_grad) against the CPU oracle's adjoint and against central
differences of the GPU forward functional."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


@pytest.mark.parametrize("N,nsteps,ckpt", [(129, 40, 16), (1025, 24, 8)])
def test_grad_matches_oracle_adjoint(ad, orc, N, nsteps, ckpt):
    B, K, Jm = 3, 6, 8
    rng = np.random.default_rng(N)
    a = rng.uniform(0.0, 0.8, (B, K)) * np.exp(-np.arange(K) / 2.0)
    s = ad.Solver([N] * B, ko_sigma=0.5, spec_J=Jm, ckpt_every=ckpt)
    dt, _ = s.clock()
    J, g = s.grad(a, nsteps * dt[0])
    for b in range(B):
        Jo, go = orc.grad(a[b], N, nsteps, dt[0], sigma=0.5, Jm=Jm)
        assert abs(J[b] - Jo) <= 1e-10 * abs(Jo), (b, J[b], Jo)
        big = np.abs(go) > 1e-3 * np.abs(go).max()
        assert np.all(np.abs(g[b] - go)[big] <= 1e-9 * np.abs(go)[big]), (b, g[b], go)


def test_grad_against_central_differences_of_gpu_forward(ad):
    N, nsteps, K, Jm = 257, 30, 5, 8
    rng = np.random.default_rng(7)
    a0 = rng.uniform(0.1, 0.6, K) * np.exp(-np.arange(K) / 2.0)
    s = ad.Solver([N], ko_sigma=0.5, spec_J=Jm, ckpt_every=7)
    dt, _ = s.clock()
    T = nsteps * dt[0]
    J, g = s.grad(a0[None, :], T)
    eps = 1e-6
    for k in range(K):
        ap, am = a0.copy(), a0.copy()
        ap[k] += eps
        am[k] -= eps
        Jp, _ = s.grad(ap[None, :], T)
        Jm_, _ = s.grad(am[None, :], T)
        fd = (Jp[0] - Jm_[0]) / (2 * eps)
        if abs(g[0, k]) > 1e-3 * np.abs(g).max():
            assert abs(fd - g[0, k]) <= 1e-5 * abs(g[0, k]), (k, fd, g[0, k])


def test_autograd_function_matches_grad(ad):
    """torch.autograd.Function wrapper: backward of sum(w * J) is w * dJ/da from adscl_grad,
    for device tensors (asynchronous call on the solver's stream) and host tensors."""
    import torch
    from paper_1706_07413_b300.autograd import mode_drift
    N, B, K, Jm = 257, 3, 6, 8
    rng = np.random.default_rng(3)
    a0 = rng.uniform(0.1, 0.5, (B, K)) * np.exp(-np.arange(K) / 2.0)
    st = torch.cuda.Stream()
    s = ad.Solver([N] * B, ko_sigma=0.5, spec_J=Jm, ckpt_every=9, stream=st.cuda_stream)
    dt, _ = s.clock()
    T = 40 * dt[0]
    Jref, gref = s.grad(a0, T)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    for dev in ("cuda", "cpu"):
        a = torch.tensor(a0, dtype=torch.float64, device=dev, requires_grad=True)
        J = mode_drift(s, a, T)
        (J * w.to(dev)).sum().backward()
        assert np.array_equal(J.detach().cpu().numpy(), Jref)
        assert np.allclose(a.grad.cpu().numpy(), w.numpy()[:, None] * gref, rtol=1e-15, atol=0)


def test_adjoint_refinement_reduces_drift_of_qp_seeds(ad):
    """Adjoint-driven refinement of the 8 approximate quasi-periodic seeds (k_d in {3, 5}, mu in
    {1, 1.75}, eps in {0.05, 0.1}): the spectral drift J decreases monotonically."""
    from paper_1706_07413_b300 import workloads as W
    from paper_1706_07413_b300.autograd import refine_modes
    N, K = 513, 32
    seeds = W.qp_seeds(N=N, K=K)
    a0 = np.stack([it.coeffs for it in seeds])
    s = ad.Solver([N] * len(seeds), ko_sigma=0.5, spec_J=32, ckpt_every=64)
    dt, _ = s.clock()
    a, hist = refine_modes(s, a0, 200 * dt[0], iters=4, step=0.02)
    h = hist.numpy()
    assert np.all(np.diff(h, axis=0) <= 0.0)
    assert np.all(h[-1] < h[0])


@pytest.mark.parametrize("N", [257, 1025])
def test_one_and_two_cta_adjoint_agree(ad, orc, N):
    """The adjoint kernel on one CTA per instance and on a 2-CTA cluster (node blocks split between
    the two CTAs, scan totals carried across) gives the same gradient up to the rounding of the
    re-associated scans; both match the oracle's adjoint."""
    B, K, Jm = 4, 6, 8
    rng = np.random.default_rng(11)
    a = rng.uniform(0.0, 0.8, (B, K)) * np.exp(-np.arange(K) / 2.0)
    out = {}
    for ctas in (1, 2):
        s = ad.Solver([N] * B, ko_sigma=0.5, spec_J=Jm, ckpt_every=9, adjoint_ctas=ctas)
        dt, _ = s.clock()
        out[ctas] = s.grad(a, 30 * dt[0])
        s.close()
    J1, g1 = out[1]
    J2, g2 = out[2]
    assert np.abs(J1 - J2).max() <= 1e-12 * np.abs(J1).max()
    assert np.abs(g1 - g2).max() <= 1e-11 * np.abs(g1).max()
    Jo, go = orc.grad(a[2], N, 30, dt[0], sigma=0.5, Jm=Jm)
    assert abs(J2[2] - Jo) <= 1e-10 * abs(Jo)
    assert np.abs(g2[2] - go).max() <= 1e-9 * np.abs(go).max()


@pytest.mark.parametrize("bufs", [1, 2, 0])
def test_stage_storage_modes_agree(ad, orc, bufs):
    """One stage buffer (recompute, then sweep, per segment), two (recomputation beside the
    sweep) and one per segment (the forward pass stores every stage) give the oracle's gradient;
    the context ends on the final slice at step n in every mode."""
    N, B, K, Jm, n = 257, 3, 6, 8, 40
    rng = np.random.default_rng(21)
    a = rng.uniform(0.0, 0.8, (B, K)) * np.exp(-np.arange(K) / 2.0)
    s = ad.Solver([N] * B, ko_sigma=0.5, spec_J=Jm, ckpt_every=9, adjoint_stage_buffers=bufs)
    dt, _ = s.clock()
    assert s.adjoint_storage() == (0, 0, 0, 0)
    J, g = s.grad(a, n * dt[0])
    assert s.adjoint_storage()[2:] == (5, 0 if bufs == 0 else 5)   # phase F recomputes every segment
    for b in (0, 2):
        Jo, go = orc.grad(a[b], N, n, dt[0], sigma=0.5, Jm=Jm)
        assert abs(J[b] - Jo) <= 1e-10 * abs(Jo)
        assert np.abs(g[b] - go).max() <= 1e-9 * np.abs(go).max()
    assert np.all(s.clock()[1] == n)
    # the final slice equals a plain forward evolution (to rounding)
    ref = ad.Solver([N] * B, ko_sigma=0.5, spec_J=Jm, collapse_threshold=-1.0)
    ref.set_initial_modes(a)
    ref.evolve(n * dt[0])
    for b in range(B):
        x, y = s.get_state(b), ref.get_state(b)
        assert np.abs(x[0] - y[0]).max() < 1e-12 and np.abs(x[1] - y[1]).max() < 1e-12
    # and the context keeps evolving from it
    s.evolve((n + 5) * dt[0])
    assert np.all(s.clock()[1] == n + 5)


@pytest.mark.parametrize("extra", [5, "quarter"])
def test_recording_forward_pass_for_batches_filling_the_gpu(ad, orc, extra):
    """A batch with at least one evolution CTA per SM records its stages in the evolution
    kernel's stage-recording variant: with a buffer per segment the forward pass writes them all
    in one launch; with a cap of one or two buffers the forward pass writes the last one or two
    segments and each earlier one is recomputed from its checkpoint on a second slice before its
    sweep.  A quarter of that on the default one-CTA shapes runs these passes on 4-CTA clusters.  The three storage modes give the same gradients up to rounding and the
    oracle's adjoint, and each leaves the context on the final slice."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    N, K, Jm, n = 129, 6, 8, 20
    B = sms + 5 if extra == 5 else sms // 4 + 3
    rng = np.random.default_rng(31)
    a = rng.uniform(0.0, 0.8, (B, K)) * np.exp(-np.arange(K) / 2.0)
    out = {}
    ref = None
    for bufs in (0, 1, 2):
        s = ad.Solver([N] * B, ko_sigma=0.5, spec_J=Jm, ckpt_every=9, adjoint_stage_buffers=bufs)
        dt, _ = s.clock()
        if ref is None:
            ref = ad.Solver([N] * 2, ko_sigma=0.5, spec_J=Jm, collapse_threshold=-1.0)
            ref.set_initial_modes(a[[0, B - 1]])
            ref.evolve(n * dt[0])
        out[bufs] = s.grad(a, n * dt[0])
        assert np.all(s.clock()[1] == n)
        nbytes, nbuf, nseg, nrecomp = s.adjoint_storage()
        assert nseg == 3 and nrecomp == {0: 0, 1: 2, 2: 1}[bufs]
        assert nbuf == (3 if bufs == 0 else bufs) and nbytes == nbuf * B * 9 * 4 * 6 * N * 8
        for k, b in enumerate((0, B - 1)):   # the context ends on the final slice
            x, y = s.get_state(b), ref.get_state(k)
            if extra == 5:   # same shape: the recording variant does the same arithmetic
                assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
            else:            # recorded on 4-CTA clusters: the scans associate differently
                assert np.abs(x[0] - y[0]).max() < 1e-13 and np.abs(x[1] - y[1]).max() < 1e-13
        s.close()
    ref.close()
    (J0, g0) = out[0]
    for bufs in (1, 2):
        J1, g1 = out[bufs]
        assert np.abs(J0 - J1).max() <= 1e-12 * np.abs(J1).max()
        assert np.abs(g0 - g1).max() <= 1e-10 * np.abs(g1).max()
    for b in (0, B // 2, B - 1):
        Jo, go = orc.grad(a[b], N, n, dt[0], sigma=0.5, Jm=Jm)
        assert abs(J0[b] - Jo) <= 1e-10 * abs(Jo)
        assert np.abs(g0[b] - go).max() <= 1e-9 * np.abs(go).max()


@pytest.mark.parametrize("shape", [(8, 512, 9), (8, 512, 16)])
def test_recording_on_non_portable_cluster_shapes(ad, orc, shape):
    """The stage-recording variant of the evolution kernel on the 9- and 16-CTA clusters: a batch
    set to that shape spreads over every SM, so its forward pass records the stages, with one
    buffer per segment or with one buffer and the earlier segments recomputed; both match the
    oracle's adjoint."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    N, K, Jm, n = 289, 6, 8, 20
    B = -(-sms // shape[2])   # enough clusters for one CTA per SM
    rng = np.random.default_rng(37)
    a = rng.uniform(0.0, 0.8, (B, K)) * np.exp(-np.arange(K) / 2.0)
    grads = {}
    for bufs in (0, 1):
        s = ad.Solver([N] * B, ko_sigma=0.5, spec_J=Jm, ckpt_every=9, adjoint_stage_buffers=bufs)
        s.set_shape(N, *shape)
        dt, _ = s.clock()
        grads[bufs] = s.grad(a, n * dt[0])
        assert np.all(s.clock()[1] == n)
        _, nbuf, nseg, nrecomp = s.adjoint_storage()
        assert nseg == 3 and nrecomp == (0 if bufs == 0 else 2)
        assert s.shape(0) == shape   # the context's shape is kept
        s.close()
    (J0, g0), (J1, g1) = grads[0], grads[1]
    assert np.abs(J0 - J1).max() <= 1e-12 * np.abs(J1).max()
    assert np.abs(g0 - g1).max() <= 1e-10 * np.abs(g1).max()
    for b in (0, B - 1):
        Jo, go = orc.grad(a[b], N, n, dt[0], sigma=0.5, Jm=Jm)
        assert abs(J0[b] - Jo) <= 1e-10 * abs(Jo)
        assert np.abs(g0[b] - go).max() <= 1e-9 * np.abs(go).max()


@pytest.mark.parametrize("ctas", [1, 2])
def test_grad_without_dissipation_matches_oracle(ad, orc, ctas):
    """sigma = 0: the dissipation terms of the transposed step are switched off as in the
    forward step."""
    N, B, K, Jm, n = 129, 2, 6, 8, 30
    rng = np.random.default_rng(41)
    a = rng.uniform(0.0, 0.8, (B, K)) * np.exp(-np.arange(K) / 2.0)
    s = ad.Solver([N] * B, ko_sigma=0.0, spec_J=Jm, ckpt_every=9, adjoint_ctas=ctas)
    dt, _ = s.clock()
    J, g = s.grad(a, n * dt[0])
    for b in range(B):
        Jo, go = orc.grad(a[b], N, n, dt[0], sigma=0.0, Jm=Jm)
        assert abs(J[b] - Jo) <= 1e-10 * abs(Jo)
        assert np.abs(g[b] - go).max() <= 1e-9 * np.abs(go).max()


def test_grad_at_8193_points_matches_oracle(ad, orc):
    """N = 8193 (the large-grid configuration): the adjoint kernel runs each instance on a 2-CTA
    cluster with 8 nodes per thread."""
    # 200 steps (t = 0.019): long enough that J = sum (E_j(T) - E_j(0))^2 is not dominated by
    # the cancellation in E_j(T) - E_j(0)
    N, B, K, Jm, n = 8193, 2, 6, 8, 200
    rng = np.random.default_rng(51)
    a = rng.uniform(0.0, 0.8, (B, K)) * np.exp(-np.arange(K) / 2.0)
    s = ad.Solver([N] * B, ko_sigma=0.5, spec_J=Jm, ckpt_every=64)
    dt, _ = s.clock()
    J, g = s.grad(a, n * dt[0])
    for b in range(B):
        Jo, go = orc.grad(a[b], N, n, dt[0], sigma=0.5, Jm=Jm)
        assert abs(J[b] - Jo) <= 1e-10 * abs(Jo)
        assert np.abs(g[b] - go).max() <= 1e-9 * np.abs(go).max()
    s.close()
    s1 = ad.Solver([N], ko_sigma=0.5, spec_J=Jm, adjoint_ctas=1)
    with pytest.raises(ad.AdsclError) as e:
        s1.grad(a[:1], n * dt[0])
    assert e.value.status == ad.ADSCL_EUNSUPPORTED


def test_qp_seed_refinement_at_8193_points(ad):
    """The large-grid configuration's refinement: the 8 approximate quasi-periodic seeds at
    N = 8193, a few adjoint-driven steps lower every seed's spectral drift."""
    from paper_1706_07413_b300 import workloads as W
    from paper_1706_07413_b300.autograd import refine_modes
    N, K = 8193, 32
    seeds = W.qp_seeds(N=N, K=K)
    a0 = np.stack([it.coeffs for it in seeds])
    s = ad.Solver([N] * len(seeds), ko_sigma=0.5, spec_J=32, ckpt_every=64)
    dt, _ = s.clock()
    a, hist = refine_modes(s, a0, 128 * dt[0], iters=3, step=0.02)
    h = hist.numpy()
    assert np.all(np.diff(h, axis=0) <= 0.0)
    assert np.all(h[-1] < h[0])
