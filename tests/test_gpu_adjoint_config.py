"""Discrete-adjoint parity at the adjoint configuration's own settings: N = 4097, checkpoints
every 256 steps, a 768-step window (three segments), mode data a_j = U(0, 0.1) e^{-j/4}, j < 32,
J = sum_{j<32} (E_j(T) - E_j(0))^2, in every stage-storage mode and on both adjoint kernels:

- the 64-instance batch (it fills the GPU on 4-CTA recording shapes): every stage stored by the
  recording forward pass, and one buffer (the last segment recorded by the forward pass, the two
  earlier ones recomputed by the recording evolution kernel before their sweeps);
- two instances (they do not fill the GPU): phase F (the recomputation) on the adjoint kernel,
  with one buffer and with two (recomputation of one segment beside the sweep of the next).

Bars: J within 1e-10 relative and dJ/da within 1e-9 of the largest component, against the
oracle's hand-written adjoint; and central differences (h = 1e-6) of the GPU functional on the
three largest components within 1e-5 relative.  Oracle cost: ~9 s per instance (768 steps
forward and backward at N = 4097 on one host core); four instances run on host threads."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu

N, K, JM, CKPT, NSTEPS = 4097, 32, 32, 256, 768
SAMPLE = (0, 1, 33, 63)


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


@pytest.fixture(scope="module")
def case(orc):
    a = np.stack([it.coeffs for it in W.adjoint_batch(N=N, J=K)])
    dt = orc.dt_for(N)

    def run(b):
        return b, orc.grad(a[b], N, NSTEPS, dt, sigma=0.5, Jm=JM)

    with ThreadPoolExecutor(max_workers=max(1, min(len(SAMPLE), os.cpu_count() or 1))) as ex:
        ref = dict(ex.map(run, SAMPLE))
    return a, dt, ref


def _check(J, g, b_gpu, ref):
    Jo, go = ref
    assert abs(J[b_gpu] - Jo) <= 1e-10 * abs(Jo), (b_gpu, J[b_gpu], Jo)
    assert np.abs(g[b_gpu] - go).max() <= 1e-9 * np.abs(go).max(), (b_gpu, np.abs(g[b_gpu] - go).max())


@pytest.mark.parametrize("ctas", [1, 2])
@pytest.mark.parametrize("bufs", [0, 1])
def test_full_adjoint_batch_matches_oracle(ad, case, ctas, bufs):
    a, dt, ref = case
    s = ad.Solver([N] * a.shape[0], ko_sigma=0.5, spec_J=JM, ckpt_every=CKPT, adjoint_ctas=ctas,
                  adjoint_stage_buffers=bufs)
    assert abs(s.clock()[0][0] - dt) == 0.0
    J, g = s.grad(a, NSTEPS * dt)
    _, nbuf, nseg, nrec = s.adjoint_storage()
    assert nseg == 3 and nrec == (0 if bufs == 0 else 2) and nbuf == (3 if bufs == 0 else 1)
    for b in SAMPLE:
        _check(J, g, b, ref[b])
    s.close()


@pytest.mark.parametrize("ctas", [1, 2])
@pytest.mark.parametrize("bufs", [1, 2])
def test_small_batch_phase_f_on_the_adjoint_kernel(ad, case, ctas, bufs):
    a, dt, ref = case
    s = ad.Solver([N] * 2, ko_sigma=0.5, spec_J=JM, ckpt_every=CKPT, adjoint_ctas=ctas,
                  adjoint_stage_buffers=bufs)
    J, g = s.grad(a[:2], NSTEPS * dt)
    _, nbuf, nseg, nrec = s.adjoint_storage()
    assert nseg == 3 and nrec == 3 and nbuf == bufs
    for b in (0, 1):
        _check(J, g, b, ref[b])
    s.close()


def test_central_differences_at_4097_points(ad, case):
    a, dt, ref = case
    s = ad.Solver([N], ko_sigma=0.5, spec_J=JM, ckpt_every=CKPT)
    T = NSTEPS * dt
    a0 = a[0].copy()
    J0, g0 = s.grad(a0[None, :], T)
    h = 1e-6
    for k in np.argsort(-np.abs(g0[0]))[:3]:
        ap, am = a0.copy(), a0.copy()
        ap[k] += h
        am[k] -= h
        fd = (s.grad(ap[None, :], T)[0][0] - s.grad(am[None, :], T)[0][0]) / (2 * h)
        assert abs(fd - g0[0, k]) <= 1e-5 * abs(g0[0, k]), (k, fd, g0[0, k])
    s.close()
