"""adscl_evolve_noalloc: the evolution for callers that cannot allocate device memory.

Such callers are, for example, programs that give the whole GPU memory to their own pool when
they start and forbid allocations outside it, latency-critical loops that cannot afford the
device-wide synchronisation of cudaMalloc/cudaFree, and plug-ins inside frameworks that own
every allocation.  The entry point takes the caller's device buffers for the fields and the
results and keeps all other working storage in one fixed device array of the library.

Its results must agree with the allocating path (adscl_create + adscl_set_initial +
adscl_evolve + adscl_get_state) within the parity tolerance of the other GPU tests, on two calls
in a row with different batch shapes (the second call finds the first call's data in the fixed
array).  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def _allocating_path(ad, N, Phi0, Pi0, t_end):
    B = Phi0.size // N
    s = ad.Solver([N] * B, ko_sigma=0.5, collapse_threshold=2.0 ** -7)
    s.set_initial(Phi0, Pi0)
    tr, tc, m, st = s.evolve(t_end)
    states = [s.get_state(b) for b in range(B)]
    Phi = np.concatenate([x[0] for x in states])
    Pi = np.concatenate([x[1] for x in states])
    return tr, tc, m, st, Phi, Pi


def _noalloc_path(ad, N, Phi0, Pi0, t_end):
    import torch
    dev = torch.device("cuda", 0)
    B = Phi0.size // N
    Phi = torch.from_numpy(Phi0.copy()).to(dev)
    Pi = torch.from_numpy(Pi0.copy()).to(dev)
    outs = [torch.full((B,), -1.0, dtype=torch.float64, device=dev) for _ in range(3)]
    outs.append(torch.full((B,), -1, dtype=torch.int32, device=dev))
    torch.cuda.synchronize()
    rc = ad.evolve_noalloc(Phi, Pi, N, t_end, *outs, ko_sigma=0.5, collapse_threshold=2.0 ** -7,
                           stream=torch.cuda.current_stream().cuda_stream)
    assert rc == ad.ADSCL_OK, ad.STATUS_NAMES.get(rc, rc)
    torch.cuda.synchronize()
    tr, tc, m, st = (o.cpu().numpy() for o in outs)
    return tr, tc, m, st, Phi.cpu().numpy(), Pi.cpu().numpy()


def _compare(ref, got):
    tr0, tc0, m0, st0, P0, Q0 = ref
    tr1, tc1, m1, st1, P1, Q1 = got
    assert np.array_equal(st0, st1)
    assert np.array_equal(tr0, tr1)
    assert np.array_equal(np.isinf(tc0), np.isinf(tc1))
    fin = ~np.isinf(tc0)
    assert np.allclose(tc0[fin], tc1[fin], rtol=1e-3, atol=0)
    assert np.all(np.abs(m1 - m0) <= 1e-12 * np.abs(m0) + 1e-300)
    scale = max(1.0, np.abs(Q0).max(), np.abs(P0).max())
    assert np.abs(P1 - P0).max() <= 1e-11 * scale
    assert np.abs(Q1 - Q0).max() <= 1e-11 * scale


def test_noalloc_matches_allocating_path_twice_in_a_row(ad):
    # call 1: 16 pulses of the amplitude scan at N = 4097 (the full capacity), 40 RK4 steps
    N1 = 4097
    insts = W.amp_scan()[:16]
    Pi1 = W.packed([W.gaussian_pi(N1, it.eps, it.sigma) for it in insts])
    Phi1 = np.zeros_like(Pi1)
    t1 = 40.0 / 5216.0
    _compare(_allocating_path(ad, N1, Phi1, Pi1, t1), _noalloc_path(ad, N1, Phi1, Pi1, t1))
    # call 2: a different shape (5 slices at N = 1025, one pulse strong enough to collapse)
    N2 = 1025
    fields = [W.smooth_random(N2, seed=500 + i, amp=3.0) for i in range(4)]
    Phi2 = W.packed([f[0] for f in fields] + [np.zeros(N2)])
    Pi2 = W.packed([f[1] for f in fields] + [W.gaussian_pi(N2, 40.0)])
    t2 = 5.0
    ref2 = _allocating_path(ad, N2, Phi2, Pi2, t2)
    assert (ref2[3] == ad.COLLAPSED).any()
    _compare(ref2, _noalloc_path(ad, N2, Phi2, Pi2, t2))


def test_noalloc_rejects_requests_beyond_its_capacity(ad):
    import torch
    dev = torch.device("cuda", 0)
    for B, N in ((ad.NOALLOC_MAX_INSTANCES + 1, 129), (17, 4097)):
        Phi = torch.zeros(B * N, dtype=torch.float64, device=dev)
        Pi = torch.ones(B * N, dtype=torch.float64, device=dev)
        outs = [torch.zeros(B, dtype=torch.float64, device=dev) for _ in range(3)]
        outs.append(torch.zeros(B, dtype=torch.int32, device=dev))
        rc = ad.evolve_noalloc(Phi, Pi, N, 0.1, *outs)
        assert rc == ad.ADSCL_ECAPACITY
        torch.cuda.synchronize()
        assert float(Pi.min()) == 1.0 and float(Phi.abs().max()) == 0.0   # nothing ran


def test_noalloc_refuses_bad_arguments_before_queuing_anything(ad):
    """A refused call (bad N, or a t_end whose step count the work queue cannot hold) returns
    ADSCL_EINVAL with the caller's fields and outputs untouched."""
    import torch
    dev = torch.device("cuda", 0)
    for B, N, t_end in ((4, 1003, 0.1), (4, 129, 1e300), (64, 4097 // 8 + 1, 4.0e6), (2, 129, -1.0),
                        (2, 129, float("nan"))):
        Phi = torch.zeros(B * N, dtype=torch.float64, device=dev)
        Pi = torch.ones(B * N, dtype=torch.float64, device=dev)
        outs = [torch.full((B,), 7.0, dtype=torch.float64, device=dev) for _ in range(3)]
        outs.append(torch.full((B,), 7, dtype=torch.int32, device=dev))
        torch.cuda.synchronize()
        rc = ad.evolve_noalloc(Phi, Pi, N, t_end, *outs)
        assert rc == ad.ADSCL_EINVAL, (B, N, t_end, rc)
        torch.cuda.synchronize()
        assert float(Pi.min()) == 1.0 and float(Pi.max()) == 1.0 and float(Phi.abs().max()) == 0.0
        for o in outs:
            assert bool((o == 7).all())


def test_noalloc_reports_a_nonfinite_instance_and_evolves_the_others(ad):
    """An instance whose initial slice holds a NaN is reported NONFINITE at t = 0; the other
    instances of the batch match the allocating path run without it."""
    N = 513
    fields = [W.smooth_random(N, seed=900 + i, amp=2.0) for i in range(3)]
    Phi0 = W.packed([f[0] for f in fields])
    Pi0 = W.packed([f[1] for f in fields])
    t_end = 0.5
    ref = _allocating_path(ad, N, Phi0, Pi0, t_end)
    bad_Pi = Pi0.copy()
    bad_Pi[N + N // 3] = np.nan                          # instance 1, an interior node
    got = _noalloc_path(ad, N, Phi0, bad_Pi, t_end)
    assert got[3][1] == ad.NONFINITE and got[0][1] == 0.0
    keep = [0, 2]
    sl = np.concatenate([np.arange(b * N, (b + 1) * N) for b in keep])
    _compare(tuple(x[keep] for x in ref[:4]) + (ref[4][sl], ref[5][sl]),
             tuple(x[keep] for x in got[:4]) + (got[4][sl], got[5][sl]))
