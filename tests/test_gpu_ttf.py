"""GPU TTF quantities (adscl_ttf) and spectrum tracking (adscl_track) against the CPU oracle
(oracle.ttf on oracle.spectrum of the oracle's own slices), through the C ABI.  The FP64
spectrum agrees with the oracle to ~1e-12 of the mass, so E and N do too; T = E / N likewise."""
import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def _oracle_ttf(orc, Phi, Pi, J):
    A, _, _, M = orc.constraints(Phi, Pi)
    E, _, _ = orc.spectrum(Phi, Pi, A, J)
    return orc.ttf(E), E, M


def test_ttf_of_an_uneven_batch_matches_oracle(ad, orc):
    Ns = [257, 1025, 4097, 1025, 129]
    fields = []
    for i, n in enumerate(Ns):
        if i % 2 == 0:
            a = 0.2 * np.exp(-np.arange(12) / 3.0) * (1 + 0.1 * np.sin(np.arange(12) + i))
            fields.append(orc.synthesize(n, a))
        else:
            fields.append(W.smooth_random(n, seed=40 + i, amp=1.5))
    s = ad.Solver(Ns, ko_sigma=0.5)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    for J in (64, 20):
        q, E = s.ttf(J, ad.PREC_FP64, with_energies=True)
        assert np.array_equal(E, s.spectrum(J, ad.PREC_FP64))
        for b, n in enumerate(Ns):
            qo, Eo, M = _oracle_ttf(orc, fields[b][0], fields[b][1], J)
            assert np.abs(E[b] - Eo).max() <= 1e-12 * M
            assert abs(q[b, 0] - qo[0]) <= 1e-12 * M
            assert abs(q[b, 1] - qo[1]) <= 1e-12 * M
            assert abs(q[b, 2] / qo[2] - 1.0) <= 1e-11
            if J == 64 and n >= 1025:
                assert abs(q[b, 0] / M - 1.0) <= 1e-8      # total energy = mass


def test_track_matches_oracle_snapshots(ad, orc):
    """Three instances at N = 257 tracked at t = 0.25 k, k < 7: one collapses (min A < 0.05) (its rows stay on
    its last slice), two evolve; every snapshot's time, E, N, T and mode energies match the
    oracle run step by step to the same slices."""
    N, J, cad, n_snap = 257, 32, 0.25, 7
    theta = 0.05
    a = 0.3 * np.exp(-np.arange(8) / 2.0)
    fields = [orc.synthesize(N, a), W.smooth_random(N, seed=77, amp=1.0),
              (np.zeros(N), W.gaussian_pi(N, 40.0, sigma=0.1))]
    s = ad.Solver([N] * 3, ko_sigma=0.5, out_dt=cad, spec_J=J, collapse_threshold=theta)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    dt, _ = s.clock()
    th, qh, Eh = s.track(0.0, cad, n_snap, J, ad.PREC_FP64, energies=True)
    _, tc, _, st = s.evolve(cad * (n_snap - 1))
    assert st[2] == ad.COLLAPSED and st[0] == ad.DONE and st[1] == ad.DONE
    for b in range(3):
        Phi, Pi = fields[b]
        n_done, minA, stopped = 0, float("nan"), False
        for k in range(n_snap):
            n_k = int(round(k * cad / dt[b]))
            if n_k > n_done and not stopped:
                r = orc.evolve(Phi, Pi, dt[b], n_k - n_done, sigma=0.5, theta=theta, n0=n_done,
                               minA_in=minA)
                Phi, Pi, minA = r.Phi, r.Pi, r.minA
                n_done += r.steps
                stopped = r.status == orc.COLLAPSED
            assert th[k, b] == n_done * dt[b]
            qo, Eo, M = _oracle_ttf(orc, Phi, Pi, J)
            scale = max(M, 1e-300)
            assert np.abs(Eh[k, b] - Eo).max() <= 1e-10 * scale, (k, b)
            assert abs(qh[k, b, 0] - qo[0]) <= 1e-10 * scale and abs(qh[k, b, 1] - qo[1]) <= 1e-10 * scale
            assert abs(qh[k, b, 2] / qo[2] - 1.0) <= 1e-9
    # the collapsed instance stays on its last slice
    kc = int(np.searchsorted(cad * np.arange(n_snap), tc[2]))
    assert np.all(th[kc:, 2] == th[kc, 2]) and th[kc, 2] < cad * kc


def test_track_device_pointers_equal_host_pointers(ad):
    import torch
    N, J, cad, n_snap = 129, 16, 0.5, 3
    a = np.array([[0.3, 0.1, 0.05], [0.2, -0.2, 0.1]])
    out = []
    for dev in (False, True):
        s = ad.Solver([N] * 2, ko_sigma=0.5, out_dt=cad)
        s.set_initial_modes(a)
        if not dev:
            th, qh, Eh = s.track(0.0, cad, n_snap, J, ad.PREC_FP64, energies=True)
        else:
            d = torch.device("cuda", 0)
            th = torch.empty((n_snap, 2), dtype=torch.float64, device=d)
            qh = torch.empty((n_snap, 2, 3), dtype=torch.float64, device=d)
            Eh = torch.empty((n_snap, 2, J), dtype=torch.float64, device=d)
            assert s.lib.adscl_track(s.ctx, 0.0, cad, n_snap, J, ad.PREC_FP64, th.data_ptr(),
                                     qh.data_ptr(), Eh.data_ptr(), 1) == ad.ADSCL_OK
            torch.cuda.synchronize()
            th, qh, Eh = th.cpu().numpy(), qh.cpu().numpy(), Eh.cpu().numpy()
        out.append((th, qh, Eh))
    for x, y in zip(*out):
        assert np.array_equal(x, y)


def test_track_rejects_bad_arguments(ad):
    s = ad.Solver([129], ko_sigma=0.5)
    s.set_initial_modes(np.array([[0.3]]))
    for args in ((0.0, 0.5, 0), (-1.0, 0.5, 2), (0.0, 0.0, 2), (0.0, float("inf"), 2)):
        with pytest.raises(ad.AdsclError) as e:
            s.track(*args, J=8)
        assert e.value.status == ad.ADSCL_EINVAL
    with pytest.raises(ad.AdsclError):
        s.track(0.0, 0.5, 2, J=65)


def test_ttf_of_static_ads_is_zero_energy_and_undefined_temperature(ad, orc):
    """Static AdS (Phi = Pi = 0): every mode energy is 0, so E = N = 0 and T = 0/0 = NaN, as in
    the oracle; a normal mode beside it in the same batch is unaffected."""
    s = ad.Solver([129, 129], ko_sigma=0.5)
    Phi1, Pi1 = orc.synthesize(129, np.array([0.0, 0.02]))
    s.set_initial(np.concatenate([np.zeros(129), Phi1]), np.concatenate([np.zeros(129), Pi1]))
    q = s.ttf(16)
    assert q[0, 0] == 0.0 and q[0, 1] == 0.0 and np.isnan(q[0, 2])
    assert np.isnan(orc.ttf(np.zeros(16))[2])
    assert abs(q[1, 2] - 5.0) < 1e-6                       # single mode j = 1: T = omega_1


@pytest.mark.parametrize("prec", ["BF16X3", "TF32X3"])
def test_track_on_tensor_cores_within_the_derived_bound(ad, prec):
    """A tracked job of an uneven batch with the tensor-core spectrum: every snapshot's mode
    energies agree with those of the same job tracked with the FP64 projection within the derived
    bound of the split-precision projection (tests/test_gpu_spectrum.py tc_bound), relative to the
    slice's mass; the TTF quantities follow."""
    from test_gpu_spectrum import tc_bound
    rng = np.random.default_rng(12)
    Ns = [2049] * 3 + [4097] * 2 + [1025] * 4
    a = np.stack([rng.uniform(0.05, 0.2) * np.exp(-np.arange(16) / 3.0) for _ in Ns])
    res = {}
    for p in ("FP64", prec):
        s = ad.Solver(Ns, ko_sigma=0.5, out_dt=0.25)
        s.set_initial_modes(a)
        res[p] = s.track(0.0, 0.25, 4, 64, getattr(ad, "PREC_" + p), energies=True)
        s.close()
    (t0, q0, E0), (t1, q1, E1) = res["FP64"], res[prec]
    assert np.array_equal(t0, t1)
    bound = tc_bound(prec, 1)
    for k in range(4):
        rel = np.abs(E1[k] - E0[k]).max(axis=1) / q0[k, :, 0]
        assert rel.max() <= bound, (k, rel.max(), bound)
        assert np.all(np.abs(q1[k, :, 0] - q0[k, :, 0]) <= 64 * bound * q0[k, :, 0])
