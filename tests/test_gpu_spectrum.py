"""GPU parity of the normal-mode machinery (mode-sum initial data, FP64 mode-energy spectrum)
with the CPU oracle, and the paper's printed temperatures through the GPU path."""
import json
import math
import os

import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def test_mode_sum_initial_data_matches_oracle(ad, orc):
    Ns = [129, 1025, 4097]
    rng = np.random.default_rng(3)
    a = np.zeros((3, 64))
    a[:, :24] = rng.uniform(-1, 1, (3, 24)) * np.exp(-np.arange(24) / 5.0)
    s = ad.Solver(Ns)
    s.set_initial_modes(np.ascontiguousarray(a[:, :24]))
    for b, N in enumerate(Ns):
        Phi, Pi, A, dl = s.get_state(b)
        oPhi, oPi = orc.synthesize(N, a[b, :24])
        oA, odl, _, _ = orc.constraints(oPhi, oPi)
        assert np.all(Phi == 0.0)
        assert np.abs(Pi - oPi).max() < 1e-11 * max(1.0, np.abs(oPi).max())
        assert np.abs(A - oA).max() < 1e-11 and np.abs(dl - odl).max() < 1e-11


@pytest.mark.parametrize("kind", ["random", "gauss"])
def test_fp64_spectrum_matches_oracle(ad, orc, kind):
    Ns = [257, 2049, 4097]
    if kind == "random":
        fields = [W.smooth_random(n, seed=60 + i, amp=2.0) for i, n in enumerate(Ns)]
    else:
        fields = [(np.zeros(n), W.gaussian_pi(n, 8.0, sigma=0.25)) for n in Ns]
    s = ad.Solver(Ns)
    s.set_initial(W.packed([f[0] for f in fields]), W.packed([f[1] for f in fields]))
    if kind == "gauss":
        s.evolve(0.3)          # a slice with both Phi and Pi populated
    E = s.spectrum(64)
    for b, N in enumerate(Ns):
        Phi, Pi, A, _ = s.get_state(b)
        oA, _, _, M = orc.constraints(Phi, Pi)
        Eo, _, _ = orc.spectrum(Phi, Pi, oA, 64)
        assert np.abs(E[b] - Eo).max() <= 1e-12 * M, (b, np.abs(E[b] - Eo).max(), M)


def test_paper_temperatures_through_the_gpu_path(ad):
    """Approximate QP data (Eq. (eq:approxQP)) synthesised on the GPU and projected back by the
    GPU spectrum give the temperatures printed in the paper (Sec. II)."""
    gold = json.load(open(os.path.join(GOLDEN, "qp_temperatures.json")))
    N = 2049
    cases = gold["cases"]
    a = np.stack([W.approx_qp_coefficients(c["kd"], c["mu"], eps=1e-4, K=32) for c in cases])
    s = ad.Solver([N] * len(cases))
    s.set_initial_modes(np.ascontiguousarray(a))
    E = s.spectrum(40)
    w = 3.0 + 2.0 * np.arange(40)
    for b, c in enumerate(cases):
        T = E[b].sum() / (E[b] / w).sum()
        tol = 0.5 * 10 ** (math.floor(math.log10(c["T"])) - c["digits"] + 1)
        assert abs(T - c["T"]) <= tol, (c, T)


def tc_bound(prec, chunks):
    """Derived bound on max_j |E_j(TC) - E_j| / M of the split-precision projection: 2 eps with
    eps = 3 2^-2p (1 + 2^-p)  (operand split: the dropped lo*lo and the remainders)
        + c n 2^-23 (1 + 2^{1-p})  (FP32 accumulation: at most one unit in the last place per
                                    MMA instruction, n per 64 points, over runs of c chunks),
    p = 8 / 11 bits and n = 4 / 8 instructions for BF16 / TF32; the factor 2 M follows from
    |dE_j| <= 2 |P_j| |dP_j| and Cauchy-Schwarz, sum |u_k b_k| <= sqrt(M) |b| with |e_j| = 1 and
    |e_j'| = omega_j in the weighted norm."""
    p, n = (8, 4) if prec == "BF16X3" else (11, 8)
    eps = 3 * 2.0 ** (-2 * p) * (1 + 2.0 ** -p) + chunks * n * 2.0 ** -23 * (1 + 2.0 ** (1 - p))
    return 2 * eps


@pytest.mark.parametrize("chunks", [1, 4, 129])
@pytest.mark.parametrize("prec", ["BF16X3", "TF32X3"])
def test_tensor_core_spectrum_error_vs_oracle(ad, orc, prec, chunks):
    """Split-precision tensor-core projection (tcgen05, FP32 accumulation) against the oracle's
    FP64 projection of the same slices, on an uneven batch (five grid sizes up to 8193, two
    128-row tiles for one of them), with FP32 accumulation runs of 1, 4 and up to 129 chunks of
    64 grid points (129: a whole N = 8193 row): max_j |E_j(TC) - E_j(oracle)| / M stays below
    the derived bound tc_bound.  Small E_j (<< M) are not relatively accurate at this
    precision."""
    rng = np.random.default_rng(9)
    # N = 257 needs two 128-row tiles; the other sizes are those of the uneven configuration
    Ns = [257] * 140 + [1025] * 5 + [2049] * 5 + [4097] * 2 + [8193] * 2
    a = np.zeros((len(Ns), 16))
    j = np.arange(16)
    for b in range(len(Ns)):
        a[b] = rng.uniform(0.05, 0.2) * np.exp(-j / 3.0) * (1 + 0.05 * rng.standard_normal(16))
    s = ad.Solver(Ns, spectrum_chunks=chunks)
    s.set_initial_modes(a)
    s.evolve(0.25)
    Etc = s.spectrum(64, getattr(ad, "PREC_" + prec))
    E64 = s.spectrum(64, ad.PREC_FP64)
    assert np.all(np.isfinite(Etc))
    worst = 0.0
    for b in (0, 77, 139, 140, 144, 145, 150, 152, 153):
        Phi, Pi, _, _ = s.get_state(b)
        oA, _, _, M = orc.constraints(Phi, Pi)
        Eo, _, _ = orc.spectrum(Phi, Pi, oA, 64)
        assert np.abs(E64[b] - Eo).max() <= 1e-12 * M
        worst = max(worst, np.abs(Etc[b] - Eo).max() / M)
    _, _, mass, _ = s.evolve(0.25)
    every = (np.abs(Etc - E64).max(axis=1) / mass).max()
    print(f"{prec} chunks={chunks}: max_j |dE_j|/M vs oracle {worst:.3e}, over the batch vs the "
          f"FP64 path {every:.3e}, derived bound {tc_bound(prec, chunks):.3e}")
    assert worst <= tc_bound(prec, chunks) and every <= tc_bound(prec, chunks)
