"""Seeded synthetic inputs for the AdS4 collapse workloads.

This module holds random draws and initial-profile formulas only: none of the scheme's
arithmetic (constraint solve, right-hand side, time stepping, eigenbasis, spectrum).  Both
the CUDA path and the CPU oracle take their inputs from here.  Draws use
``numpy.random.default_rng(seed)``.

Workloads (sizes follow the runs described in arXiv:1706.07413 Sec. II-III and the solver's
benchmark set):

- ``single``:   one Gaussian pulse, N = 1025, eps = 40, sigma = 1/16, to t = 10.
- ``amp_scan``: B = 256 Gaussian pulses, N = 4097, sigma = 1/16, eps log-uniform in [5, 80],
  to t = 100 or collapse (min A < 2^-7).
- ``uneven``:   192 mode-sum instances, N drawn from {2049, 4097, 8193},
  a_j = eps exp(-j/3)(1 + 0.05 n_j), j < 16, eps ~ U[0.05, 0.2], to t = 200.
- ``adjoint``:  64 mode-sum instances, N = 4097, a_j = U(0, 0.1) exp(-j/4), j < 32, T = 2 pi.
- ``large``:    148 instances at N = 8193, half Gaussian (sigma ~ U[1/32, 1/8], eps as
  amp_scan), half two-mode Pi = eps (e_0 + r e_1)/sqrt(1 + r^2), r ~ U[0.5, 2],
  eps log-uniform in [0.05, 0.2]; plus 8 approximate quasi-periodic seeds (Eq. (eq:approxQP)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAUSS_SIGMA = 1.0 / 16.0


def grid(N: int) -> np.ndarray:
    """Sample points x_i = i*pi/(2(N-1)) of the node-centred grid on [0, pi/2]."""
    return np.arange(N, dtype=np.float64) * (0.5 * math.pi / (N - 1))


def gaussian_pi(N: int, eps: float, sigma: float = GAUSS_SIGMA) -> np.ndarray:
    """Pi(x,0) = (2 eps / pi) exp(-4 tan^2 x / (pi^2 sigma^2)) on the grid (Phi(x,0) = 0)."""
    x = grid(N)
    with np.errstate(over="ignore"):
        t2 = np.tan(x) ** 2
    pi0 = (2.0 * eps / math.pi) * np.exp(-4.0 * t2 / (math.pi ** 2 * sigma ** 2))
    pi0[-1] = 0.0
    return pi0


def approx_qp_amplitudes(kd: int, mu: float, eps: float, K: int = 32) -> np.ndarray:
    """TTF amplitudes A_k = eps exp(-mu |k - kd|), k < K (Eq. (eq:approxQP))."""
    k = np.arange(K, dtype=np.float64)
    return eps * np.exp(-mu * np.abs(k - kd))


def approx_qp_coefficients(kd: int, mu: float, eps: float, K: int = 32) -> np.ndarray:
    """Mode coefficients a_k = omega_k A_k of Pi(x,0) = sum_k a_k e_k(x) for the approximate
    quasi-periodic data (mode energy E_k = a_k^2 = omega_k^2 A_k^2, omega_k = 3 + 2k)."""
    k = np.arange(K, dtype=np.float64)
    return (3.0 + 2.0 * k) * approx_qp_amplitudes(kd, mu, eps, K)


@dataclass
class Instance:
    N: int
    kind: str                  # "gauss" or "modes"
    eps: float = 0.0
    sigma: float = GAUSS_SIGMA
    coeffs: np.ndarray = field(default_factory=lambda: np.zeros(0))


def single() -> list:
    return [Instance(N=1025, kind="gauss", eps=40.0, sigma=GAUSS_SIGMA)]


def amp_scan(B: int = 256, N: int = 4097, seed: int = 0) -> list:
    rng = np.random.default_rng(seed)
    eps = np.exp(rng.uniform(math.log(5.0), math.log(80.0), size=B))
    return [Instance(N=N, kind="gauss", eps=float(e), sigma=GAUSS_SIGMA) for e in eps]


def uneven(B: int = 192, seed: int = 1, J: int = 16) -> list:
    rng = np.random.default_rng(seed)
    Ns = rng.choice(np.array([2049, 4097, 8193]), size=B)
    eps = rng.uniform(0.05, 0.2, size=B)
    out = []
    j = np.arange(J, dtype=np.float64)
    for b in range(B):
        a = eps[b] * np.exp(-j / 3.0) * (1.0 + 0.05 * rng.standard_normal(J))
        out.append(Instance(N=int(Ns[b]), kind="modes", coeffs=a))
    return out


def adjoint_batch(B: int = 64, N: int = 4097, seed: int = 2, J: int = 32) -> list:
    rng = np.random.default_rng(seed)
    j = np.arange(J, dtype=np.float64)
    return [Instance(N=N, kind="modes", coeffs=rng.uniform(0.0, 0.1, size=J) * np.exp(-j / 4.0))
            for _ in range(B)]


def large(B: int = 148, N: int = 8193, seed: int = 3) -> list:
    rng = np.random.default_rng(seed)
    out = []
    for b in range(B):
        if b % 2 == 0:
            sig = rng.uniform(1.0 / 32.0, 1.0 / 8.0)
            eps = math.exp(rng.uniform(math.log(5.0), math.log(80.0)))
            out.append(Instance(N=N, kind="gauss", eps=eps, sigma=sig))
        else:
            r = rng.uniform(0.5, 2.0)
            eps = math.exp(rng.uniform(math.log(0.05), math.log(0.2)))
            a = np.zeros(2)
            a[0], a[1] = eps / math.sqrt(1 + r * r), eps * r / math.sqrt(1 + r * r)
            out.append(Instance(N=N, kind="modes", coeffs=a))
    return out


def production(B: int = 15, N: int = 32769, seed: int = 4) -> list:
    """Gaussian pulses at the paper's production resolution (its Table I grid of 2^15 + 1 points):
    one 8-CTA cluster per instance; a B300 holds 15 such clusters at once (120 of its 148 SMs)."""
    rng = np.random.default_rng(seed)
    eps = np.exp(rng.uniform(math.log(5.0), math.log(80.0), size=B))
    return [Instance(N=N, kind="gauss", eps=float(e), sigma=GAUSS_SIGMA) for e in eps]


def qp_seeds(N: int = 8193, K: int = 32) -> list:
    out = []
    for kd in (3, 5):
        for mu in (1.0, 1.75):
            for eps in (0.05, 0.1):
                out.append(Instance(N=N, kind="modes", coeffs=approx_qp_coefficients(kd, mu, eps, K)))
    return out


def smooth_random(N: int, seed: int, amp: float = 1.0, terms: int = 5):
    """A smooth random slice with the boundary parities of the fields:
    Pi = amp cos^3 x sum_k c_k sin^{2k} x,  Phi = amp sin x cos^2 x sum_k d_k sin^{2k} x,
    c_k, d_k ~ N(0, 1) / (k + 1).  Returns (Phi, Pi)."""
    rng = np.random.default_rng(seed)
    x = grid(N)
    s2 = np.sin(x) ** 2
    c = rng.standard_normal(terms) / (1.0 + np.arange(terms))
    dd = rng.standard_normal(terms) / (1.0 + np.arange(terms))
    poly_c = sum(c[k] * s2 ** k for k in range(terms))
    poly_d = sum(dd[k] * s2 ** k for k in range(terms))
    Pi = amp * np.cos(x) ** 3 * poly_c
    Phi = amp * np.sin(x) * np.cos(x) ** 2 * poly_d
    Pi[-1] = 0.0
    Phi[0] = Phi[-1] = 0.0
    return Phi, Pi


def packed(fields):
    """Concatenate per-instance arrays into the packed layout of the C ABI."""
    return np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.float64) for f in fields]))
