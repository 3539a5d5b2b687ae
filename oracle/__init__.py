"""CPU oracle for the AdS4 Einstein-Klein-Gordon evolution (arXiv:1706.07413, Sec. II).

TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library and its Python binding) never
imports, links or runs anything under ``oracle/``; only ``tests/``, the package smoke check
and the CPU-baseline leg of ``bench.py`` do.  The oracle shares no code with the CUDA path.

The arithmetic lives in ``adscl_oracle.c`` (plain sequential FP64 C); this module only builds
it with gcc and marshals numpy arrays through ctypes.  Parity status of each function:

- ``constraints``, ``rhs``, ``rk4_step``, ``evolve``: pinned by static AdS, closed-form
  delta and m solutions, linear normal-mode dynamics, 4th-order self-convergence, mass and
  momentum-constraint convergence (tests/test_oracle_pins.py).
- ``eigen``, ``spectrum``, ``synthesize``: pinned by the hypergeometric closed form at high
  precision, Gauss-Legendre orthonormality, the eigen-equation and the paper's printed
  temperatures (tests/test_oracle_eigen.py).
- ``ttf`` (total energy, particle number, temperature): pinned by single-mode data
  (T = omega_j), the paper's printed temperatures reached through synthesis, constraint solve
  and spectrum, the total energy equal to the mass, exact conservation of every mode energy by
  the linear (fixed-metric) evolution up to truncation error, and the O(eps^2) drift of the
  particle number under the full scheme (tests/test_oracle_ttf.py).
- collapse time: the detection rule is pinned by invariants; the value itself is
  "parity unpinned" (the paper prints no collapse time).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adscl_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

RUNNING, DONE, COLLAPSED, NONFINITE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        I, L, F = ctypes.c_int, ctypes.c_long, ctypes.c_double
        _lib.orc_constraints.argtypes = [I, D, D, D, D, D, D]
        _lib.orc_constraints.restype = None
        _lib.orc_rhs.argtypes = [I, F, D, D, D, D, D, D]
        _lib.orc_rhs.restype = None
        _lib.orc_rk4_step.argtypes = [I, F, F, D, D]
        _lib.orc_rk4_step.restype = None
        _lib.orc_evolve.argtypes = [I, F, L, L, F, F, F, D, D, D, D, D, D, D]
        _lib.orc_evolve.restype = I
        _lib.orc_eigen_at.argtypes = [I, I, D, D, D]
        _lib.orc_eigen_at.restype = None
        _lib.orc_eigen.argtypes = [I, I, D, D]
        _lib.orc_eigen.restype = None
        _lib.orc_spectrum.argtypes = [I, I, D, D, D, D, D, D]
        _lib.orc_spectrum.restype = None
        _lib.orc_ttf.argtypes = [I, D, D]
        _lib.orc_ttf.restype = None
        _lib.orc_synthesize.argtypes = [I, I, D, D, D]
        _lib.orc_synthesize.restype = None
        _lib.orc_constraints_vjp.argtypes = [I, D, D, D, D, D, D]
        _lib.orc_constraints_vjp.restype = None
        _lib.orc_rhs_vjp.argtypes = [I, F, D, D, D, D, D, D, D, D, D, D]
        _lib.orc_rhs_vjp.restype = None
        _lib.orc_rk4_step_vjp.argtypes = [I, F, F, D, D, D, D]
        _lib.orc_rk4_step_vjp.restype = None
        _lib.orc_spectrum_vjp.argtypes = [I, I, D, D, D, D, D]
        _lib.orc_spectrum_vjp.restype = None
        _lib.orc_grad.argtypes = [I, I, D, L, F, F, I, D, D]
        _lib.orc_grad.restype = None
        _lib.orc_adot.argtypes = [I, D, D, D, D, D]
        _lib.orc_adot.restype = None
        _lib.orc_mass_simpson.argtypes = [I, D, D, D]
        _lib.orc_mass_simpson.restype = F
        _lib.orc_ea_step.argtypes = [I, I, F, F, D, D, D]
        _lib.orc_ea_step.restype = None
        _lib.orc_ea_evolve.argtypes = [I, I, I, F, L, L, F, F, F, D, D, D, D, D]
        _lib.orc_ea_evolve.restype = I
        _lib.orc_fixed_step.argtypes = [I, I, F, F, D, D]
        _lib.orc_fixed_step.restype = None
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def grid(N: int) -> np.ndarray:
    """Node-centred grid x_i = i*pi/(2(N-1))."""
    return np.arange(N, dtype=np.float64) * (0.5 * math.pi / (N - 1))


def dt_for(N: int, cfl: float = 0.5, cadence: float = 1.0) -> float:
    """Time step dt = D / ceil(D / (cfl*h)): the largest step <= cfl*h that lands on multiples
    of the output cadence D."""
    h = 0.5 * math.pi / (N - 1)
    return cadence / math.ceil(cadence / (cfl * h))


def constraints(Phi, Pi):
    """Returns (A, delta, m, mass) for one slice (Eqs. (eq:aprime), (eq:delta))."""
    Phi, Pi = _f64(Phi), _f64(Pi)
    N = Phi.size
    A, dl, m = np.empty(N), np.empty(N), np.empty(N)
    mass = ctypes.c_double()
    lib().orc_constraints(N, _p(Phi), _p(Pi), _p(A), _p(dl), _p(m), ctypes.byref(mass))
    return A, dl, m, mass.value


def rhs(Phi, Pi, A, delta, sigma=0.0):
    """Returns (dPhi/dt, dPi/dt) (Eqs. (eq:phi), (eq:pi)) plus Kreiss-Oliger dissipation."""
    Phi, Pi, A, delta = map(_f64, (Phi, Pi, A, delta))
    N = Phi.size
    dPhi, dPi = np.empty(N), np.empty(N)
    lib().orc_rhs(N, sigma, _p(Phi), _p(Pi), _p(A), _p(delta), _p(dPhi), _p(dPi))
    return dPhi, dPi


def rk4_step(Phi, Pi, dt, sigma=0.0):
    Phi, Pi = _f64(Phi).copy(), _f64(Pi).copy()
    lib().orc_rk4_step(Phi.size, dt, sigma, _p(Phi), _p(Pi))
    return Phi, Pi


class EvolveResult:
    __slots__ = ("Phi", "Pi", "A", "delta", "t_reached", "t_collapse", "mass", "minA",
                 "steps", "status", "delta0", "mass_hist", "minA_hist")


def evolve(Phi, Pi, dt, nsteps, sigma=0.5, theta=2.0 ** -7, n0=0, minA_in=float("nan"),
           history=False):
    """Evolve one instance by at most nsteps RK4 steps from step index n0 (stops at collapse)."""
    Phi, Pi = _f64(Phi).copy(), _f64(Pi).copy()
    N = Phi.size
    A, dl = np.empty(N), np.empty(N)
    out = np.empty(7)
    mh = np.empty(nsteps + 1) if history else None
    ah = np.empty(nsteps + 1) if history else None
    lib().orc_evolve(N, dt, n0, nsteps, sigma, theta, minA_in, _p(Phi), _p(Pi), _p(A), _p(dl),
                     _p(out), _p(mh), _p(ah))
    r = EvolveResult()
    r.Phi, r.Pi, r.A, r.delta = Phi, Pi, A, dl
    r.t_reached, r.t_collapse, r.mass, r.minA = out[0], out[1], out[2], out[3]
    r.steps, r.status, r.delta0 = int(out[4]), int(out[5]), out[6]
    if history:
        r.mass_hist, r.minA_hist = mh[: r.steps + 1], ah[: r.steps + 1]
    else:
        r.mass_hist = r.minA_hist = None
    return r


def adot(Phi, Pi, A, delta):
    """A-dot of Eq. (eq:adot) on one slice."""
    Phi, Pi, A, delta = map(_f64, (Phi, Pi, A, delta))
    dA = np.empty(Phi.size)
    lib().orc_adot(Phi.size, _p(Phi), _p(Pi), _p(A), _p(delta), _p(dA))
    return dA


def mass_simpson(Phi, Pi, A):
    """The paper's mass integral by the composite Simpson rule on the nodes."""
    Phi, Pi, A = map(_f64, (Phi, Pi, A))
    return lib().orc_mass_simpson(Phi.size, _p(Phi), _p(Pi), _p(A))


def ea_step(Phi, Pi, A, dt, order=3, sigma=0.0):
    """One SSP Runge-Kutta step (order 2 or 3) of the evolved-A scheme."""
    Phi, Pi, A = _f64(Phi).copy(), _f64(Pi).copy(), _f64(A).copy()
    lib().orc_ea_step(Phi.size, order, dt, sigma, _p(Phi), _p(Pi), _p(A))
    return Phi, Pi, A


def ea_evolve(Phi, Pi, A, dt, nsteps, order=3, reint=0, sigma=0.5, theta=2.0 ** -7, n0=0,
              minA_in=float("nan")):
    """Evolve one instance with the evolved-A scheme (A given; re-integrated every `reint`
    steps when reint > 0).  Returns an EvolveResult (mass = Simpson mass)."""
    Phi, Pi, A = _f64(Phi).copy(), _f64(Pi).copy(), _f64(A).copy()
    N = Phi.size
    dl = np.empty(N)
    out = np.empty(7)
    lib().orc_ea_evolve(N, order, reint, dt, n0, nsteps, sigma, theta, minA_in, _p(Phi), _p(Pi),
                        _p(A), _p(dl), _p(out))
    r = EvolveResult()
    r.Phi, r.Pi, r.A, r.delta = Phi, Pi, A, dl
    r.t_reached, r.t_collapse, r.mass, r.minA = out[0], out[1], out[2], out[3]
    r.steps, r.status, r.delta0 = int(out[4]), int(out[5]), out[6]
    r.mass_hist = r.minA_hist = None
    return r


def fixed_evolve(Phi, Pi, dt, nsteps, order=3, sigma=0.5):
    """nsteps SSP Runge-Kutta steps of the fixed-metric case (A = 1, delta = 0)."""
    Phi, Pi = _f64(Phi).copy(), _f64(Pi).copy()
    for _ in range(nsteps):
        lib().orc_fixed_step(Phi.size, order, dt, sigma, _p(Phi), _p(Pi))
    return Phi, Pi


def eigen_at(J, x):
    """e_j(x), e_j'(x) for j < J at arbitrary points x; arrays of shape (J, len(x))."""
    x = _f64(x)
    e, de = np.empty(J * x.size), np.empty(J * x.size)
    lib().orc_eigen_at(J, x.size, _p(x), _p(e), _p(de))
    return e.reshape(J, x.size), de.reshape(J, x.size)


def eigen(N, J):
    e, de = np.empty(J * N), np.empty(J * N)
    lib().orc_eigen(N, J, _p(e), _p(de))
    return e.reshape(J, N), de.reshape(J, N)


def omega(j):
    return 3.0 + 2.0 * np.asarray(j, dtype=np.float64)


def spectrum(Phi, Pi, A, J):
    """E_j, Pi_j, Phi_j for j < J on one slice."""
    Phi, Pi, A = map(_f64, (Phi, Pi, A))
    N = Phi.size
    E, pj, fj = np.empty(J), np.empty(J), np.empty(J)
    lib().orc_spectrum(N, J, _p(Phi), _p(Pi), _p(A), _p(E), _p(pj), _p(fj))
    return E, pj, fj


def ttf(E):
    """(E, N, T) of one slice from its mode energies E_j: total energy, particle number
    sum_j E_j / omega_j and temperature E / N (the two TTF conserved quantities fixed by the
    spectrum, and their ratio)."""
    E = _f64(E)
    out = np.empty(3)
    lib().orc_ttf(E.size, _p(E), _p(out))
    return out


def synthesize(N, a):
    """Pi(x,0) = sum_j a_j e_j(x), Phi(x,0) = 0."""
    a = _f64(a)
    Phi, Pi = np.empty(N), np.empty(N)
    lib().orc_synthesize(N, a.size, _p(a), _p(Phi), _p(Pi))
    return Phi, Pi


def constraints_vjp(Phi, Pi, Abar, dbar):
    """Sensitivities to (Phi, Pi) of sum(Abar*A + dbar*delta): transpose of constraints()."""
    Phi, Pi, Abar, dbar = map(_f64, (Phi, Pi, Abar, dbar))
    N = Phi.size
    gP, gQ = np.zeros(N), np.zeros(N)
    lib().orc_constraints_vjp(N, _p(Phi), _p(Pi), _p(Abar), _p(dbar), _p(gP), _p(gQ))
    return gP, gQ


def rhs_vjp(Phi, Pi, A, delta, vP, vQ, sigma=0.0):
    """Sensitivities to (Phi, Pi, A, delta) of sum(vP*dPhi + vQ*dPi) at fixed A, delta."""
    Phi, Pi, A, delta, vP, vQ = map(_f64, (Phi, Pi, A, delta, vP, vQ))
    N = Phi.size
    out = [np.zeros(N) for _ in range(4)]
    lib().orc_rhs_vjp(N, sigma, _p(Phi), _p(Pi), _p(A), _p(delta), _p(vP), _p(vQ), *map(_p, out))
    return tuple(out)


def rk4_step_vjp(Phi, Pi, lP, lQ, dt, sigma=0.0):
    """Transpose of one RK4 step at the input (Phi, Pi): sensitivity to the input."""
    Phi, Pi = _f64(Phi), _f64(Pi)
    lP, lQ = _f64(lP).copy(), _f64(lQ).copy()
    lib().orc_rk4_step_vjp(Phi.size, dt, sigma, _p(Phi), _p(Pi), _p(lP), _p(lQ))
    return lP, lQ


def spectrum_vjp(Phi, Pi, Ebar):
    """Sensitivities to (Phi, Pi) of sum(Ebar*E) (E with A from the same slice)."""
    Phi, Pi, Ebar = map(_f64, (Phi, Pi, Ebar))
    N = Phi.size
    gP, gQ = np.zeros(N), np.zeros(N)
    lib().orc_spectrum_vjp(N, Ebar.size, _p(Phi), _p(Pi), _p(Ebar), _p(gP), _p(gQ))
    return gP, gQ


def grad(a, N, nsteps, dt, sigma=0.5, Jm=32):
    """J = sum_{j<Jm}(E_j(T) - E_j(0))^2 for Pi(x,0) = sum a_k e_k and dJ/da (discrete adjoint)."""
    a = _f64(a)
    out = np.zeros(1)
    g = np.zeros(a.size)
    lib().orc_grad(N, a.size, _p(a), nsteps, dt, sigma, Jm, _p(out), _p(g))
    return float(out[0]), g


def functional(a, N, nsteps, dt, sigma=0.5, Jm=32):
    """J alone, by the forward routines only (for finite-difference checks)."""
    Phi, Pi = synthesize(N, a)
    A, _, _, _ = constraints(Phi, Pi)
    E0, _, _ = spectrum(Phi, Pi, A, Jm)
    for _ in range(nsteps):
        Phi, Pi = rk4_step(Phi, Pi, dt, sigma)
    A, _, _, _ = constraints(Phi, Pi)
    ET, _, _ = spectrum(Phi, Pi, A, Jm)
    return float(np.sum((ET - E0) ** 2))


def temperature_from_energies(E):
    """T = sum_j E_j / sum_j (E_j / omega_j): energy over particle number of the modes
    (the third output of ttf)."""
    return float(ttf(E)[2])


def momentum_residual(A_levels, dt, Phi, Pi, A, delta):
    """RMS over interior points of the momentum constraint (Eq. (eq:adot)) residual at level n:
    (A^{n-2} - 8A^{n-1} + 8A^{n+1} - A^{n+2})/(12 dt) + 2 sin x cos x A^2 e^{-delta} Phi Pi,
    with A_levels = [A^{n-2}, A^{n-1}, A^{n+1}, A^{n+2}] and the other fields at level n."""
    N = Phi.size
    x = grid(N)
    a2, a1, p1, p2 = A_levels
    adot = (a2 - 8 * a1 + 8 * p1 - p2) / (12 * dt)
    r = adot + 2 * np.sin(x) * np.cos(x) * A ** 2 * np.exp(-delta) * Phi * Pi
    return float(np.sqrt(np.mean(r[1:-1] ** 2)))
