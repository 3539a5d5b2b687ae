"""Python binding of the C ABI in include/adscl.h (ctypes; argument marshalling only).

Every computation runs in ``libadscl.so`` (CUDA, sm_103a).  There is no CPU fallback: if the
library is missing or cannot be loaded, importing a solver raises.  The functions below keep
the C names; ``Solver`` is a thin object wrapper that accepts numpy arrays (host pointers,
synchronous calls) or CUDA torch tensors (device pointers, asynchronous on the solver's
stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ADSCL_OK, ADSCL_EINVAL, ADSCL_ENOMEM, ADSCL_ECUDA, ADSCL_ETIMEOUT, ADSCL_ENONFINITE, \
    ADSCL_EUNSUPPORTED, ADSCL_ECAPACITY = range(8)
RUNNING, DONE, COLLAPSED, NONFINITE, TIMEOUT = range(5)
PREC_FP64, PREC_BF16X3, PREC_TF32X3 = range(3)
SCHEME_RK4, SCHEME_EVOLVED_A_RK3, SCHEME_EVOLVED_A_RK2, SCHEME_FIXED_METRIC_RK3 = range(4)

STATUS_NAMES = {0: "ADSCL_OK", 1: "ADSCL_EINVAL", 2: "ADSCL_ENOMEM", 3: "ADSCL_ECUDA",
                4: "ADSCL_ETIMEOUT", 5: "ADSCL_ENONFINITE", 6: "ADSCL_EUNSUPPORTED",
                7: "ADSCL_ECAPACITY"}
NOALLOC_MAX_INSTANCES, NOALLOC_MAX_POINTS = 64, 65552


class adscl_config(ctypes.Structure):
    _fields_ = [("num_instances", ctypes.c_int32),
                ("N", ctypes.POINTER(ctypes.c_int32)),
                ("cfl", ctypes.c_double),
                ("ko_sigma", ctypes.c_double),
                ("collapse_threshold", ctypes.c_double),
                ("out_dt", ctypes.c_double),
                ("spec_J", ctypes.c_int32),
                ("ckpt_every", ctypes.c_int32),
                ("max_device_iters", ctypes.c_int64),
                ("device", ctypes.c_int32),
                ("one_per_launch", ctypes.c_int32),
                ("chunk_steps", ctypes.c_int32),
                ("direct_launch", ctypes.c_int32),
                ("scheme", ctypes.c_int32),
                ("a_reint_every", ctypes.c_int32),
                ("adjoint_ctas", ctypes.c_int32),
                ("adjoint_stage_buffers", ctypes.c_int32),
                ("stream", ctypes.c_void_p),
                ("spectrum_chunks", ctypes.c_int32)]


# exported symbols and their signatures (kept in one table so tests can check the .so)
_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_I32, _I64, _F = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "adscl_max_points": ([], _I32),
    "adscl_create": ([ctypes.POINTER(adscl_config), ctypes.POINTER(_VP)], ctypes.c_int),
    "adscl_set_initial": ([_VP, _VP, _VP, ctypes.c_int], ctypes.c_int),
    "adscl_set_initial_modes": ([_VP, _VP, _I32, ctypes.c_int], ctypes.c_int),
    "adscl_evolve": ([_VP, _F, _VP, _VP, _VP, _VP, ctypes.c_int], ctypes.c_int),
    "adscl_evolve_wide": ([_VP, _F, _VP, _VP, _VP, _VP, ctypes.c_int], ctypes.c_int),
    "adscl_spectrum": ([_VP, _I32, ctypes.c_int, _VP, ctypes.c_int], ctypes.c_int),
    "adscl_ttf": ([_VP, _I32, ctypes.c_int, _VP, _VP, ctypes.c_int], ctypes.c_int),
    "adscl_track": ([_VP, _F, _F, _I32, _I32, ctypes.c_int, _VP, _VP, _VP, ctypes.c_int], ctypes.c_int),
    "adscl_grad": ([_VP, _VP, _I32, _F, _VP, _VP, ctypes.c_int], ctypes.c_int),
    "adscl_get_state": ([_VP, _I32, _VP, _VP, _VP, _VP, ctypes.c_int], ctypes.c_int),
    "adscl_set_state": ([_VP, _I32, _VP, _VP, _I64], ctypes.c_int),
    "adscl_get_clock": ([_VP, _VP, _VP], ctypes.c_int),
    "adscl_adjoint_storage": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "adscl_launch_count": ([_VP], _I64),
    "adscl_autotune": ([_VP, _I32], ctypes.c_int),
    "adscl_get_shape": ([_VP, _I32, _VP, _VP, _VP], ctypes.c_int),
    "adscl_set_shape": ([_VP, _I32, _I32, _I32, _I32], ctypes.c_int),
    "adscl_probe_fp64": ([_I32, _VP, _VP], ctypes.c_int),
    "adscl_exp_neg": ([_I32, _VP, _VP, _I64], ctypes.c_int),
    "adscl_exp_neg_scaled": ([_I32, _VP, _VP, _I64], ctypes.c_int),
    "adscl_evolve_noalloc": ([_I32, _VP, _I32, _I32, _VP, _VP, _F, _F, _F, _F, _VP, _VP, _VP, _VP],
                             ctypes.c_int),
    "adscl_last_error": ([_VP], ctypes.c_char_p),
    "adscl_destroy": ([_VP], None),
}

_lib = None


def load(path: str | None = None):
    """Load libadscl.so (building it first if the sources are newer).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path) or _build.needs_build():
        try:
            _build.build()
        except Exception as e:  # noqa: BLE001 - reported with the cause below
            if not os.path.exists(path):
                raise RuntimeError(f"libadscl.so is not built and nvcc failed: {e}") from e
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def probe_fp64(device=0, stream=None):
    """Measured FP64 TFLOP/s of the device (FMA = 2 flops)."""
    lib = load()
    out = ctypes.c_double()
    st = lib.adscl_probe_fp64(device, stream, ctypes.byref(out))
    if st != ADSCL_OK:
        raise AdsclError(st, "FP64 probe failed")
    return out.value


def exp_neg(x, device=0):
    """The solver's e^{-x} on a host array (verification of the library's exp)."""
    lib = load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    st = lib.adscl_exp_neg(device, x.ctypes.data, y.ctypes.data, x.size)
    if st != ADSCL_OK:
        raise AdsclError(st, "exp_neg failed")
    return y


def exp_neg_scaled(X, device=0):
    """The solver's e^{-X ln2/256} (argument in units of ln2/256, as the kernels use it) on a
    host array."""
    lib = load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.empty_like(X)
    st = lib.adscl_exp_neg_scaled(device, X.ctypes.data, y.ctypes.data, X.size)
    if st != ADSCL_OK:
        raise AdsclError(st, "exp_neg_scaled failed")
    return y


def evolve_noalloc(Phi, Pi, N, t_end, t_reached, t_collapse, mass, status, cfl=0.5,
                   ko_sigma=0.5, collapse_threshold=2.0 ** -7, device=0, stream=None):
    """adscl_evolve_noalloc on CUDA torch tensors that the caller allocated: Phi, Pi (packed
    B x N, updated in place) and the four length-B outputs.  Asynchronous on `stream`; returns
    the status code (no exception, so that the capacity limit can be probed)."""
    lib = load()
    B = Phi.numel() // N
    return lib.adscl_evolve_noalloc(device, stream, B, N, Phi.data_ptr(), Pi.data_ptr(),
                                    float(t_end), cfl, ko_sigma, collapse_threshold,
                                    t_reached.data_ptr(), t_collapse.data_ptr(), mass.data_ptr(),
                                    status.data_ptr())


class AdsclError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(x):
    """(address, is_device) of a numpy array or a torch tensor; None -> (None, None)."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data, 0
    # torch tensor
    assert x.is_contiguous()
    return x.data_ptr(), 1 if x.is_cuda else 0


class Solver:
    """One adscl context: a batch of instances with grid sizes N[b]."""

    def __init__(self, N, cfl=0.5, ko_sigma=0.5, collapse_threshold=2.0 ** -7, out_dt=1.0,
                 spec_J=64, ckpt_every=256, device=0, one_per_launch=False, stream=None,
                 max_device_iters=0, chunk_steps=0, direct_launch=False, scheme=0,
                 a_reint_every=0, adjoint_ctas=0, adjoint_stage_buffers=0, spectrum_chunks=0):
        self.lib = load()
        self.N = np.ascontiguousarray(np.asarray(N, dtype=np.int32).ravel())
        self.B = int(self.N.size)
        self.offsets = np.concatenate([[0], np.cumsum(self.N.astype(np.int64))])
        cfg = adscl_config()
        cfg.num_instances = self.B
        cfg.N = self.N.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        cfg.cfl = cfl
        cfg.ko_sigma = ko_sigma
        cfg.collapse_threshold = collapse_threshold
        cfg.out_dt = out_dt
        cfg.spec_J = spec_J
        cfg.ckpt_every = ckpt_every
        cfg.max_device_iters = max_device_iters
        cfg.device = device
        cfg.one_per_launch = 1 if one_per_launch else 0
        cfg.chunk_steps = chunk_steps
        cfg.direct_launch = 1 if direct_launch else 0
        cfg.scheme = scheme
        cfg.a_reint_every = a_reint_every
        cfg.adjoint_ctas = adjoint_ctas
        cfg.adjoint_stage_buffers = adjoint_stage_buffers
        cfg.stream = stream
        cfg.spectrum_chunks = spectrum_chunks
        self.stream = stream
        h = ctypes.c_void_p()
        st = self.lib.adscl_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != ADSCL_OK:
            msg = self.lib.adscl_last_error(h).decode() if h.value else "invalid configuration"
            if h.value:
                self.lib.adscl_destroy(h)
            raise AdsclError(st, msg)
        self.ctx = h

    # -- helpers
    def _check(self, st):
        if st != ADSCL_OK:
            raise AdsclError(st, self.lib.adscl_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.adscl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    @property
    def total(self):
        return int(self.offsets[-1])

    # -- API
    def set_initial(self, Phi, Pi):
        p, dev = _ptr(Phi)
        q, _ = _ptr(Pi)
        self._check(self.lib.adscl_set_initial(self.ctx, p, q, dev))

    def set_initial_modes(self, a):
        p, dev = _ptr(a)
        K = a.shape[-1]
        self._check(self.lib.adscl_set_initial_modes(self.ctx, p, K, dev))

    def evolve(self, t_end, out=None):
        """Evolve to t_end.  out: optional (t_reached, t_collapse, mass, status) buffers (torch
        CUDA tensors for an asynchronous call); otherwise numpy arrays are returned."""
        if out is None:
            tr, tc, m = np.empty(self.B), np.empty(self.B), np.empty(self.B)
            s = np.empty(self.B, dtype=np.int32)
            self._check(self.lib.adscl_evolve(self.ctx, float(t_end), tr.ctypes.data, tc.ctypes.data,
                                              m.ctypes.data, s.ctypes.data, 0))
            return tr, tc, m, s
        ptrs = [_ptr(x)[0] for x in out]
        dev = _ptr(out[0])[1]
        self._check(self.lib.adscl_evolve(self.ctx, float(t_end), *ptrs, dev))
        return out

    def evolve_wide(self, t_end, out=None):
        """adscl_evolve_wide: evolve the context's single fixed-metric instance to t_end on the
        whole GPU (one cooperative launch, a grid-wide barrier per stage).  Same outputs as
        evolve."""
        if out is None:
            tr, tc, m = np.empty(self.B), np.empty(self.B), np.empty(self.B)
            s = np.empty(self.B, dtype=np.int32)
            self._check(self.lib.adscl_evolve_wide(self.ctx, float(t_end), tr.ctypes.data, tc.ctypes.data,
                                                   m.ctypes.data, s.ctypes.data, 0))
            return tr, tc, m, s
        ptrs = [_ptr(x)[0] for x in out]
        dev = _ptr(out[0])[1]
        self._check(self.lib.adscl_evolve_wide(self.ctx, float(t_end), *ptrs, dev))
        return out

    def get_state(self, inst):
        n = int(self.N[inst])
        Phi, Pi, A, dl = (np.empty(n) for _ in range(4))
        self._check(self.lib.adscl_get_state(self.ctx, inst, Phi.ctypes.data, Pi.ctypes.data,
                                             A.ctypes.data, dl.ctypes.data, 0))
        return Phi, Pi, A, dl

    def set_state(self, inst, Phi, Pi, step):
        Phi = np.ascontiguousarray(Phi, dtype=np.float64)
        Pi = np.ascontiguousarray(Pi, dtype=np.float64)
        self._check(self.lib.adscl_set_state(self.ctx, inst, Phi.ctypes.data, Pi.ctypes.data, int(step)))

    def clock(self):
        dt = np.empty(self.B)
        step = np.empty(self.B, dtype=np.int64)
        self._check(self.lib.adscl_get_clock(self.ctx, dt.ctypes.data, step.ctypes.data))
        return dt, step

    def adjoint_storage(self):
        """(bytes, buffers, segments, recomputed) of the stage storage (adscl_adjoint_storage)."""
        by, nb = ctypes.c_int64(), ctypes.c_int32()
        ns, nr = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.adscl_adjoint_storage(self.ctx, ctypes.byref(by), ctypes.byref(nb),
                                                   ctypes.byref(ns), ctypes.byref(nr)))
        return by.value, nb.value, ns.value, nr.value

    def spectrum(self, J=64, precision=PREC_FP64):
        E = np.empty((self.B, J))
        self._check(self.lib.adscl_spectrum(self.ctx, J, precision, E.ctypes.data, 0))
        return E

    def ttf(self, J=64, precision=PREC_FP64, with_energies=False):
        """(E, N, T) per instance (B x 3): total energy, particle number and temperature of the
        current slices (adscl_ttf); with_energies also returns the mode energies (B x J)."""
        q = np.empty((self.B, 3))
        E = np.empty((self.B, J)) if with_energies else None
        self._check(self.lib.adscl_ttf(self.ctx, J, precision, q.ctypes.data,
                                       E.ctypes.data if E is not None else None, 0))
        return (q, E) if with_energies else q

    def track(self, t_first, cadence, n_snap, J=64, precision=PREC_FP64, energies=False):
        """Evolve to t_first + k cadence, k < n_snap, with the spectrum and the TTF quantities of
        every slice reached (adscl_track).  Returns (t_hist (n_snap x B), ttf_hist
        (n_snap x B x 3), E_hist (n_snap x B x J) or None)."""
        th = np.empty((n_snap, self.B))
        qh = np.empty((n_snap, self.B, 3))
        Eh = np.empty((n_snap, self.B, J)) if energies else None
        self._check(self.lib.adscl_track(self.ctx, float(t_first), float(cadence), int(n_snap), J,
                                         precision, th.ctypes.data, qh.ctypes.data,
                                         Eh.ctypes.data if Eh is not None else None, 0))
        return th, qh, Eh

    def grad(self, a, T):
        """(J, dJ/da) of J = sum_{j<spec_J} (E_j(T) - E_j(0))^2 for Pi(x,0) = sum_k a_k e_k."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        K = a.shape[-1]
        J = np.empty(self.B)
        g = np.empty((self.B, K))
        self._check(self.lib.adscl_grad(self.ctx, a.ctypes.data, K, float(T), J.ctypes.data,
                                        g.ctypes.data, 0))
        return J, g

    def launch_count(self):
        return int(self.lib.adscl_launch_count(self.ctx))

    # -- kernel shapes and the autotuner
    def autotune(self, trial_steps=8):
        """Pick the fastest kernel shape for every grid size (state unchanged); returns
        {N: (P, NT, CL)}.  Cached per batch signature and number of running instances: calling
        it again after collapses have thinned the batch re-tunes (adscl_autotune)."""
        self._check(self.lib.adscl_autotune(self.ctx, int(trial_steps)))
        return self.shapes()

    def shape(self, inst):
        v = [ctypes.c_int32() for _ in range(3)]
        self._check(self.lib.adscl_get_shape(self.ctx, int(inst), *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def shapes(self):
        return {int(n): self.shape(int(np.argmax(self.N == n))) for n in np.unique(self.N)}

    def set_shape(self, N, P, NT, CL):
        self._check(self.lib.adscl_set_shape(self.ctx, int(N), int(P), int(NT), int(CL)))

    def apply_shapes(self, table):
        """Apply {N: (P, NT, CL)} (e.g. a saved autotune() result; JSON keys may be strings)
        to the grid sizes of this context that appear in it."""
        present = set(int(n) for n in self.N)
        for n, shp in table.items():
            if int(n) in present:
                self.set_shape(int(n), *shp)
