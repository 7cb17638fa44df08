"""Python binding of the FP64 CPU oracle (``teuk_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, independent CPU
implementation of the time-domain Teukolsky solver (two-step Lax-Wendroff,
Eqs. 3-4 of arXiv:1206.0270).  Only the test-suite, the package smoke check
and the benchmark's CPU-baseline / reference legs may import this module.  It
shares no code with the CUDA path and never imports the product package.

Arrays of complex values are numpy ``complex128`` of shape (nr, nth), theta
fastest, which is the interleaved (re, im) layout the C code reads.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "teuk_oracle.c")
_LIB = os.path.join(_HERE, "libteuk_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            vp = C.c_void_p
            L.oracle_rstar_of_r.restype = C.c_double
            L.oracle_rstar_of_r.argtypes = [C.c_double, C.c_double]
            L.oracle_r_of_rstar.restype = None
            L.oracle_r_of_rstar.argtypes = [C.c_double, C.c_double, dp, dp]
            L.oracle_coefficients.restype = None
            L.oracle_coefficients.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double,
                                              C.c_int, C.c_int, dp]
            L.oracle_orbit_omega.restype = C.c_double
            L.oracle_orbit_omega.argtypes = [C.c_double, C.c_double, C.c_int]
            L.oracle_angular_op.restype = None
            L.oracle_angular_op.argtypes = [C.c_int, C.c_int, dp, dp]
            L.oracle_lw_step_generic.restype = None
            L.oracle_lw_step_generic.argtypes = ([C.c_int, C.c_int, C.c_int, C.c_double, C.c_double]
                                                 + [dp] * 13 + [C.c_double] * 5 + [dp] * 4)
            L.oracle_set_dissipation.restype = C.c_int
            L.oracle_set_dissipation.argtypes = [vp, C.c_double]
            L.oracle_create.restype = vp
            L.oracle_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_int, C.c_int]
            L.oracle_destroy.restype = None
            L.oracle_destroy.argtypes = [vp]
            L.oracle_set_initial.restype = C.c_int
            L.oracle_set_initial.argtypes = [vp, dp, dp]
            L.oracle_set_source.restype = C.c_int
            L.oracle_set_source.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_int]
            L.oracle_clear_source.restype = None
            L.oracle_clear_source.argtypes = [vp]
            L.oracle_set_extraction.restype = C.c_int
            L.oracle_set_extraction.argtypes = [vp, C.c_double, C.c_int]
            L.oracle_step.restype = C.c_int
            L.oracle_step.argtypes = [vp, C.c_long]
            L.oracle_num_samples.restype = C.c_long
            L.oracle_num_samples.argtypes = [vp]
            L.oracle_step_count.restype = C.c_long
            L.oracle_step_count.argtypes = [vp]
            L.oracle_get_samples.restype = C.c_long
            L.oracle_get_samples.argtypes = [vp, dp, dp, C.c_long]
            L.oracle_get_state.restype = C.c_int
            L.oracle_get_state.argtypes = [vp, dp, dp]
            L.oracle_get_coefficients.restype = C.c_int
            L.oracle_get_coefficients.argtypes = [vp, C.c_int, dp]
            L.oracle_get_source_profile.restype = C.c_int
            L.oracle_get_source_profile.argtypes = [vp, C.c_int, dp]
            L.oracle_stable_dt.restype = C.c_double
            L.oracle_stable_dt.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                           C.c_int, C.c_int, C.c_double, C.c_double]
            _lib = L
    return _lib


def _p(x):
    if x is None:
        return None
    assert x.flags["C_CONTIGUOUS"]
    return x.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------------------
# Pointwise functions
# ---------------------------------------------------------------------------

def rstar_of_r(r: float, a: float) -> float:
    return lib().oracle_rstar_of_r(float(r), float(a))


def r_of_rstar(rstar: float, a: float):
    r = C.c_double()
    D = C.c_double()
    lib().oracle_r_of_rstar(float(rstar), float(a), C.byref(r), C.byref(D))
    return r.value, D.value


def coefficients(r: float, Delta: float, theta: float, a: float, s: int, m: int) -> dict:
    out = np.zeros(8)
    lib().oracle_coefficients(float(r), float(Delta), float(theta), float(a), int(s), int(m), _p(out))
    return dict(b=out[0], d=out[1] + 1j * out[2], ct=out[3] + 1j * out[4],
                W=out[5] + 1j * out[6], kappa=out[7])


def orbit_omega(r0: float, a: float, prograde: bool = True) -> float:
    return lib().oracle_orbit_omega(float(r0), float(a), 1 if prograde else 0)


def angular_op(row: np.ndarray, parity: int) -> np.ndarray:
    row = np.ascontiguousarray(row, dtype=np.complex128)
    out = np.zeros_like(row)
    lib().oracle_angular_op(row.size, int(parity), _p(row.view(np.float64)), _p(out.view(np.float64)))
    return out


def stable_dt(nr, nth, rstar_min, rstar_max, a, s, m, c_r=0.5, c_theta=0.1) -> float:
    return lib().oracle_stable_dt(int(nr), int(nth), float(rstar_min), float(rstar_max), float(a),
                                  int(s), int(m), float(c_r), float(c_theta))


def lw_step_generic(Phi, Pi, *, h, dt, parity, b_node, b_mid, d_node, d_mid, ct_node, ct_mid,
                    W_node, W_mid, kap_node, kap_mid, cot, G_node=None, G_mid=None,
                    phase_n=0j, phase_half=0j, eps=0.0):
    """One Lax-Wendroff step with caller-supplied coefficient fields and
    Kreiss-Oliger strength eps."""
    nr, nth = Phi.shape
    f = lambda x, dt_=np.float64: np.ascontiguousarray(x, dtype=dt_)
    c = lambda x: f(x, np.complex128).view(np.float64)
    Phi = f(Phi, np.complex128)
    Pi = f(Pi, np.complex128)
    Po = np.zeros_like(Phi)
    Qo = np.zeros_like(Pi)
    args = [f(b_node), f(b_mid), c(d_node), c(d_mid), c(ct_node), c(ct_mid), c(W_node), c(W_mid),
            f(kap_node), f(kap_mid), f(cot)]
    Gn = None if G_node is None else f(G_node)
    Gm = None if G_mid is None else f(G_mid)
    lib().oracle_lw_step_generic(nr, nth, int(parity), float(h), float(dt), *[_p(a) for a in args],
                                 _p(Gn), _p(Gm), phase_n.real, phase_n.imag, phase_half.real,
                                 phase_half.imag, float(eps), _p(Phi.view(np.float64)), _p(Pi.view(np.float64)),
                                 _p(Po.view(np.float64)), _p(Qo.view(np.float64)))
    return Po, Qo


# ---------------------------------------------------------------------------
# Solver
# ---------------------------------------------------------------------------

class Solver:
    """One (a, s, m) evolution on an nr x nth grid with time step dt."""

    def __init__(self, nr, nth, rstar_min, rstar_max, dt, a, s, m):
        self.nr, self.nth = int(nr), int(nth)
        self.rstar_min, self.rstar_max = float(rstar_min), float(rstar_max)
        self.dt, self.a, self.s, self.m = float(dt), float(a), int(s), int(m)
        self._h = lib().oracle_create(self.nr, self.nth, self.rstar_min, self.rstar_max,
                                      self.dt, self.a, self.s, self.m)
        if not self._h:
            raise ValueError("oracle_create: bad argument")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_destroy(h)
            self._h = None

    def set_initial(self, phi, pi=None):
        phi = np.ascontiguousarray(phi, dtype=np.complex128)
        assert phi.shape == (self.nr, self.nth)
        if pi is not None:
            pi = np.ascontiguousarray(pi, dtype=np.complex128)
            assert pi.shape == (self.nr, self.nth)
        lib().oracle_set_initial(self._h, _p(phi.view(np.float64)),
                                 None if pi is None else _p(pi.view(np.float64)))

    def set_source(self, r0, sigma, amplitude=1.0, prograde=True):
        rc = lib().oracle_set_source(self._h, float(r0), float(sigma), float(amplitude),
                                     1 if prograde else 0)
        if rc:
            raise ValueError("oracle_set_source: bad argument")

    def set_dissipation(self, eps):
        if lib().oracle_set_dissipation(self._h, float(eps)):
            raise ValueError("oracle_set_dissipation: eps outside [0, 2)")

    def clear_source(self):
        lib().oracle_clear_source(self._h)

    def set_extraction(self, rstar_ext, every):
        if lib().oracle_set_extraction(self._h, float(rstar_ext), int(every)):
            raise ValueError("oracle_set_extraction: bad argument")

    def step(self, n):
        lib().oracle_step(self._h, int(n))

    @property
    def step_count(self):
        return lib().oracle_step_count(self._h)

    def samples(self):
        n = lib().oracle_num_samples(self._h)
        t = np.zeros(n)
        phi = np.zeros((n, self.nth), dtype=np.complex128)
        lib().oracle_get_samples(self._h, _p(t), _p(phi.view(np.float64)), n)
        return t, phi

    def state(self):
        phi = np.zeros((self.nr, self.nth), dtype=np.complex128)
        pi = np.zeros_like(phi)
        lib().oracle_get_state(self._h, _p(phi.view(np.float64)), _p(pi.view(np.float64)))
        return phi, pi

    def coefficient_fields(self, mid=False):
        rows = self.nr - 1 if mid else self.nr
        out = np.zeros((rows, self.nth, 8))
        lib().oracle_get_coefficients(self._h, 1 if mid else 0, _p(out))
        return dict(b=out[..., 0], d=out[..., 1] + 1j * out[..., 2], ct=out[..., 3] + 1j * out[..., 4],
                    W=out[..., 5] + 1j * out[..., 6], kappa=out[..., 7])

    def source_profile(self, mid=False):
        rows = self.nr - 1 if mid else self.nr
        out = np.zeros((rows, self.nth))
        lib().oracle_get_source_profile(self._h, 1 if mid else 0, _p(out))
        return out
