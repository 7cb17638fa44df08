"""Thin Python binding of libteuk.so (the C ABI declared in include/teuk.h).

Argument marshalling only: every step of the time evolution runs in the CUDA
kernels of the library.  The functions keep the C names (teuk_create,
teuk_set_initial, teuk_set_source, teuk_set_extraction, teuk_step,
teuk_extract, ...); ``Solver`` wraps one handle with numpy in/out.  Streams
may be given as a ``torch.cuda.Stream`` or a raw ``cudaStream_t`` integer.

If libteuk.so is missing this module raises at import time: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libteuk.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libteuk.so not found at %s: build it with `python -m paper_1206_0270_gb300.build` "
        "(the solver has no CPU fallback)" % LIB_PATH)

_lib = C.CDLL(LIB_PATH)

TEUK_OK = 0
TEUK_OPT_PDL = 1
TEUK_OPT_GRAPH_CHUNK = 2
TEUK_OPT_BLOCK_THREADS = 3
TEUK_OPT_REAL_PATH = 4
TEUK_OPT_SPLIT_ROWS = 5
TEUK_OPT_BATCH_MODE = 6
TEUK_OPT_FIXED_POINT = 7
TEUK_OPT_BATCH_CTAS = 8
BATCH_FORMS = ("per-job launches", "multi-job launches, one CTA per tile",
               "multi-job launches, one CTA per tile, 64-thread tiles", "persistent multi-job launches")
ERRORS = {-1: "TEUK_ERR_BAD_ARG", -2: "TEUK_ERR_OOM", -3: "TEUK_ERR_CUDA", -4: "TEUK_ERR_NONFINITE",
          -5: "TEUK_ERR_STATE", -6: "TEUK_ERR_OVERFLOW"}


class teuk_grid(C.Structure):
    _fields_ = [("nr", C.c_int), ("nth", C.c_int), ("rstar_min", C.c_double),
                ("rstar_max", C.c_double), ("dt", C.c_double)]


class teuk_orbit(C.Structure):
    _fields_ = [("r0", C.c_double), ("sigma", C.c_double), ("amplitude", C.c_double),
                ("prograde", C.c_int)]


_dp = C.POINTER(C.c_double)
_vp = C.c_void_p
_SIGS = {
    "teuk_stable_dt": (C.c_int, [C.POINTER(teuk_grid), C.c_double, C.c_int, C.c_int, C.c_double,
                                 C.c_double, _dp]),
    "teuk_create": (C.c_int, [C.POINTER(teuk_grid), C.c_double, C.c_int, C.c_int, _vp, C.POINTER(_vp)]),
    "teuk_destroy": (C.c_int, [_vp]),
    "teuk_set_initial": (C.c_int, [_vp, _dp, _dp]),
    "teuk_set_initial_device": (C.c_int, [_vp, _vp, _vp]),
    "teuk_set_state": (C.c_int, [_vp, _dp, _dp, C.c_long]),
    "teuk_set_source": (C.c_int, [_vp, C.POINTER(teuk_orbit)]),
    "teuk_set_extraction": (C.c_int, [_vp, C.c_double, C.c_int, C.c_long]),
    "teuk_step": (C.c_int, [_vp, C.c_long]),
    "teuk_set_dissipation": (C.c_int, [_vp, C.c_double]),
    "teuk_set_stream": (C.c_int, [_vp, _vp]),
    "teuk_extract": (C.c_int, [_vp, _dp, _dp, C.c_long, C.POINTER(C.c_long)]),
    "teuk_get_state": (C.c_int, [_vp, _dp, _dp]),
    "teuk_get_state_device": (C.c_int, [_vp, _vp, _vp]),
    "teuk_step_count": (C.c_long, [_vp]),
    "teuk_check_finite": (C.c_int, [_vp, C.POINTER(C.c_int)]),
    "teuk_set_kernel": (C.c_int, [_vp, C.c_int]),
    "teuk_launches_for": (C.c_long, [_vp, C.c_long]),
    "teuk_set_launch": (C.c_int, [_vp, C.c_int]),
    "teuk_get_launch": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "teuk_step_noalloc": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_long]),
    "teuk_set_option": (C.c_int, [_vp, C.c_int, C.c_long]),
    "teuk_time_kernels": (C.c_int, [_vp, C.c_long, _dp]),
    "teuk_fixed_dot": (C.c_int, [C.c_int, C.c_int, C.c_long, _dp, _dp, C.POINTER(C.c_uint), _dp,
                                 C.POINTER(C.c_int)]),
    "teuk_fixed_d6": (C.c_int, [C.c_int, C.c_long, _dp, _dp]),
    "teuk_batch_create": (C.c_int, [_vp, C.POINTER(_vp)]),
    "teuk_batch_add": (C.c_int, [_vp, _vp, C.c_long, C.POINTER(C.c_int)]),
    "teuk_batch_remove": (C.c_int, [_vp, C.c_int]),
    "teuk_batch_step": (C.c_int, [_vp, C.c_long, C.POINTER(C.c_long)]),
    "teuk_batch_remaining": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_long)]),
    "teuk_batch_sync": (C.c_int, [_vp]),
    "teuk_batch_set_option": (C.c_int, [_vp, C.c_int, C.c_long]),
    "teuk_batch_autotune": (C.c_int, [_vp, C.POINTER(C.c_int)]),
    "teuk_batch_launches_for": (C.c_long, [_vp, C.c_long]),
    "teuk_batch_last_error": (C.c_char_p, [_vp]),
    "teuk_batch_destroy": (C.c_int, [_vp]),
    "teuk_last_error": (C.c_char_p, [_vp]),
    "teuk_strerror": (C.c_char_p, [C.c_int]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = tuple(_SIGS)


class TeukError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


def _check(rc, handle=None, what=""):
    if rc != TEUK_OK:
        msg = teuk_last_error(handle).decode() if handle else teuk_strerror(rc).decode()
        raise TeukError(rc, "%s: %s" % (what, msg))
    return rc


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def fixed_dot(c, x, flip=None, device=False):
    """Fixed-point sums of the Pi rows (teuk_fixed_dot): c, x of shape
    (count, nterms) float64, flip the same shape (0/1, default 0).  Returns
    (out float64 (count,), ok bool (count,)); device=True runs the device
    build of the arithmetic."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    if c.ndim != 2 or c.shape != x.shape:
        raise ValueError("c and x must have the same shape (count, nterms)")
    fl = np.zeros(c.shape, np.uint32) if flip is None else np.ascontiguousarray(flip, dtype=np.uint32)
    if fl.shape != c.shape:
        raise ValueError("flip must have the shape of c")
    out = np.zeros(c.shape[0])
    ok = np.zeros(c.shape[0], np.int32)
    rc = teuk_fixed_dot(1 if device else 0, c.shape[1], c.shape[0], c.ctypes.data_as(_dp), x.ctypes.data_as(_dp),
                        fl.ctypes.data_as(C.POINTER(C.c_uint)), out.ctypes.data_as(_dp),
                        ok.ctypes.data_as(C.POINTER(C.c_int)))
    _check(rc, None, "teuk_fixed_dot")
    return out, ok.astype(bool)


def fixed_d6(u, device=False):
    """Exact sixth differences of the angular dissipation (teuk_fixed_d6):
    u of shape (count, 7) float64, u[i, q] = u_{j-3+q}.  Returns out float64
    (count,); device=True runs the device build of the arithmetic."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    if u.ndim != 2 or u.shape[1] != 7:
        raise ValueError("u must have shape (count, 7)")
    out = np.zeros(u.shape[0])
    rc = teuk_fixed_d6(1 if device else 0, u.shape[0], u.ctypes.data_as(_dp), out.ctypes.data_as(_dp))
    _check(rc, None, "teuk_fixed_d6")
    return out


def stable_dt(nr, nth, rstar_min, rstar_max, a, s, m, c_r=0.5, c_theta=0.1):
    g = teuk_grid(int(nr), int(nth), float(rstar_min), float(rstar_max), 0.0)
    out = C.c_double()
    _check(teuk_stable_dt(C.byref(g), float(a), int(s), int(m), float(c_r), float(c_theta),
                          C.byref(out)), what="teuk_stable_dt")
    return out.value


class Solver:
    """One (a, s, m) evolution; fields are numpy complex128 arrays (nr, nth)."""

    def __init__(self, nr, nth, rstar_min, rstar_max, dt, a, s, m, stream=None, kernel=None):
        self.nr, self.nth = int(nr), int(nth)
        self.grid = teuk_grid(self.nr, self.nth, float(rstar_min), float(rstar_max), float(dt))
        self.dt = float(dt)
        h = _vp()
        _check(teuk_create(C.byref(self.grid), float(a), int(s), int(m), _stream_handle(stream),
                           C.byref(h)), what="teuk_create")
        self.h = h
        self._stream = stream  # keeps a caller's stream object alive as long as the handle uses it
        if kernel is not None:
            self.set_kernel(kernel)

    def close(self):
        if getattr(self, "h", None):
            teuk_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_kernel(self, variant):
        _check(teuk_set_kernel(self.h, int(variant)), self.h, "teuk_set_kernel")

    def set_initial(self, phi, pi=None):
        phi = np.ascontiguousarray(phi, dtype=np.complex128)
        assert phi.shape == (self.nr, self.nth)
        if pi is not None:
            pi = np.ascontiguousarray(pi, dtype=np.complex128)
            assert pi.shape == (self.nr, self.nth)
        _check(teuk_set_initial(self.h, _ptr(phi.view(np.float64)),
                                None if pi is None else _ptr(pi.view(np.float64))), self.h,
               "teuk_set_initial")

    def set_state(self, phi, pi, step):
        phi = np.ascontiguousarray(phi, dtype=np.complex128)
        pi = np.ascontiguousarray(pi, dtype=np.complex128)
        assert phi.shape == pi.shape == (self.nr, self.nth)
        _check(teuk_set_state(self.h, _ptr(phi.view(np.float64)), _ptr(pi.view(np.float64)), int(step)),
               self.h, "teuk_set_state")

    def set_initial_device(self, phi_ptr, pi_ptr=None):
        _check(teuk_set_initial_device(self.h, phi_ptr, pi_ptr), self.h, "teuk_set_initial_device")

    def set_source(self, r0=None, sigma=0.05, amplitude=1.0, prograde=True):
        if r0 is None:
            _check(teuk_set_source(self.h, None), self.h, "teuk_set_source")
            return
        o = teuk_orbit(float(r0), float(sigma), float(amplitude), 1 if prograde else 0)
        _check(teuk_set_source(self.h, C.byref(o)), self.h, "teuk_set_source")

    def set_extraction(self, rstar_ext, every, capacity=4096):
        _check(teuk_set_extraction(self.h, float(rstar_ext), int(every), int(capacity)), self.h,
               "teuk_set_extraction")

    def step(self, n):
        _check(teuk_step(self.h, int(n)), self.h, "teuk_step")

    def set_stream(self, stream=None):
        """Run future work on `stream` (torch.cuda.Stream, a raw handle, or None
        for a stream of the handle's own); waits for the current stream."""
        _check(teuk_set_stream(self.h, _stream_handle(stream)), self.h, "teuk_set_stream")
        self._stream = stream

    @property
    def step_count(self):
        return teuk_step_count(self.h)

    def extract(self, cap=1 << 20):
        t = np.zeros(cap)
        phi = np.zeros((cap, self.nth), dtype=np.complex128)
        n = C.c_long()
        rc = teuk_extract(self.h, _ptr(t), _ptr(phi.view(np.float64)), int(cap), C.byref(n))
        _check(rc, self.h, "teuk_extract")
        return t[:n.value].copy(), phi[:n.value].copy()

    def state(self):
        phi = np.zeros((self.nr, self.nth), dtype=np.complex128)
        pi = np.zeros_like(phi)
        _check(teuk_get_state(self.h, _ptr(phi.view(np.float64)), _ptr(pi.view(np.float64))), self.h,
               "teuk_get_state")
        return phi, pi

    def state_device(self, phi_ptr, pi_ptr):
        _check(teuk_get_state_device(self.h, phi_ptr, pi_ptr), self.h, "teuk_get_state_device")

    def check_finite(self):
        f = C.c_int()
        rc = teuk_check_finite(self.h, C.byref(f))
        if rc not in (TEUK_OK, -4):
            _check(rc, self.h, "teuk_check_finite")
        return bool(f.value)

    def set_option(self, option, value):
        _check(teuk_set_option(self.h, int(option), int(value)), self.h, "teuk_set_option")

    def set_dissipation(self, eps):
        _check(teuk_set_dissipation(self.h, float(eps)), self.h, "teuk_set_dissipation")

    def set_launch(self, rows_per_block):
        _check(teuk_set_launch(self.h, int(rows_per_block)), self.h, "teuk_set_launch")

    def launch_shape(self):
        r, b = C.c_int(), C.c_int()
        _check(teuk_get_launch(self.h, C.byref(r), C.byref(b)), self.h, "teuk_get_launch")
        return r.value, b.value

    def launches_for(self, n):
        return teuk_launches_for(self.h, int(n))

    def time_kernels(self, n):
        out = np.zeros(2)
        _check(teuk_time_kernels(self.h, int(n), _ptr(out)), self.h, "teuk_time_kernels")
        return float(out[0]), float(out[1])


def _bcheck(rc, b, what):
    if rc != TEUK_OK:
        raise TeukError(rc, "%s: %s" % (what, teuk_batch_last_error(b).decode()))
    return rc


class Batch:
    """Many handles stepped together (teuk_batch_*).  Jobs are Solver objects."""

    def __init__(self, stream=None):
        b = _vp()
        _check(teuk_batch_create(_stream_handle(stream), C.byref(b)), what="teuk_batch_create")
        self.b = b
        self.solvers = {}

    def close(self):
        if getattr(self, "b", None):
            teuk_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add(self, solver, steps):
        jid = C.c_int()
        _bcheck(teuk_batch_add(self.b, solver.h, int(steps), C.byref(jid)), self.b, "teuk_batch_add")
        self.solvers[jid.value] = solver
        return jid.value

    def remove(self, job_id):
        _bcheck(teuk_batch_remove(self.b, int(job_id)), self.b, "teuk_batch_remove")
        self.solvers.pop(job_id, None)

    def step(self, max_steps):
        done = C.c_long()
        _bcheck(teuk_batch_step(self.b, int(max_steps), C.byref(done)), self.b, "teuk_batch_step")
        return done.value

    def remaining(self, job_id):
        r = C.c_long()
        _bcheck(teuk_batch_remaining(self.b, int(job_id), C.byref(r)), self.b, "teuk_batch_remaining")
        return r.value

    def sync(self):
        _bcheck(teuk_batch_sync(self.b), self.b, "teuk_batch_sync")

    def set_option(self, option, value):
        _bcheck(teuk_batch_set_option(self.b, int(option), int(value)), self.b, "teuk_batch_set_option")

    def autotune(self):
        """Time the launch forms and keep the fastest; returns its index in
        BATCH_FORMS."""
        best = C.c_int()
        _bcheck(teuk_batch_autotune(self.b, C.byref(best)), self.b, "teuk_batch_autotune")
        return best.value

    def launches_for(self, n):
        return teuk_batch_launches_for(self.b, int(n))
