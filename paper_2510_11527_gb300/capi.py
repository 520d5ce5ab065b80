"""ctypes binding of libaf (include/af.h): one Python function per C entry point, with
the same name, doing argument marshalling only. Every step of the method runs in the
CUDA library; there is no CPU path. Importing this module loads libaf.so and raises if
it is missing or cannot be loaded.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libaf.so")

AF_OK, AF_E_ARG, AF_E_CUDA, AF_E_OOM, AF_E_STATE, AF_E_CFL, AF_E_TIMEOUT, AF_E_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "AF_OK", -1: "AF_E_ARG", -2: "AF_E_CUDA", -3: "AF_E_OOM", -4: "AF_E_STATE", -5: "AF_E_CFL",
                -6: "AF_E_TIMEOUT", -7: "AF_E_UNSUPPORTED"}
FLUX = {"zero": 0, "linear": 1, "burgers": 2, "bl": 3}
DIFF = {"none": 0, "const": 1, "pwl": 2, "pme": 3, "cubic": 4}
PREC = {"fp64": 0, "fp32_mixed": 1}
BLEND = {"off": 0, "plain": 1, "external": 2}


class AfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class af_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x0", ctypes.c_double),
                ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double)]


class af_flux(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("p", ctypes.c_double * 4)]


class af_diff(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("p", ctypes.c_double * 4)]


class af_bounds_t(ctypes.Structure):
    _fields_ = [("umin", ctypes.c_double), ("umax", ctypes.c_double), ("from_initial_data", ctypes.c_int)]


class af_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("rk", ctypes.c_int), ("cfl", ctypes.c_double),
                ("cfl_diff", ctypes.c_double), ("limiter", ctypes.c_int), ("blend", ctypes.c_int),
                ("gamma", ctypes.c_double)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_V = ctypes.c_void_p


def lib():
    """Load libaf.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libaf.so not built at {LIB_PATH}: run paper_2510_11527_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "af_create": [ctypes.POINTER(af_grid), ctypes.POINTER(af_flux), ctypes.POINTER(af_diff),
                      ctypes.POINTER(af_bounds_t), ctypes.POINTER(af_opts), ctypes.POINTER(_V)],
        "af_destroy": [_V],
        "af_set_stream": [_V, _V],
        "af_set_state": [_V, _D, _D, _D, _D],
        "af_get_state": [_V, _D, _D, _D, _D],
        "af_device_ptrs": [_V, ctypes.POINTER(_V), ctypes.POINTER(ctypes.c_int)],
        "af_set_indicator": [_V, _D],
        "af_set_indicator_device": [_V, _V],
        "af_forward_euler": [_V, ctypes.c_double],
        "af_stage": [_V, ctypes.c_int, ctypes.c_double],
        "af_dt_device": [_V],
        "af_step": [_V, ctypes.c_double, _D],
        "af_run": [_V, ctypes.c_double, ctypes.POINTER(ctypes.c_longlong)],
        "af_time": [_V, _D],
        "af_mass": [_V, _D],
        "af_bounds": [_V, _D, _D],
        "af_dt_cfl": [_V, _D],
        "af_stats": [_V, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), _D],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.af_last_error.argtypes = [_V]
    L.af_last_error.restype = ctypes.c_char_p
    L.af_num_stages.argtypes = [_V]
    L.af_num_stages.restype = ctypes.c_int
    _lib = L
    return L


def exported_symbols():
    """Names of the entry points declared in include/af.h (for the export test)."""
    return ["af_create", "af_destroy", "af_last_error", "af_set_stream", "af_set_state", "af_get_state",
            "af_device_ptrs", "af_set_indicator", "af_set_indicator_device", "af_forward_euler", "af_stage", "af_dt_device",
            "af_num_stages", "af_step", "af_run", "af_time", "af_mass", "af_bounds", "af_dt_cfl", "af_stats"]


def _check(ctx, st):
    if st != AF_OK:
        msg = lib().af_last_error(ctx).decode() if ctx else ""
        raise AfError(st, msg)


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _host(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).ravel()
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


# ---- one function per entry point ----------------------------------------------------

def af_create(grid, flux, diff, bounds, opts):
    ctx = _V()
    st = lib().af_create(ctypes.byref(grid), ctypes.byref(flux), ctypes.byref(diff), ctypes.byref(bounds),
                         ctypes.byref(opts), ctypes.byref(ctx))
    if st != AF_OK:
        raise AfError(st, "af_create failed")
    return ctx


def af_destroy(ctx):
    _check(None, lib().af_destroy(ctx))


def af_set_stream(ctx, stream_handle):
    _check(ctx, lib().af_set_stream(ctx, _V(stream_handle)))


def af_set_state(ctx, n, ub, V, X=None, Y=None):
    arrs = [_host(ub, n), _host(V, n), None if X is None else _host(X, n), None if Y is None else _host(Y, n)]
    _check(ctx, lib().af_set_state(ctx, *[_dp(a) for a in arrs]))


def af_get_state(ctx, n, dim):
    out = [np.empty(n) for _ in range(4 if dim == 2 else 2)] + ([None, None] if dim == 1 else [])
    _check(ctx, lib().af_get_state(ctx, *[_dp(a) for a in out]))
    return [a for a in out if a is not None]


def af_device_ptrs(ctx):
    ptrs = (_V * 4)()
    dt = (ctypes.c_int * 2)()
    _check(ctx, lib().af_device_ptrs(ctx, ptrs, dt))
    return [p for p in ptrs], (dt[0], dt[1])


def af_set_indicator(ctx, n, s):
    _check(ctx, lib().af_set_indicator(ctx, _dp(_host(s, n))))


def af_set_indicator_device(ctx, dev_ptr):
    _check(ctx, lib().af_set_indicator_device(ctx, _V(dev_ptr)))


def af_forward_euler(ctx, tau):
    _check(ctx, lib().af_forward_euler(ctx, float(tau)))


def af_stage(ctx, k, dt):
    _check(ctx, lib().af_stage(ctx, int(k), float(dt)))


def af_dt_device(ctx):
    _check(ctx, lib().af_dt_device(ctx))


def af_num_stages(ctx):
    return lib().af_num_stages(ctx)


def af_step(ctx, dt=0.0, want_dt=False):
    used = ctypes.c_double(0.0)
    _check(ctx, lib().af_step(ctx, float(dt), ctypes.byref(used) if want_dt else None))
    return used.value if want_dt else None


def af_run(ctx, T):
    n = ctypes.c_longlong(0)
    _check(ctx, lib().af_run(ctx, float(T), ctypes.byref(n)))
    return n.value


def af_time(ctx):
    t = ctypes.c_double()
    _check(ctx, lib().af_time(ctx, ctypes.byref(t)))
    return t.value


def af_mass(ctx):
    m = ctypes.c_double()
    _check(ctx, lib().af_mass(ctx, ctypes.byref(m)))
    return m.value


def af_bounds(ctx):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().af_bounds(ctx, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def af_dt_cfl(ctx):
    d = ctypes.c_double()
    _check(ctx, lib().af_dt_cfl(ctx, ctypes.byref(d)))
    return d.value


def af_stats(ctx):
    c, e, m = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
    _check(ctx, lib().af_stats(ctx, ctypes.byref(c), ctypes.byref(e), ctypes.byref(m)))
    return {"clamps": c.value, "errors": e.value, "max_excess": m.value}
