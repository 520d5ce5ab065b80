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
DIFF = {"none": 0, "const": 1, "pwl": 2, "pme": 3, "cubic": 4, "ramp": 5, "cubic01": 6}
BC = {"periodic": 0, "dirichlet": 1, "outflow": 2}
FORM = {"dc": 0, "nodc": 1}
PREC = {"fp64": 0, "fp32_mixed": 1}
BLEND = {"off": 0, "plain": 1, "external": 2}


class AfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class af_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x0", ctypes.c_double),
                ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double), ("bc", ctypes.c_int),
                ("bc_left", ctypes.c_double), ("bc_right", ctypes.c_double), ("nz", ctypes.c_int),
                ("z0", ctypes.c_double), ("z1", ctypes.c_double)]


class af_flux(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("p", ctypes.c_double * 4)]


class af_diff(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("p", ctypes.c_double * 4)]


class af_bounds_t(ctypes.Structure):
    _fields_ = [("umin", ctypes.c_double), ("umax", ctypes.c_double), ("from_initial_data", ctypes.c_int)]


class af_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("rk", ctypes.c_int), ("cfl", ctypes.c_double),
                ("cfl_diff", ctypes.c_double), ("limiter", ctypes.c_int), ("blend", ctypes.c_int),
                ("gamma", ctypes.c_double), ("diffusion_form", ctypes.c_int)]


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
        "af_set_state_arrays": [_V, ctypes.c_int, ctypes.POINTER(_D)],
        "af_get_state_arrays": [_V, ctypes.c_int, ctypes.POINTER(_D)],
        "af_device_ptrs_arrays": [_V, ctypes.c_int, ctypes.POINTER(_V), ctypes.POINTER(ctypes.c_int)],
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
        "af_stats": [_V, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), _D, _D],
        "af_stats_detail": [_V, ctypes.POINTER(ctypes.c_longlong)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.af_last_error.argtypes = [_V]
    L.af_last_error.restype = ctypes.c_char_p
    L.af_num_stages.argtypes = [_V]
    L.af_num_stages.restype = ctypes.c_int
    L.af_mass_noalloc.argtypes = [_V, ctypes.c_longlong, ctypes.c_double, _D, _V]
    L.af_mass_noalloc.restype = ctypes.c_int
    I = ctypes.POINTER(ctypes.c_int)
    bsig = {
        "af_batch_create": [ctypes.c_int, ctypes.POINTER(af_grid), ctypes.POINTER(af_flux), ctypes.POINTER(af_diff),
                            ctypes.POINTER(af_bounds_t), ctypes.POINTER(af_opts), ctypes.POINTER(_V)],
        "af_batch_destroy": [_V],
        "af_batch_set_stream": [_V, _V],
        "af_batch_info": [_V, ctypes.POINTER(ctypes.c_longlong), I, I, I],
        "af_batch_set_tile": [_V, ctypes.c_int, ctypes.c_int],
        "af_batch_autotune": [_V, I, I],
        "af_batch_set_state": [_V, ctypes.c_int, _D, _D, _D, _D],
        "af_batch_get_state": [_V, ctypes.c_int, _D, _D, _D, _D],
        "af_batch_device_ptrs": [_V, ctypes.c_int, ctypes.POINTER(_V), I],
        "af_batch_step": [_V, ctypes.c_int],
        "af_batch_sync": [_V],
        "af_batch_time": [_V, ctypes.c_int, _D],
        "af_batch_mass": [_V, ctypes.c_int, _D],
        "af_batch_bounds": [_V, ctypes.c_int, _D, _D],
        "af_batch_stats": [_V, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), _D],
    }
    for name, args in bsig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.af_batch_last_error.argtypes = [_V]
    L.af_batch_last_error.restype = ctypes.c_char_p
    F = ctypes.POINTER(ctypes.c_float)
    msig = {
        "af_mlp_create": [ctypes.POINTER(_V)],
        "af_mlp_destroy": [_V],
        "af_mlp_set_params": [_V, F, ctypes.c_int],
        "af_mlp_get_params": [_V, F],
        "af_mlp_features": [_V, _V, _V],
        "af_mlp_infer": [_V, _V, ctypes.c_longlong, _V],
        "af_mlp_indicator": [_V, _V, _V],
        "af_mlp_grad": [_V, _V, _V, ctypes.c_int, F, F],
        "af_mlp_train": [_V, _V, _V, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                         ctypes.c_ulonglong, F],
        "af_set_mlp": [_V, _V],
        "af_batch_set_mlp": [_V, _V],
    }
    for name, args in msig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    _lib = L
    return L


def exported_symbols():
    """Names of the entry points declared in include/af.h (for the export test)."""
    return ["af_create", "af_destroy", "af_last_error", "af_set_stream", "af_set_state", "af_get_state",
            "af_device_ptrs", "af_set_state_arrays", "af_get_state_arrays", "af_device_ptrs_arrays", "af_set_indicator", "af_set_indicator_device", "af_forward_euler", "af_stage", "af_dt_device",
            "af_num_stages", "af_step", "af_run", "af_time", "af_mass", "af_bounds", "af_dt_cfl", "af_stats", "af_stats_detail",
            "af_mass_noalloc", "af_batch_create", "af_batch_destroy", "af_batch_last_error", "af_batch_set_stream",
            "af_batch_info", "af_batch_set_tile", "af_batch_autotune", "af_batch_set_state", "af_batch_get_state",
            "af_batch_device_ptrs", "af_batch_step", "af_batch_sync", "af_batch_time", "af_batch_mass",
            "af_batch_bounds", "af_batch_stats", "af_mlp_create", "af_mlp_destroy", "af_mlp_set_params",
            "af_mlp_get_params", "af_mlp_features", "af_mlp_infer", "af_mlp_indicator", "af_mlp_grad",
            "af_mlp_train", "af_set_mlp", "af_batch_set_mlp"]


AF_MLP_NPARAM = 1793
_FP = ctypes.POINTER(ctypes.c_float)


def af_mlp_create():
    net = _V()
    st = lib().af_mlp_create(ctypes.byref(net))
    if st != AF_OK:
        raise AfError(st, "af_mlp_create failed")
    return net


def af_mlp_destroy(net):
    _check(None, lib().af_mlp_destroy(net))


def af_mlp_set_params(net, params):
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    _check(None, lib().af_mlp_set_params(net, p.ctypes.data_as(_FP), int(p.size)))


def af_mlp_get_params(net):
    p = np.empty(AF_MLP_NPARAM, dtype=np.float32)
    _check(None, lib().af_mlp_get_params(net, p.ctypes.data_as(_FP)))
    return p


def af_mlp_features(ctx, feat_dev_ptr, label_dev_ptr=None):
    _check(ctx, lib().af_mlp_features(ctx, _V(feat_dev_ptr), _V(label_dev_ptr) if label_dev_ptr else None))


def af_mlp_infer(net, feat_dev_ptr, n, out_dev_ptr):
    _check(None, lib().af_mlp_infer(net, _V(feat_dev_ptr), int(n), _V(out_dev_ptr)))


def af_mlp_indicator(net, ctx, s_dev_ptr):
    _check(ctx, lib().af_mlp_indicator(net, ctx, _V(s_dev_ptr)))


def af_mlp_grad(net, feat_dev_ptr, label_dev_ptr, n):
    g = np.empty(AF_MLP_NPARAM, dtype=np.float32)
    loss = ctypes.c_float()
    _check(None, lib().af_mlp_grad(net, _V(feat_dev_ptr), _V(label_dev_ptr), int(n), g.ctypes.data_as(_FP),
                                   ctypes.byref(loss)))
    return g, loss.value


def af_mlp_train(net, feat_dev_ptr, label_dev_ptr, nsamples, batch, steps, lr, seed):
    loss = ctypes.c_float()
    _check(None, lib().af_mlp_train(net, _V(feat_dev_ptr), _V(label_dev_ptr), int(nsamples), int(batch),
                                    int(steps), float(lr), int(seed), ctypes.byref(loss)))
    return loss.value


def af_set_mlp(ctx, net):
    _check(ctx, lib().af_set_mlp(ctx, net))


def _bcheck(b, st):
    if st != AF_OK:
        msg = lib().af_batch_last_error(b).decode() if b else ""
        raise AfError(st, msg)


def af_batch_set_mlp(b, net):
    _bcheck(b, lib().af_batch_set_mlp(b, net))


def af_batch_create(grids, fluxes, diffs, bounds, opts):
    n = len(grids)
    G = (af_grid * n)(*grids)
    F = (af_flux * n)(*fluxes)
    D = (af_diff * n)(*diffs)
    B = (af_bounds_t * n)(*bounds)
    b = _V()
    st = lib().af_batch_create(n, G, F, D, B, ctypes.byref(opts), ctypes.byref(b))
    if st != AF_OK:
        raise AfError(st, "af_batch_create failed")
    return b


def af_batch_destroy(b):
    _bcheck(None, lib().af_batch_destroy(b))


def af_batch_set_stream(b, stream_handle):
    _bcheck(b, lib().af_batch_set_stream(b, _V(stream_handle)))


def af_batch_info(b):
    c, t, x, y = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _bcheck(b, lib().af_batch_info(b, ctypes.byref(c), ctypes.byref(t), ctypes.byref(x), ctypes.byref(y)))
    return {"cells": c.value, "tiles": t.value, "tile": (x.value, y.value)}


def af_batch_set_tile(b, tx, ty):
    _bcheck(b, lib().af_batch_set_tile(b, int(tx), int(ty)))


def af_batch_autotune(b):
    x, y = ctypes.c_int(), ctypes.c_int()
    _bcheck(b, lib().af_batch_autotune(b, ctypes.byref(x), ctypes.byref(y)))
    return x.value, y.value


def af_batch_set_state(b, i, n, ub, V, X, Y):
    arrs = [_host(a, n) for a in (ub, V, X, Y)]
    _bcheck(b, lib().af_batch_set_state(b, int(i), *[_dp(a) for a in arrs]))


def af_batch_get_state(b, i, n):
    out = [np.empty(n) for _ in range(4)]
    _bcheck(b, lib().af_batch_get_state(b, int(i), *[_dp(a) for a in out]))
    return out


def af_batch_device_ptrs(b, i):
    ptrs = (_V * 4)()
    dt = (ctypes.c_int * 2)()
    _bcheck(b, lib().af_batch_device_ptrs(b, int(i), ptrs, dt))
    return [p for p in ptrs], (dt[0], dt[1])


def af_batch_step(b, nsteps=1):
    _bcheck(b, lib().af_batch_step(b, int(nsteps)))


def af_batch_sync(b):
    _bcheck(b, lib().af_batch_sync(b))


def af_batch_time(b, i):
    t = ctypes.c_double()
    _bcheck(b, lib().af_batch_time(b, int(i), ctypes.byref(t)))
    return t.value


def af_batch_mass(b, i):
    m = ctypes.c_double()
    _bcheck(b, lib().af_batch_mass(b, int(i), ctypes.byref(m)))
    return m.value


def af_batch_bounds(b, i):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _bcheck(b, lib().af_batch_bounds(b, int(i), ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def af_batch_stats(b):
    c, e, m = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
    _bcheck(b, lib().af_batch_stats(b, ctypes.byref(c), ctypes.byref(e), ctypes.byref(m)))
    return {"clamps": c.value, "errors": e.value, "max_excess": m.value}


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


def af_set_state(ctx, n, ub, V, X=None, Y=None, npts=None, sizes=None):
    """npts: values per point array (default n; n + 1 on a bounded 1D interval); sizes:
    the values of ub, V, X, Y one by one (a 2D rectangle with ends)."""
    m = n if npts is None else npts
    sz = sizes if sizes is not None else [n, m, m, m]
    arrs = [_host(ub, sz[0]), _host(V, sz[1]), None if X is None else _host(X, sz[2]),
            None if Y is None else _host(Y, sz[3])]
    _check(ctx, lib().af_set_state(ctx, *[_dp(a) for a in arrs]))


def af_get_state(ctx, n, dim, out=None, npts=None, sizes=None):
    """Copy the state to host float64 arrays: `out` (C-contiguous float64 arrays, e.g.
    views of pinned memory) or new arrays; n averages, npts (default n) point values
    per point array, or the values of each array in `sizes`."""
    k = 4 if dim == 2 else 2
    m = n if npts is None else npts
    sizes = list(sizes[:k]) if sizes is not None else [n] + [m] * (k - 1)
    if out is None:
        out = [np.empty(z) for z in sizes]
    else:
        out = list(out)
        if len(out) != k or any(not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.size == z and
                                     a.flags.c_contiguous) for a, z in zip(out, sizes)):
            raise ValueError(f"out must be {k} C-contiguous float64 arrays of {sizes} values")
    full = out + ([None, None] if dim == 1 else [])
    _check(ctx, lib().af_get_state(ctx, *[_dp(a) for a in full]))
    return out


def af_set_state_arrays(ctx, arrays, sizes):
    """The state as 2^dim host arrays (3D: the 8 arrays by kind), `sizes` values each."""
    hs = [_host(a, n) for a, n in zip(arrays, sizes)]
    ptrs = (_D * len(hs))(*[_dp(a) for a in hs])
    _check(ctx, lib().af_set_state_arrays(ctx, len(hs), ptrs))


def af_get_state_arrays(ctx, sizes, out=None):
    out = [np.empty(n) for n in sizes] if out is None else list(out)
    for a, n in zip(out, sizes):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.size == n and a.flags.c_contiguous):
            raise ValueError(f"out arrays must be C-contiguous float64 with {sizes} values")
    ptrs = (_D * len(out))(*[_dp(a) for a in out])
    _check(ctx, lib().af_get_state_arrays(ctx, len(out), ptrs))
    return out


def af_device_ptrs_arrays(ctx, narr):
    ptrs = (_V * narr)()
    dt = (ctypes.c_int * 2)()
    _check(ctx, lib().af_device_ptrs_arrays(ctx, narr, ptrs, dt))
    return [p for p in ptrs], (dt[0], dt[1])


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


AF_MASS_NOALLOC_MAX_CELLS = 134217728


def af_mass_noalloc(ub_dev_ptr, ncells, cell_area, stream_handle=None):
    """Allocation-free total mass of a caller-owned device array of cell averages
    (for callers that cannot allocate device memory; see include/af.h)."""
    m = ctypes.c_double()
    st = lib().af_mass_noalloc(_V(ub_dev_ptr), int(ncells), float(cell_area), ctypes.byref(m),
                               _V(stream_handle) if stream_handle else None)
    if st != AF_OK:
        raise AfError(st, f"af_mass_noalloc(ncells={ncells}) failed (maximum {AF_MASS_NOALLOC_MAX_CELLS} cells)")
    return m.value


def af_stats(ctx):
    c, e, m, a = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().af_stats(ctx, ctypes.byref(c), ctypes.byref(e), ctypes.byref(m), ctypes.byref(a)))
    ac = ctypes.c_longlong()
    _check(ctx, lib().af_stats_detail(ctx, ctypes.byref(ac)))
    return {"clamps": c.value, "errors": e.value, "max_excess": m.value, "mass_adjust": a.value,
            "avg_clamps": ac.value}
