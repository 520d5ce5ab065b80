"""FP64 CPU oracle for the compact fourth-order doubly conservative active flux method
with monolithic convex MPP limiting (arXiv 2510.11527).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package. The CUDA
library shares no code with it and never calls it.

What lives here:
  * ``af_oracle.cpp`` (loaded through ctypes): one forward-Euler evaluation of the
    method (Sections 2, 4, 5), SSP-RK3 / SSP-RK(5,4) steps, the CFL time step, and a
    flop-counting instantiation of the same source.
  * ``fourier.py``: the semi-discrete Fourier matrix G and the von Neumann CFL search
    (Section 3).
  * ``mlp.py``: FP64 forward/backward of the small indicator network.

Problem descriptions are any object with the attributes of ``af_inputs.Spec``.
"""
import contextlib
import ctypes
import math

import numpy as np

from .build import build_oracle

FLUX_KINDS = {"zero": 0, "linear": 1, "burgers": 2, "bl": 3}
DIFF_KINDS = {"none": 0, "const": 1, "pwl": 2, "pme": 3, "cubic": 4, "ramp": 5, "cubic01": 6}
BC_KINDS = {"periodic": 0, "dirichlet": 1, "outflow": 2}
BLEND_KINDS = {"off": 0, "plain": 1, "external": 2}


class Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("flux_kind", ctypes.c_int), ("flux_p", ctypes.c_double * 4),
        ("diff_kind", ctypes.c_int), ("diff_p", ctypes.c_double * 4),
        ("umin", ctypes.c_double), ("umax", ctypes.c_double),
        ("limiter", ctypes.c_int), ("blend", ctypes.c_int), ("gamma", ctypes.c_double),
        ("clamp_tol", ctypes.c_double),
        ("bc", ctypes.c_int), ("bc_left", ctypes.c_double), ("bc_right", ctypes.c_double),
        ("nodc", ctypes.c_int), ("nz", ctypes.c_int), ("dz", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [("clamps", ctypes.c_longlong), ("max_excess", ctypes.c_double),
                ("error", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build_oracle())
    return _lib


@contextlib.contextmanager
def planted(**defines):
    """Run the oracle API on a variant build with a planted mistake (preprocessor
    macros of af_oracle.cpp), to show that a pin catches it. Restores the oracle on
    exit."""
    global _lib
    saved = lib()
    _lib = _load(build_oracle(defines=defines))
    try:
        yield
    finally:
        _lib = saved


def _load(path):
    lb = ctypes.CDLL(path)
    P = ctypes.POINTER(Problem)
    dpp = ctypes.POINTER(ctypes.c_double)
    arr = ctypes.POINTER(dpp)
    lb.ao_fe.argtypes = [P, arr, ctypes.c_double, dpp, arr]
    lb.ao_step.argtypes = [P, ctypes.c_int, arr, ctypes.c_double, dpp, ctypes.POINTER(Stats)]
    lb.ao_dt.argtypes = [P, dpp, ctypes.c_double, ctypes.c_double]
    lb.ao_dt.restype = ctypes.c_double
    lb.ao_kappa_max.argtypes = [P]
    lb.ao_kappa_max.restype = ctypes.c_double
    lb.ao_alpha_interval.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lb.ao_alpha_interval.restype = ctypes.c_double
    lb.ao_point_funcs.argtypes = [P, ctypes.c_int, ctypes.c_double, dpp, dpp, dpp]
    lb.ao_theta.argtypes = [P, ctypes.c_double, ctypes.c_double]
    lb.ao_theta.restype = ctypes.c_double
    lb.ao_rk54_coefs.argtypes = [dpp, dpp]
    lb.ao_flop_count.argtypes = [P, arr, ctypes.c_double, dpp, ctypes.POINTER(ctypes.c_longlong)]
    lb.ao_fe_generic.argtypes = [P, arr, ctypes.c_double, dpp, arr]
    lb.ao_run.argtypes = [P, ctypes.c_int, arr, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                          ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(Stats)]
    lb.ao_first_order_run.argtypes = [P, dpp, ctypes.c_double, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_longlong)]
    return lb


def make_problem(spec) -> Problem:
    """Translate a problem description (af_inputs.Spec-like) into the oracle's struct."""
    p = Problem()
    p.dim = spec.dim
    p.nx = spec.nx
    p.ny = spec.ny if spec.dim >= 2 else 1
    p.dx = (spec.x1 - spec.x0) / spec.nx
    p.dy = (spec.y1 - spec.y0) / spec.ny if spec.dim >= 2 else 1.0
    p.nz = getattr(spec, "nz", 1) if spec.dim == 3 else 1
    p.dz = (spec.z1 - spec.z0) / spec.nz if spec.dim == 3 else 1.0
    p.flux_kind = FLUX_KINDS[spec.flux[0]]
    for k, v in enumerate(spec.flux[1]):
        p.flux_p[k] = float(v)
    p.diff_kind = DIFF_KINDS[spec.diff[0]]
    for k, v in enumerate(spec.diff[1]):
        p.diff_p[k] = float(v)
    p.umin, p.umax = float(spec.umin), float(spec.umax)
    p.limiter = int(spec.limiter)
    p.blend = BLEND_KINDS[spec.blend]
    p.gamma = float(spec.gamma)
    scale = max(abs(spec.umin), abs(spec.umax), 1e-300)
    p.clamp_tol = 8.0 * np.finfo(np.float64).eps * scale
    p.bc = BC_KINDS[getattr(spec, "bc", "periodic")]
    p.bc_left, p.bc_right = (float(v) for v in getattr(spec, "bc_values", (0.0, 0.0)))
    p.nodc = int(getattr(spec, "diffusion_form", "dc") == "nodc")
    return p


def _ptrs(arrays):
    dpp = ctypes.POINTER(ctypes.c_double)
    return (dpp * len(arrays))(*[a.ctypes.data_as(dpp) for a in arrays])


def _prep(spec, state):
    n = 1 << spec.dim
    assert len(state) == n
    out = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)).copy() for a in state]
    bounded = getattr(spec, "bc", "periodic") != "periodic"
    if bounded and spec.dim == 1:
        assert out[0].size == spec.nx and out[1].size == spec.nx + 1, "bounded 1D state: nx averages, nx+1 points"
    if bounded and spec.dim == 2:
        nx, ny = spec.nx, spec.ny
        want = [nx * ny, (nx + 1) * (ny + 1), (nx + 1) * ny, nx * (ny + 1)]
        assert [a.size for a in out] == want, "2D rectangle with ends: ub, V, X, Y sizes"
    return out


def _sext(s_ext):
    if s_ext is None:
        return None, None
    s = np.ascontiguousarray(np.asarray(s_ext, dtype=np.float64))
    return s, s.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def fe(spec, state, tau, s_ext=None):
    """One forward-Euler evaluation FE(state, tau) -> new state (list of arrays)."""
    p = make_problem(spec)
    a = _prep(spec, state)
    out = [np.zeros_like(x) for x in a]
    s, sp = _sext(s_ext)
    if lib().ao_fe(ctypes.byref(p), _ptrs(a), float(tau), sp, _ptrs(out)) == -2:
        raise ValueError("combination not supported by the oracle")
    return out


def fe_generic(spec, state, tau, s_ext=None):
    """The dimension-generic fine-grid evaluation of a periodic state (arrays in the
    library's order); for 1D and 2D it restates fe() in another form."""
    p = make_problem(spec)
    a = _prep(spec, state)
    out = [np.zeros_like(x) for x in a]
    s, sp = _sext(s_ext)
    if lib().ao_fe_generic(ctypes.byref(p), _ptrs(a), float(tau), sp, _ptrs(out)) == -2:
        raise ValueError("combination not supported by the oracle")
    return out


def diffusion_spectral_radius(dim, n=4):
    """Spectral radius (in units of kappa / h^2) of the unlimited scheme's semi-discrete
    operator for a = u on a periodic mesh of n cells per direction with h = 1, assembled
    column by column from the oracle's forward-Euler step (the scheme is linear, so
    FE(u, 1) - u is the operator applied to u)."""
    import af_inputs
    kw = dict(dim=dim, nx=n, x0=0.0, x1=float(n), flux=("zero", ()), diff=("const", (1.0,)), umin=-1e9,
              umax=1e9, limiter=False)
    if dim >= 2:
        kw.update(ny=n, y0=0.0, y1=float(n))
    if dim == 3:
        kw.update(nz=n, z0=0.0, z1=float(n))
    spec = af_inputs.Spec(**kw)
    cells = n ** dim
    nk = 1 << dim
    size = cells * nk
    A = np.zeros((size, size))
    for col in range(size):
        st = [np.zeros(cells) for _ in range(nk)]
        st[col // cells][col % cells] = 1.0
        out = fe(spec, st, 1.0)
        A[:, col] = np.concatenate([o.ravel() - x.ravel() for o, x in zip(out, st)])
    return float(np.max(np.abs(np.linalg.eigvals(A))))


def step(spec, rk, state, dt, s_ext=None):
    """One SSP-RK time step (rk = 3 or 54). Returns (new_state, stats dict)."""
    p = make_problem(spec)
    a = _prep(spec, state)
    st = Stats()
    s, sp = _sext(s_ext)
    rc = lib().ao_step(ctypes.byref(p), int(rk), _ptrs(a), float(dt), sp, ctypes.byref(st))
    if rc == -1:
        raise ValueError("unknown rk scheme")
    if rc == -2:
        raise ValueError("combination not supported by the oracle")
    return a, {"clamps": st.clamps, "max_excess": st.max_excess, "error": st.error}


# 0.9 x the linear (von Neumann) stability limit of the unlimited scheme for pure
# diffusion, kappa dt / h^2: 1D from Table 1 (0.157, 0.333), 2D from the 4x4 symbol
# (spectral radius 40.78 kappa/h^2 -> 0.0616 for SSP-RK3, 0.1307 for SSP-RK(5,4)), 3D
# from the 8x8 symbol (63.335 kappa/h^2; the stability intervals of SSP-RK3 and
# SSP-RK(5,4) on the negative real axis reach 2.5127 and 5.330).
DIFF_CAP = {(1, 3): 0.9 * 0.157, (1, 54): 0.9 * 0.333, (2, 3): 0.9 * 0.0616, (2, 54): 0.9 * 0.1307,
            (3, 3): 0.9 * 2.5127 / 63.335, (3, 54): 0.9 * 5.330 / 63.335}


def default_cfl_diff(spec, rk):
    """Default diffusive cap Cd: 0.9 x the linear diffusive limit of the unlimited
    scheme, for every scheme. At the printed C = 0.33/d alone the 2D high-order scheme
    is linearly unstable wherever kappa dt/h^2 exceeds that limit: unlimited runs blow
    up, limited SSP-RK3 runs develop point-value oscillations (Example 6.4), and limited
    SSP-RK(5,4) runs stay bounded but lose accuracy (the porous-medium workload at
    1024^2 ends 1000x further from the closed form) and amplify rounding."""
    return DIFF_CAP[(spec.dim, rk)]


def dt_cfl(spec, ub, cfl=None, cfl_diff=None):
    """dt = min(C / max(alpha/h + kappa_max/h^2), Cd h^2 / kappa_max); C defaults to
    0.33/d (the paper's experiments) and Cd to default_cfl_diff."""
    p = make_problem(spec)
    u = np.ascontiguousarray(np.asarray(ub, dtype=np.float64))
    if cfl is None:
        cfl = spec.cfl if getattr(spec, "cfl", 0.0) else 0.33 / spec.dim
    if cfl_diff is None:
        cfl_diff = default_cfl_diff(spec, getattr(spec, "rk", 3))
    return lib().ao_dt(ctypes.byref(p), u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(cfl),
                       float(cfl_diff))


def kappa_max(spec):
    p = make_problem(spec)
    return lib().ao_kappa_max(ctypes.byref(p))


def alpha_interval(spec, direction, a, b):
    p = make_problem(spec)
    return lib().ao_alpha_interval(ctypes.byref(p), int(direction), float(a), float(b))


def point_funcs(spec, direction, u):
    """(f_l(u), f_l'(u), a(u)) as the oracle evaluates them."""
    p = make_problem(spec)
    f, d, a = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().ao_point_funcs(ctypes.byref(p), int(direction), float(u), ctypes.byref(f), ctypes.byref(d),
                         ctypes.byref(a))
    return f.value, d.value, a.value


def theta(spec, zL, zH):
    p = make_problem(spec)
    return lib().ao_theta(ctypes.byref(p), float(zL), float(zH))


def rk54_coefficients():
    """Shu-Osher (alpha, beta) 5x5 tables of the oracle's SSP-RK(5,4)."""
    a = np.zeros(25)
    b = np.zeros(25)
    dpp = ctypes.POINTER(ctypes.c_double)
    lib().ao_rk54_coefs(a.ctypes.data_as(dpp), b.ctypes.data_as(dpp))
    return a.reshape(5, 5), b.reshape(5, 5)


def flop_count(spec, state, tau, s_ext=None):
    """Flops of one FE evaluation: dict(add, mul, div, exp, cmp)."""
    p = make_problem(spec)
    a = _prep(spec, state)
    s, sp = _sext(s_ext)
    out = (ctypes.c_longlong * 5)()
    lib().ao_flop_count(ctypes.byref(p), _ptrs(a), float(tau), sp, out)
    return dict(zip(["add", "mul", "div", "exp", "cmp"], list(out)))


def mass(spec, ub):
    """Total mass sum(ub) * dx * dy (FP64, plain summation in index order)."""
    p = make_problem(spec)
    return float(math.fsum(np.asarray(ub, dtype=np.float64).ravel())) * p.dx * p.dy


def bounds(state):
    """Min and max over all DoFs."""
    return (min(float(np.min(a)) for a in state), max(float(np.max(a)) for a in state))


def run(spec, rk, state, T, cfl=None, dt_fixed=None, max_steps=10**7, cfl_diff=None):
    """Integrate to time T (last step clipped). Returns (state, nsteps, stats)."""
    t = 0.0
    n = 0
    tot = {"clamps": 0, "max_excess": 0.0, "error": 0}
    state = _prep(spec, state)
    while t < T * (1 - 1e-14) and n < max_steps:
        if dt_fixed is not None:
            dt = dt_fixed
        else:
            cd = cfl_diff if cfl_diff is not None else default_cfl_diff(spec, rk)
            dt = dt_cfl(spec, state[0], cfl, cd)
        dt = min(dt, T - t)
        state, st = step(spec, rk, state, dt)
        tot["clamps"] += st["clamps"]
        tot["max_excess"] = max(tot["max_excess"], st["max_excess"])
        tot["error"] |= st["error"]
        t += dt
        n += 1
    return state, n, tot


def run_native(spec, rk, state, T, cfl=None, cfl_diff=None):
    """Integrate to time T with the CFL step inside the oracle library (same clipping
    rule as ``run``). Returns (state, nsteps, stats)."""
    p = make_problem(spec)
    a = _prep(spec, state)
    if cfl is None:
        cfl = spec.cfl if getattr(spec, "cfl", 0.0) else 0.33 / spec.dim
    if cfl_diff is None:
        cfl_diff = default_cfl_diff(spec, rk)
    st = Stats()
    n = ctypes.c_longlong(0)
    rc = lib().ao_run(ctypes.byref(p), int(rk), _ptrs(a), float(T), float(cfl), float(cfl_diff),
                      ctypes.byref(n), ctypes.byref(st))
    if rc == -2:
        raise ValueError("combination not supported by the oracle")
    if rc not in (0, -4):
        raise ValueError(f"oracle run failed ({rc})")
    return a, n.value, {"clamps": st.clamps, "max_excess": st.max_excess, "error": st.error}


def first_order_run(spec, ub, T, cfl=0.9):
    """First-order LLF + central-difference reference scheme for the cell averages of a
    1D problem (forward Euler, dt = cfl / max(alpha/h + 2 kappa_max/h^2)) to time T.
    Returns (ub, nsteps)."""
    p = make_problem(spec)
    u = np.ascontiguousarray(np.asarray(ub, dtype=np.float64)).copy()
    n = ctypes.c_longlong(0)
    rc = lib().ao_first_order_run(ctypes.byref(p), u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  float(T), float(cfl), ctypes.byref(n))
    if rc:
        raise ValueError("combination not supported by the oracle")
    return u, n.value
