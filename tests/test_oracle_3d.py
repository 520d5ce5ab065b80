"""Pins of the oracle's 3D evaluation (Section 4's 3D DoFs: averages, face-, edge- and
corner-point values; Section 5.2 with d = 3, limiter factor 18).

The 3D step is a dimension-generic evaluation on the fine grid of half-cell spacing,
where every 5-point line of the paper is the fine points p - 2e .. p + 2e along one axis
and every Simpson average takes weights 1, 4, 1 per axis. It is pinned by:
  * agreeing with the dedicated (pinned) 1D and 2D evaluations in d = 1, 2;
  * 3D data independent of z reducing exactly to the 2D scheme (limiter off, blend on);
  * the orders of its operators on exact nodal data (fourth for diffusion and for the
    averages; third for convection at points, as the one-sided D+- stencils are);
  * conservation, MPP on rough data, constant states, and axis-permutation symmetry;
  * the diffusion symbol's spectral radius: 16 (1D), 40.78 (2D), 63.34 (3D) kappa/h^2.
"""
import dataclasses
import math

import numpy as np
import pytest

import af_inputs as ai
import oracle


def _np(st):
    return [np.asarray(a, dtype=np.float64) for a in st]


@pytest.mark.parametrize("flux,diff", [(("burgers", (0.5,)), ("pwl", (0.05, 0.25, 0.05, 0.75))),
                                       (("bl", (5.0,)), ("cubic", (0.0, 0.02, -0.04 / 3))),
                                       (("linear", (1.0, -0.6)), ("ramp", (0.05, 0.4, 0.2))),
                                       (("zero", ()), ("pme", (2,)))])
@pytest.mark.parametrize("limiter,blend", [(True, "off"), (False, "off"), (True, "plain"), (True, "external")])
@pytest.mark.parametrize("dim", [1, 2])
def test_generic_evaluation_equals_dedicated(flux, diff, limiter, blend, dim):
    kw = dict(dim=dim, nx=13, x0=0.0, x1=1.3, flux=flux, diff=diff, umin=0.0, umax=1.0, limiter=limiter, blend=blend)
    if dim == 2:
        kw.update(ny=7, y0=0.0, y1=0.9)
    sp = ai.Spec(**kw)
    st = _np(ai.random_state_1d(sp, 3) if dim == 1 else ai.random_state_2d(sp, 3))
    s_ext = np.random.default_rng(1).random(st[0].shape) if blend == "external" else None
    tau = oracle.dt_cfl(sp, st[0])
    a = oracle.fe(sp, st, tau, s_ext)
    b = oracle.fe_generic(sp, st, tau, s_ext)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) < 2e-14


@pytest.mark.parametrize("blend", ["off", "plain"])
def test_z_independent_3d_data_reduce_to_2d(blend):
    nx, ny, nz = 9, 7, 4
    common = dict(flux=("burgers", (0.5,)), diff=("pwl", (0.05, 0.25, 0.05, 0.75)), umin=-2.0, umax=2.0,
                  limiter=False, blend=blend)
    s2 = ai.Spec(dim=2, nx=nx, ny=ny, x0=0, x1=0.9, y0=0, y1=0.7, **common)
    s3 = ai.Spec(dim=3, nx=nx, ny=ny, nz=nz, x0=0, x1=0.9, y0=0, y1=0.7, z0=0, z1=0.4, **common)
    ub, V, X, Y = _np(ai.random_state_2d(s2, 5, lo=0.0, hi=1.0))
    # the 2D recovered centre (the z-face value of z-independent data)
    c = (36 * ub - 4 * (np.roll(X, 1, 1) + X + np.roll(Y, 1, 0) + Y)
         - (np.roll(np.roll(V, 1, 0), 1, 1) + np.roll(V, 1, 0) + np.roll(V, 1, 1) + V)) / 16
    z = lambda a: np.repeat(a[None], nz, axis=0)
    st3 = [z(ub), z(X), z(Y), z(V), z(c), z(X), z(Y), z(V)]
    tau = 0.5 * oracle.dt_cfl(s2, ub)
    o2 = oracle.fe(s2, [ub, V, X, Y], tau)
    o3 = oracle.fe(s3, st3, tau)
    # with the blend, the low-order point residual of an xz- / yz-edge value reads the
    # z-face value (a DoF in 3D) where its 2D counterpart X / Y reads a centre, replaced
    # by the cell average: those two kinds reduce only without the blend
    pairs = ((0, 0), (1, 2), (2, 3), (3, 1), (5, 2), (6, 3), (7, 1))
    for k3, k2 in pairs:
        if blend == "plain" and k3 in (5, 6):
            continue
        assert np.max(np.abs(o3[k3] - z(o2[k2]))) < 1e-13, k3


def _smooth_3d(n, flux, k0):
    """sin(x + y + z) + 0.5 on [0, 2 pi]^3: exact point values; averages chosen so the
    recovered centre is the exact centre value (tensor Simpson of the exact values)"""
    sp = ai.Spec(dim=3, nx=n, ny=n, nz=n, x0=0, x1=2 * math.pi, y0=0, y1=2 * math.pi, z0=0, z1=2 * math.pi,
                 flux=flux, diff=("const", (k0,)), umin=-10, umax=10, limiter=False)
    h = sp.dx
    g = lambda x, y, zz: 0.5 + np.sin(x + y + zz)
    c = (np.arange(n) + 0.5) * h
    Zc, Yc, Xc = np.meshgrid(c, c, c, indexing="ij")
    pts = []
    for s in range(1, 8):
        sx, sy, sz = s & 1, (s >> 1) & 1, (s >> 2) & 1
        pts.append(g(Xc + 0.5 * h * sx, Yc + 0.5 * h * sy, Zc + 0.5 * h * sz))
    w = {-1: 1.0, 0: 4.0, 1: 1.0}
    ub = np.zeros_like(Xc)
    for mx in (-1, 0, 1):
        for my in (-1, 0, 1):
            for mz in (-1, 0, 1):
                ub += w[mx] * w[my] * w[mz] * g(Xc + 0.5 * h * mx, Yc + 0.5 * h * my, Zc + 0.5 * h * mz)
    ub /= 216.0
    return sp, [ub] + pts, (Xc, Yc, Zc), h


# Diffusion: the compact second difference and the DC potentials are fourth order at
# points and averages. Convection: the face averages are fourth order; at points the
# biased operators D+- are 4-point one-sided stencils (spacing h/2) whose O(h^3) errors
# cancel in the central part but not in the upwind dissipation (D+ - D-) (alpha z) / 2,
# so the point operator is third order.
@pytest.mark.parametrize("case,flux,k0,point_rate", [("diffusion", ("zero", ()), 0.05, 3.7),
                                                      ("convection", ("linear", (1.0, 0.7, -0.4)), 0.0, 2.8)])
def test_3d_operators_order(case, flux, k0, point_rate):
    cvec = np.array(flux[1] if flux[0] == "linear" else (0.0, 0.0, 0.0))
    rhs = lambda x, y, z: -cvec.sum() * np.cos(x + y + z) - 3 * k0 * np.sin(x + y + z)
    ep, ea = [], []
    gx, gw = np.polynomial.legendre.leggauss(6)
    for n in (6, 12, 24):
        sp, st, (Xc, Yc, Zc), h = _smooth_3d(n, flux, k0)
        out = oracle.fe(sp, st, 1.0)
        err = 0.0
        for s in range(1, 8):
            sx, sy, sz = s & 1, (s >> 1) & 1, (s >> 2) & 1
            ex = rhs(Xc + 0.5 * h * sx, Yc + 0.5 * h * sy, Zc + 0.5 * h * sz)
            err = max(err, np.max(np.abs((out[s] - st[s]) - ex)))
        ep.append(err)
        avg = np.zeros_like(Xc)
        for a, wa in zip(gx, gw):
            for b, wb in zip(gx, gw):
                for cc, wc in zip(gx, gw):
                    avg += wa * wb * wc / 8 * rhs(Xc + 0.5 * h * a, Yc + 0.5 * h * b, Zc + 0.5 * h * cc)
        ea.append(np.max(np.abs((out[0] - st[0]) - avg)))
    rp = [math.log2(ep[k] / ep[k + 1]) for k in range(2)]
    ra = [math.log2(ea[k] / ea[k + 1]) for k in range(2)]
    assert min(rp) > point_rate, (ep, rp)
    assert min(ra) > 3.7, (ea, ra)


def _rough3d(flux=("burgers", (0.5,)), diff=("pwl", (0.05, 0.25, 0.05, 0.75)), blend="off", n=(7, 6, 5)):
    sp = ai.Spec(dim=3, nx=n[0], ny=n[1], nz=n[2], x0=0, x1=0.7, y0=0, y1=0.6, z0=0, z1=0.5, flux=flux, diff=diff,
                 umin=0.0, umax=1.0, limiter=True, blend=blend)
    return sp, _np(ai.random_state_3d(sp, 17))


@pytest.mark.parametrize("blend", ["off", "plain"])
def test_3d_mass_conservation_and_mpp(blend):
    sp, st = _rough3d(blend=blend)
    m0 = float(np.sum(st[0]))
    for _ in range(4):
        st, stats = oracle.step(sp, 3, st, oracle.dt_cfl(sp, st[0]))
        assert stats["error"] == 0
        lo, hi = oracle.bounds(st)
        assert lo >= 0.0 and hi <= 1.0
    assert abs(float(np.sum(st[0])) - m0) < 1e-12 * st[0].size


def test_3d_constant_state_preserved():
    sp, st = _rough3d()
    st = [np.full_like(a, 0.37) for a in st]
    out = oracle.fe(sp, st, oracle.dt_cfl(sp, st[0]))
    for a in out:
        assert np.max(np.abs(a - 0.37)) < 1e-15


def test_3d_axis_permutation_symmetry():
    # swapping x and z (equal spacing, isotropic flux) maps the step to itself: arrays
    # transpose and the kinds swap their x and z bits
    sp = ai.Spec(dim=3, nx=6, ny=5, nz=6, x0=0, x1=0.6, y0=0, y1=0.5, z0=0, z1=0.6, flux=("burgers", (0.5,)),
                 diff=("pwl", (0.05, 0.25, 0.05, 0.75)), umin=0.0, umax=1.0, limiter=True, blend="plain")
    st = _np(ai.random_state_3d(sp, 23))
    swap = lambda s: ((s & 1) << 2) | (s & 2) | ((s >> 2) & 1)
    tr = lambda a: np.ascontiguousarray(np.transpose(a, (2, 1, 0)))
    st_t = [tr(st[swap(s)]) for s in range(8)]
    tau = oracle.dt_cfl(sp, st[0])
    a = oracle.fe(sp, st, tau)
    b = oracle.fe(sp, st_t, tau)
    for s in range(8):
        assert np.max(np.abs(tr(a[swap(s)]) - b[s])) < 1e-14, s


def test_diffusion_symbol_radius():
    assert oracle.diffusion_spectral_radius(1, 8) == pytest.approx(16.0, rel=1e-12)
    assert oracle.diffusion_spectral_radius(2, 4) == pytest.approx(40.777, rel=1e-4)
    assert oracle.diffusion_spectral_radius(3, 4) == pytest.approx(63.335, rel=1e-4)


@pytest.mark.parametrize("blend", ["off", "plain"])
@pytest.mark.parametrize("dim", [2, 3])
def test_zero_flux_skips_only_exact_zeros(blend, dim):
    """With f = 0 the generic evaluation does not form the convection terms (the Simpson
    face fluxes, the flux part of every 5-point line, the LLF fluxes and their share of
    the low-order states). A linear flux with zero velocities forms all of them, every
    one an exact zero: the two evaluations agree exactly, and the flop count of f = 0 is
    smaller by those terms alone (the diffusion, limiter and update operations stay)."""
    diff = ("pme", (2,))
    if dim == 3:
        sz, st = _rough3d(flux=("zero", ()), diff=diff, blend=blend)
        sl = dataclasses.replace(sz, flux=("linear", (0.0, 0.0, 0.0)))
    else:
        sz = ai.Spec(dim=2, nx=9, ny=7, x0=0.0, x1=0.9, y0=0.0, y1=0.7, flux=("zero", ()), diff=diff, umin=0.0,
                     umax=1.0, limiter=True, blend=blend)
        sl = dataclasses.replace(sz, flux=("linear", (0.0, 0.0)))
        st = _np(ai.random_state_2d(sz, 19))
    tau = oracle.dt_cfl(sz, st[0])
    fz = oracle.fe_generic(sz, st, tau) if dim == 2 else oracle.fe(sz, st, tau)
    fl = oracle.fe_generic(sl, st, tau) if dim == 2 else oracle.fe(sl, st, tau)
    for a, b in zip(fz, fl):
        assert np.array_equal(a, b)
    if dim == 3:
        cz = oracle.flop_count(sz, st, tau)
        cl = oracle.flop_count(sl, st, tau)
        nz = sum(cz[k] for k in ("add", "mul", "div"))
        nl = sum(cl[k] for k in ("add", "mul", "div"))
        assert 0 < nz < nl
        # per cell, at least the 21 lines' convection parts (each far above 10 operations)
        assert (nl - nz) / st[0].size > 21 * 10
