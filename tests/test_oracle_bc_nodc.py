"""Pins of the oracle's 1D boundary conditions and of the AF method without double
conservation (Appendix A of arXiv 2510.11527), against what the paper and the
mathematics fix:

  * Appendix A states that for a = kappa0 u its scheme coincides with the doubly
    conservative one; its compact operator is fourth-order for smooth kappa(u);
  * even reflection (outflow) of a mesh equals the periodic mesh of twice the size with
    mirrored data whenever the scheme is mirror-symmetric (f = 0);
  * a Dirichlet end with boundary value g and data equal to g near both ends equals the
    periodic mesh, as long as nothing reaches the ends;
  * Examples 6.5 and 6.8: the doubly conservative method matches the first-order
    2000-cell reference (the paper's reference solutions), while the method without
    double conservation does not (the figures of both examples);
  * the CFL maximum over the end faces has a closed form; MPP holds with boundaries.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import af_inputs as ai
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_column(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return np.array([float(line) for line in f if line.strip() and not line.startswith("#")])


def _np(state):
    return [np.asarray(a, dtype=np.float64) for a in state]


def _front(u, x, level=0.05):
    """right-most cell centre where u exceeds level"""
    return x[np.where(u > level)[0].max()]


# ---- Appendix A: constant kappa reduces to the doubly conservative scheme -------------

@pytest.mark.parametrize("flux", [("zero", ()), ("burgers", (0.5,)), ("linear", (1.0, 0.0))])
def test_nodc_equals_dc_for_constant_kappa(flux):
    sp = ai.Spec(dim=1, nx=41, flux=flux, diff=("const", (0.02,)), umin=0.0, umax=1.0, limiter=False)
    st = _np(ai.random_state_1d(sp, 5))
    tau = 0.4 * oracle.dt_cfl(sp, st[0])
    a = oracle.fe(sp, st, tau)
    b = oracle.fe(dataclasses.replace(sp, diffusion_form="nodc"), st, tau)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) < 1e-14


# ---- Appendix A: fourth order for a smooth, solution-dependent kappa ------------------

def _nodc_residuals(n):
    # a = 0.05 u + 0.04 u^2 + 0.02 u^3 -> kappa = 0.05 + 0.08 u + 0.06 u^2; f = 0
    sp = ai.Spec(dim=1, nx=n, x0=0.0, x1=2 * math.pi, flux=("zero", ()), diff=("cubic", (0.05, 0.04, 0.02)),
                 umin=-10.0, umax=10.0, limiter=False, diffusion_form="nodc")
    # exact point values; averages chosen so that the recovered centre value
    # (6 ub - u_{i-1/2} - u_{i+1/2}) / 4 is the exact u(x_i): the operators are then
    # applied to exact nodal values on every 5-point line
    xc = sp.x0 + (np.arange(n) + 0.5) * sp.dx
    P = 0.5 + 0.3 * np.sin(sp.x0 + (np.arange(n) + 1.0) * sp.dx)
    ub = (np.roll(P, 1) + 4.0 * (0.5 + 0.3 * np.sin(xc)) + P) / 6.0
    out = oracle.fe(sp, [ub, P], 1.0)
    return sp, out[0] - ub, out[1] - P


def _exact_flux(x):
    u = 0.5 + 0.3 * np.sin(x)
    ux = 0.3 * np.cos(x)
    return (0.05 + 0.08 * u + 0.06 * u * u) * ux


def _exact_div(x):
    u = 0.5 + 0.3 * np.sin(x)
    ux, uxx = 0.3 * np.cos(x), -0.3 * np.sin(x)
    k, dk = 0.05 + 0.08 * u + 0.06 * u * u, 0.08 + 0.12 * u
    return dk * ux * ux + k * uxx


def test_nodc_fourth_order_for_smooth_kappa():
    err_p, err_a = [], []
    for n in (16, 32, 64, 128):
        sp, rub, rp = _nodc_residuals(n)
        xf = sp.x0 + (np.arange(n) + 1.0) * sp.dx
        # point value: (kappa(u) u_x)_x at x_{i+1/2}
        err_p.append(np.max(np.abs(rp - _exact_div(xf))))
        # cell average: exact average of (kappa u_x)_x = face flux difference / h
        exact_avg = (_exact_flux(xf) - _exact_flux(xf - sp.dx)) / sp.dx
        err_a.append(np.max(np.abs(rub - exact_avg)))
    rp_ = [math.log2(err_p[k] / err_p[k + 1]) for k in range(3)]
    ra_ = [math.log2(err_a[k] / err_a[k + 1]) for k in range(3)]
    assert min(rp_) > 3.8, (err_p, rp_)
    assert min(ra_) > 3.8, (err_a, ra_)


# ---- outflow: even reflection == periodic mesh of twice the size, mirrored -------------

def _mirror(st):
    ub, pb = st  # pb: n+1 values u_{-1/2} .. u_{n-1/2}
    return [np.concatenate([ub, ub[::-1]]), np.concatenate([pb[1:], pb[::-1][1:]])]


@pytest.mark.parametrize("diff,blend", [(("pme", (2,)), "plain"), (("pwl", (0.05, 0.3, 0.08, 0.7)), "off"),
                                        (("ramp", (1.0, 0.5, 0.1)), "plain")])
def test_outflow_equals_mirrored_periodic(diff, blend):
    n = 24
    sp = ai.Spec(dim=1, nx=n, x0=0.0, x1=1.0, flux=("zero", ()), diff=diff, umin=0.0, umax=1.0,
                 limiter=True, blend=blend, bc="outflow")
    st = _np(ai.random_state_1d(sp, 11, lo=0.05, hi=0.95))
    per = dataclasses.replace(sp, nx=2 * n, x1=2.0, bc="periodic")
    sm = _mirror(st)
    assert sm[1].size == 2 * n
    dt = oracle.dt_cfl(sp, st[0])
    assert dt == pytest.approx(oracle.dt_cfl(per, sm[0]), rel=1e-15)
    a, b = st, sm
    for _ in range(3):
        a, _sa = oracle.step(sp, 3, a, dt)
        b, _sb = oracle.step(per, 3, b, dt)
    assert np.max(np.abs(a[0] - b[0][:n])) < 1e-13
    assert np.max(np.abs(a[1][1:] - b[1][:n])) < 1e-13
    assert abs(a[1][0] - b[1][-1]) < 1e-13
    # and the mirror image stays a mirror image
    assert np.max(np.abs(b[0][:n] - b[0][n:][::-1])) < 1e-13


# ---- Dirichlet: equals periodic while the ends keep the boundary value ----------------

@pytest.mark.parametrize("g", [0.0, 1.0, 0.3])
def test_dirichlet_equals_periodic_away_from_ends(g):
    n, pad = 60, 20
    sp = ai.Spec(dim=1, nx=n, x0=0.0, x1=1.0, flux=("burgers", (0.5,)), diff=("pwl", (0.05, 0.25, 0.05, 0.75)),
                 umin=0.0, umax=1.0, limiter=True, blend="plain", bc="dirichlet", bc_values=(g, g))
    st = _np(ai.random_state_1d(sp, 3))
    st[0][:pad] = g
    st[0][-pad:] = g
    st[1][:pad + 1] = g
    st[1][-pad - 1:] = g
    per = dataclasses.replace(sp, bc="periodic")
    sp_per = [st[0].copy(), st[1][1:].copy()]
    dt = oracle.dt_cfl(sp, st[0])
    assert dt == pytest.approx(oracle.dt_cfl(per, sp_per[0]), rel=1e-15)
    a, b = st, sp_per
    for _ in range(2):   # 2 steps x 3 stages x 3 cells of stencil reach < pad
        a, _ = oracle.step(sp, 3, a, dt)
        b, _ = oracle.step(per, 3, b, dt)
    assert np.max(np.abs(a[0] - b[0])) < 1e-14
    assert np.max(np.abs(a[1][1:] - b[1])) < 1e-14
    assert a[1][0] == g and a[1][-1] == g   # boundary point values held exactly


def test_dirichlet_end_face_sets_cfl():
    # interior at rest (u = 0), left boundary value 1: only the left end face moves,
    # alpha = |f'(1)| = 2 * 0.25 = 0.5 -> dt = C / (0.5 / h) without diffusion
    sp = ai.Spec(dim=1, nx=50, x0=-1.0, x1=1.0, flux=("burgers", (0.25,)), diff=("none", ()),
                 umin=0.0, umax=1.0, bc="dirichlet", bc_values=(1.0, 0.0))
    ub = np.zeros(50)
    assert oracle.dt_cfl(sp, ub, cfl=0.33) == pytest.approx(0.33 / (0.5 / sp.dx), rel=1e-14)
    per = dataclasses.replace(sp, bc="periodic")
    assert oracle.dt_cfl(per, ub, cfl=0.33) == math.inf


# ---- MPP with boundaries, both diffusion forms ------------------------------------------

@pytest.mark.parametrize("bc", ["dirichlet", "outflow"])
@pytest.mark.parametrize("form", ["dc", "nodc"])
def test_mpp_with_boundaries(bc, form):
    sp = ai.Spec(dim=1, nx=64, x0=0.0, x1=1.0, flux=("bl", (5.0,)), diff=("ramp", (0.05, 0.4, 0.2)),
                 umin=0.0, umax=1.0, limiter=True, bc=bc, bc_values=(1.0, 0.0), diffusion_form=form)
    st = _np(ai.random_state_1d(sp, 21))
    for _ in range(20):
        st, stats = oracle.step(sp, 3, st, oracle.dt_cfl(sp, st[0]))
        assert stats["error"] == 0
        lo, hi = oracle.bounds(st)
        assert lo >= 0.0 and hi <= 1.0


@pytest.mark.parametrize("form", ["dc", "nodc"])
def test_mpp_single_stage_adversarial(form):
    # averages in {0, 1/2, 1} and point values in {0, 1}: the high-order corrections are
    # as large as they get, and one limited forward-Euler stage at the CFL step must
    # still land in [0, 1] (half the limiter factor overshoots by ~0.09 here)
    rng = np.random.default_rng(0)
    for trial in range(120):
        flux = [("burgers", (0.5,)), ("bl", (5.0,)), ("zero", ())][trial % 3]
        sp = ai.Spec(dim=1, nx=32, flux=flux, diff=("ramp", (0.05, 0.4, 0.2)), limiter=True,
                     bc=["outflow", "dirichlet"][trial % 2], bc_values=(1.0, 0.0), diffusion_form=form)
        st = [rng.choice([0.0, 0.5, 1.0], 32), rng.choice([0.0, 1.0], 33)]
        st[1][0], st[1][-1] = (1.0, 0.0) if sp.bc == "dirichlet" else (st[1][0], st[1][-1])
        out = oracle.fe(sp, st, oracle.dt_cfl(sp, st[0], cfl_diff=-1.0))
        # up to round-off (the safeguard after each stage clamps up to 8 ulp)
        assert out[0].min() >= -1e-14 and out[0].max() <= 1.0 + 1e-14, trial
        assert out[1].min() >= 0.0 and out[1].max() <= 1.0, trial


# ---- the first-order reference scheme ---------------------------------------------------

def test_first_order_scheme_monotone_and_conservative():
    sp = ai.Spec(dim=1, nx=80, x0=0.0, x1=1.0, flux=("burgers", (0.5,)), diff=("pwl", (0.05, 0.25, 0.05, 0.75)),
                 umin=0.0, umax=1.0)
    ub0 = _np(ai.random_state_1d(sp, 8))[0]
    ub, n = oracle.first_order_run(sp, ub0, 0.05)
    assert n > 10
    assert ub.min() >= 0.0 and ub.max() <= 1.0
    assert abs(ub.sum() - ub0.sum()) < 1e-12


# ---- Examples 6.5 and 6.8: double conservation matters -----------------------------------

def test_example_6_5_double_conservation_matters():
    ref = _golden_column("evje_karlsen_first_order_2000.txt").reshape(200, 10).mean(axis=1)
    sp = ai.evje_karlsen(200)
    st = _np(ai.initial_state(sp))
    x = sp.x0 + (np.arange(200) + 0.5) * sp.dx
    dc, _, s1 = oracle.run_native(sp, 3, st, sp.T)
    nd, _, s2 = oracle.run_native(dataclasses.replace(sp, diffusion_form="nodc"), 3, st, sp.T)
    assert s1["error"] == 0 and s2["error"] == 0
    e_dc = np.abs(dc[0] - ref).sum() * sp.dx
    e_nd = np.abs(nd[0] - ref).sum() * sp.dx
    assert e_dc < 3e-3
    assert e_nd > 10 * e_dc
    # the wave front: doubly conservative within a cell of the reference, the other
    # method well behind it
    assert abs(_front(dc[0], x) - _front(ref, x)) <= sp.dx + 1e-12
    assert _front(ref, x) - _front(nd[0], x) > 5 * sp.dx
    assert min(dc[0].min(), dc[1].min()) >= 0.0 and max(dc[0].max(), dc[1].max()) <= 1.0


def test_example_6_8_double_conservation_matters():
    ref = _golden_column("strongly_degenerate_first_order_2000.txt").reshape(100, 20).mean(axis=1)
    sp = ai.strongly_degenerate_1d(100)
    st = _np(ai.initial_state(sp))
    x = sp.x0 + (np.arange(100) + 0.5) * sp.dx
    near = np.abs(x) < 0.3
    dc, _, _ = oracle.run_native(sp, 3, st, sp.T)
    nd, _, _ = oracle.run_native(dataclasses.replace(sp, blend="off", limiter=False, diffusion_form="nodc"),
                                 3, st, sp.T)
    e_dc = np.abs(dc[0] - ref)
    e_nd = np.abs(nd[0] - ref)
    assert e_dc.sum() * sp.dx < 0.02
    assert e_dc[near].sum() * sp.dx < 0.01
    # the method without double conservation (and without limiting) departs from the
    # reference at the interface x = 0
    assert e_nd[near].sum() * sp.dx > 10 * e_dc[near].sum() * sp.dx
    assert min(dc[0].min(), dc[1].min()) >= -1.0 and max(dc[0].max(), dc[1].max()) <= 1.0
