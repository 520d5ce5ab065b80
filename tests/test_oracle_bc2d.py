"""Pins of the oracle's 2D rectangle with outflow ends (the ends of the paper's 2D
Examples 6.7 and 6.9; their discrete form is the even reflection of every DoF kind):

  * with f = 0 the scheme is mirror-symmetric, so the rectangle equals the periodic mesh
    of twice its size in each direction holding the data mirrored about both sides;
  * data independent of y (of x) reduce the 2D scheme to the 1D scheme of the pinned
    1D outflow interval, as on periodic meshes;
  * MPP holds for one limited stage from adversarial data at the CFL step.
"""
import dataclasses

import numpy as np
import pytest

import af_inputs as ai
import oracle


def _np(st):
    return [np.asarray(a, dtype=np.float64) for a in st]


def _even_periodic(st, nx, ny):
    """the rectangle's DoFs evenly extended to the periodic mesh of 2nx x 2ny cells"""
    ub, V, X, Y = st
    ci = lambda i, n: np.where(i % (2 * n) < n, i % (2 * n), 2 * n - 1 - i % (2 * n))
    fk = lambda k, n: np.where(k % (2 * n) <= n, k % (2 * n), 2 * n - k % (2 * n))
    I = np.arange(2 * nx)
    J = np.arange(2 * ny)
    cI, cJ = ci(I, nx), ci(J, ny)
    fI, fJ = fk(I + 1, nx), fk(J + 1, ny)
    return [ub[np.ix_(cJ, cI)], V[np.ix_(fJ, fI)], X[np.ix_(cJ, fI)], Y[np.ix_(fJ, cI)]]


@pytest.mark.parametrize("diff,blend", [(("pme", (2,)), "plain"), (("pwl", (0.05, 0.3, 0.08, 0.7)), "off"),
                                        (("ramp", (0.5, 0.5, 0.1)), "plain")])
def test_outflow_rectangle_equals_mirrored_periodic(diff, blend):
    nx, ny = 11, 8
    sp = ai.Spec(dim=2, nx=nx, ny=ny, x0=0.0, x1=1.1, y0=0.0, y1=0.7, flux=("zero", ()), diff=diff,
                 umin=0.0, umax=1.0, limiter=True, blend=blend, bc="outflow")
    st = _np(ai.random_state_2d(sp, 13, lo=0.05, hi=0.95))
    per = dataclasses.replace(sp, nx=2 * nx, ny=2 * ny, x1=2.2, y1=1.4, bc="periodic")
    sm = _even_periodic(st, nx, ny)
    dt = oracle.dt_cfl(sp, st[0])
    assert dt == pytest.approx(oracle.dt_cfl(per, sm[0]), rel=1e-15)
    a, b = st, sm
    for _ in range(2):
        a, sa = oracle.step(sp, 3, a, dt)
        b, sb = oracle.step(per, 3, b, dt)
        assert sa["error"] == 0 and sb["error"] == 0
    kx = (np.arange(nx + 1) - 1) % (2 * nx)
    ky = (np.arange(ny + 1) - 1) % (2 * ny)
    assert np.max(np.abs(a[0] - b[0][:ny, :nx])) < 1e-13
    assert np.max(np.abs(a[1] - b[1][np.ix_(ky, kx)])) < 1e-13
    assert np.max(np.abs(a[2] - b[2][np.ix_(np.arange(ny), kx)])) < 1e-13
    assert np.max(np.abs(a[3] - b[3][np.ix_(ky, np.arange(nx))])) < 1e-13


@pytest.mark.parametrize("flux", [("linear", (0.8, 0.3)), ("burgers", (0.5,))])
@pytest.mark.parametrize("axis", [0, 1])
def test_outflow_rectangle_reduces_to_1d_outflow(flux, axis):
    n, m = 12, 5
    rng = np.random.default_rng(7)
    ub1 = rng.uniform(-0.5, 0.5, n)
    P1 = rng.uniform(-0.5, 0.5, n + 1)
    c1 = (6 * ub1 - P1[:-1] - P1[1:]) / 4
    tau = 1e-3
    if axis == 0:   # data independent of y, compared with the 1D scheme in x
        s1 = ai.Spec(dim=1, nx=n, x0=0, x1=1.3, flux=flux, diff=("const", (0.02,)), umin=-9, umax=9,
                     limiter=False, bc="outflow")
        s2 = ai.Spec(dim=2, nx=n, ny=m, x0=0, x1=1.3, y0=0, y1=0.7, flux=flux, diff=("const", (0.02,)),
                     umin=-9, umax=9, limiter=False, bc="outflow")
        nb1, nP1 = oracle.fe(s1, [ub1, P1], tau)
        rows = lambda a, k: np.tile(a[None, :], (k, 1))
        out = oracle.fe(s2, [rows(ub1, m), rows(P1, m + 1), rows(P1, m), rows(c1, m + 1)], tau)
        np.testing.assert_allclose(out[0], rows(nb1, m), rtol=0, atol=1e-13)
        np.testing.assert_allclose(out[1], rows(nP1, m + 1), rtol=0, atol=1e-13)
        np.testing.assert_allclose(out[2], rows(nP1, m), rtol=0, atol=1e-13)
    else:           # data independent of x, compared with the 1D scheme in y (f2 = p1 u or u^2/2)
        f1d = ("linear", (flux[1][1], 0.0)) if flux[0] == "linear" else flux
        s1 = ai.Spec(dim=1, nx=n, x0=0, x1=0.7, flux=f1d, diff=("const", (0.02,)), umin=-9, umax=9,
                     limiter=False, bc="outflow")
        s2 = ai.Spec(dim=2, nx=m, ny=n, x0=0, x1=1.3, y0=0, y1=0.7, flux=flux, diff=("const", (0.02,)),
                     umin=-9, umax=9, limiter=False, bc="outflow")
        nb1, nP1 = oracle.fe(s1, [ub1, P1], tau)
        cols = lambda a, k: np.tile(a[:, None], (1, k))
        out = oracle.fe(s2, [cols(ub1, m), cols(P1, m + 1), cols(c1, m + 1), cols(P1, m)], tau)
        np.testing.assert_allclose(out[0], cols(nb1, m), rtol=0, atol=1e-13)
        np.testing.assert_allclose(out[1], cols(nP1, m + 1), rtol=0, atol=1e-13)
        np.testing.assert_allclose(out[3], cols(nP1, m), rtol=0, atol=1e-13)


def test_outflow_rectangle_mpp_adversarial():
    rng = np.random.default_rng(1)
    for trial in range(40):
        flux = [("burgers", (0.5,)), ("bl", (5.0,))][trial % 2]
        sp = ai.Spec(dim=2, nx=9, ny=7, x0=0, x1=0.9, y0=0, y1=0.7, flux=flux, diff=("ramp", (0.05, 0.4, 0.2)),
                     limiter=True, blend=["off", "plain"][(trial // 2) % 2], bc="outflow")
        st = [rng.choice([0.0, 0.5, 1.0], (7, 9)), rng.choice([0.0, 1.0], (8, 10)), rng.choice([0.0, 1.0], (7, 10)),
              rng.choice([0.0, 1.0], (8, 9))]
        out = oracle.fe(sp, st, oracle.dt_cfl(sp, st[0], cfl_diff=-1.0))
        assert out[0].min() >= -1e-14 and out[0].max() <= 1.0 + 1e-14, trial
        for a in out[1:]:
            assert a.min() >= 0.0 and a.max() <= 1.0, trial


def test_examples_6_7_and_6_9_stay_in_bounds_and_symmetric():
    # Example 6.9: the data are antisymmetric under (x, y, u) -> (-x, -y, -u) and so is
    # f = u^2 with the odd band potential; the rectangle and its ends keep it
    sp = ai.strongly_degenerate_2d(24)
    st = _np(ai.initial_state(sp))
    u, n, stats = oracle.run(sp, 3, st, 0.05)
    assert stats["error"] == 0 and n > 5
    assert np.max(np.abs(u[0] + u[0][::-1, ::-1])) < 1e-12
    assert np.max(np.abs(u[1] + u[1][::-1, ::-1])) < 1e-12
    lo, hi = oracle.bounds(u)
    assert lo >= -1.0 and hi <= 1.0
    sp = ai.buckley_leverett_2d_outflow(24)
    st = _np(ai.initial_state(sp))
    u, n, stats = oracle.run(sp, 3, st, 0.02)
    assert stats["error"] == 0
    lo, hi = oracle.bounds(u)
    assert lo >= 0.0 and hi <= 1.0
