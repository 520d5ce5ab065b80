"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 form: relative max-norm difference <= 1e-12 (the tolerance the method's
spec target states), element by element, on seeded inputs that span several
32 x 8 tiles with a ragged tail; full-size workloads are checked on sampled cells whose
dependence cone is evaluated by the oracle on a local periodic window, and through
size-independent properties (conservation, exact bounds, symmetry).
"""
import math

import numpy as np
import pytest
import torch

import af_inputs as ai
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_11527_gb300 import build
    build.build()


def solver(spec, prec="fp64", rk=3, **kw):
    from paper_2510_11527_gb300 import Solver
    return Solver(spec, precision=prec, rk=rk, **kw)


def relerr(a, b):
    a = [np.asarray(x, dtype=np.float64) for x in a]
    b = [np.asarray(x, dtype=np.float64) for x in b]
    scale = max(max(np.max(np.abs(x)) for x in b), 1e-300)
    return max(np.max(np.abs(x - y)) for x, y in zip(a, b)) / scale


def np_state(st):
    return [np.asarray(a.cpu() if torch.is_tensor(a) else a, dtype=np.float64) for a in st]


PROBLEMS_2D = {
    "burgers_pwl": dict(flux=("burgers", (0.5,)), diff=("pwl", (0.0, 0.0, 0.1, 0.5)), umin=-1.0, umax=1.0),
    "bl_cubic": dict(flux=("bl", (5.0,)), diff=("cubic", (0.0, 0.02, -0.04 / 3)), umin=0.0, umax=1.0),
    "pme": dict(flux=("zero", ()), diff=("pme", (2,)), umin=0.0, umax=1.0),
    "linear": dict(flux=("linear", (1.0, -0.6)), diff=("const", (0.01,)), umin=-2.0, umax=2.0),
    "burgers_band": dict(flux=("burgers", (0.5,)), diff=("pwl", (0.03, 0.25, 0.03, 0.75)), umin=0.0, umax=1.0),
    # pure convection: the face limiter factor is 2d = 4 (no potential corrections)
    "burgers_none": dict(flux=("burgers", (0.5,)), diff=("none", ()), umin=-1.0, umax=1.0),
    "bl_none": dict(flux=("bl", (5.0,)), diff=("none", ()), umin=0.0, umax=1.0),
}


def spec2d(name, nx, ny, limiter=True, blend="off", x1=1.3, y1=0.9):
    return ai.Spec(dim=2, nx=nx, ny=ny, x0=0.0, x1=x1, y0=0.0, y1=y1, limiter=limiter, blend=blend,
                   **PROBLEMS_2D[name])


# ----------------------------------------------------------------------------------
# one forward-Euler evaluation

@pytest.mark.parametrize("name", list(PROBLEMS_2D))
@pytest.mark.parametrize("limiter,blend", [(True, "off"), (False, "off"), (True, "plain")])
def test_forward_euler_2d_fp64(name, limiter, blend):
    spec = spec2d(name, 70, 45, limiter=limiter, blend=blend)
    st = np_state(ai.random_state_2d(spec, seed=7))
    tau = oracle.dt_cfl(spec, st[0])
    want = oracle.fe(spec, st, tau)
    with solver(spec) as s:
        s.set_state(st)
        s.forward_euler(tau)
        got = s.get_state()
    assert relerr(got, want) <= TOL64


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 2), (5, 9), (32, 8), (33, 9), (64, 16), (100, 3)])
def test_forward_euler_2d_shapes(nx, ny):
    spec = spec2d("burgers_pwl", nx, ny)
    st = np_state(ai.random_state_2d(spec, seed=nx * 100 + ny))
    tau = oracle.dt_cfl(spec, st[0])
    want = oracle.fe(spec, st, tau)
    with solver(spec) as s:
        s.set_state(st)
        s.forward_euler(tau)
        got = s.get_state()
    assert relerr(got, want) <= TOL64


def test_forward_euler_external_indicator():
    spec = spec2d("bl_cubic", 40, 24, blend="external")
    st = np_state(ai.random_state_2d(spec, seed=3))
    sx = np.random.default_rng(1).uniform(0, 2, size=(24, 40))
    tau = oracle.dt_cfl(spec, st[0])
    want = oracle.fe(spec, st, tau, s_ext=sx)
    with solver(spec) as s:
        s.set_state(st)
        s.set_indicator(sx)
        s.forward_euler(tau)
        got = s.get_state()
    assert relerr(got, want) <= TOL64


# ----------------------------------------------------------------------------------
# full RK steps

@pytest.mark.parametrize("rk", [3, 54])
@pytest.mark.parametrize("name,blend", [("burgers_pwl", "off"), ("bl_cubic", "plain"), ("pme", "off")])
def test_rk_steps_2d_fp64(rk, name, blend):
    spec = spec2d(name, 48, 40, blend=blend)
    spec.rk = rk
    st = np_state(ai.random_state_2d(spec, seed=21))
    with solver(spec, rk=rk) as s:
        s.set_state(st)
        ref = [a.copy() for a in st]
        for _ in range(4):
            dt = oracle.dt_cfl(spec, ref[0])
            ref, stats = oracle.step(spec, rk, ref, dt)
            assert stats["error"] == 0
            s.step(dt)
        got = s.get_state()
        assert s.stats()["errors"] == 0
    assert relerr(got, ref) <= TOL64


def test_device_cfl_step_matches_oracle():
    for name in ["burgers_pwl", "bl_cubic", "pme"]:
        spec = spec2d(name, 50, 30)
        st = np_state(ai.random_state_2d(spec, seed=5))
        with solver(spec) as s:
            s.set_state(st)
            assert s.dt_cfl() == pytest.approx(oracle.dt_cfl(spec, st[0]), rel=1e-14)


def test_run_to_time_config2_small():
    spec = ai.config2(48)
    st = np_state(ai.initial_state(spec))
    T = 0.05
    ref, nref, _ = oracle.run(spec, 3, st, T)
    with solver(spec) as s:
        s.set_state(st)
        n = s.run(T)
        assert s.time() == pytest.approx(T, rel=1e-14)
        got = s.get_state()
        lo, hi = s.bounds()
        assert s.stats()["errors"] == 0
    assert n == nref
    assert relerr(got, ref) <= TOL64
    assert lo >= -1.0 and hi <= 1.0


# ----------------------------------------------------------------------------------
# 1D

def test_config1_linear_1d_matches_oracle_and_exact():
    spec = ai.config1(128)
    st = np_state(ai.sine_1d_state(spec))
    dt = ai.config1_dt(spec)
    ref, n, _ = oracle.run(spec, 3, st, 1.0, dt_fixed=dt)
    with solver(spec) as s:
        s.set_state(st)
        t = 0.0
        while t < 1.0 * (1 - 1e-14):
            d = min(dt, 1.0 - t)
            s.step(d)
            t += d
        got = s.get_state()
    assert relerr(got, ref) <= TOL64
    i = np.arange(128)
    ex = np.exp(-0.01) * np.sin((i + 1.0) * spec.dx - 1.0)
    assert np.max(np.abs(got[1] - ex)) < 1e-4


@pytest.mark.parametrize("n", [3, 7, 256, 257, 1000])
@pytest.mark.parametrize("lim,blend", [(True, "off"), (True, "plain"), (False, "off")])
@pytest.mark.parametrize("diff", [("pwl", (0.1, -0.25, 0.1, 0.25)), ("none", ())])
def test_forward_euler_1d(n, lim, blend, diff):
    spec = ai.Spec(dim=1, nx=n, x0=-2, x1=2, flux=("burgers", (1.0,)), diff=diff,
                   umin=-1.0, umax=1.0, limiter=lim, blend=blend)
    st = np_state(ai.random_state_1d(spec, seed=n))
    tau = oracle.dt_cfl(spec, st[0])
    want = oracle.fe(spec, st, tau)
    with solver(spec) as s:
        s.set_state(st)
        s.forward_euler(tau)
        got = s.get_state()
    assert relerr(got, want) <= TOL64


@pytest.mark.parametrize("rk", [3, 54])
def test_rk_steps_1d_bl(rk):
    spec = ai.Spec(dim=1, nx=300, x0=0, x1=1, flux=("bl", (5.0,)), diff=("cubic", (0.0, 0.02, -0.04 / 3)),
                   umin=0.0, umax=1.0, limiter=True, blend="plain", rk=rk)
    st = np_state(ai.random_state_1d(spec, seed=4))
    ref = [a.copy() for a in st]
    with solver(spec, rk=rk) as s:
        s.set_state(st)
        for _ in range(5):
            dt = oracle.dt_cfl(spec, ref[0])
            ref, _ = oracle.step(spec, rk, ref, dt)
            s.step(dt)
        got = s.get_state()
    assert relerr(got, ref) <= TOL64


# ----------------------------------------------------------------------------------
# invariants on the GPU at any size

def test_mass_conservation_and_exact_bounds_fp64():
    spec = ai.config2(256)
    st = np_state(ai.initial_state(spec))
    with solver(spec) as s:
        s.set_state(st)
        m0 = s.mass()
        for _ in range(20):
            s.step(0.0)
        m1 = s.mass()
        lo, hi = s.bounds()
        stt = s.stats()
    scale = np.sum(np.abs(st[0])) * spec.dx * spec.dy
    assert abs(m1 - m0) <= 20 * 4e-15 * scale
    assert lo >= -1.0 and hi <= 1.0
    assert stt["errors"] == 0


def test_constant_state_and_zero_step():
    spec = ai.config2(40)
    st = [np.full((40, 40), 0.25) for _ in range(4)]
    with solver(spec) as s:
        s.set_state(st)
        s.step(1e-3)
        got = s.get_state()
        assert np.array_equal(got[0], st[0])
        s.step(0.0)
        s2 = s.get_state()
    for a in s2[1:]:
        np.testing.assert_allclose(a, 0.25, rtol=0, atol=1e-15)


def test_transpose_symmetry_gpu():
    spec = ai.Spec(dim=2, nx=64, ny=64, flux=("burgers", (0.5,)), diff=("pwl", (0.0, 0.0, 0.1, 0.5)),
                   umin=-1.0, umax=1.0, limiter=True, blend="plain")
    ub, V, X, Y = np_state(ai.random_state_2d(spec, seed=2, lo=-1, hi=1))
    tau = oracle.dt_cfl(spec, ub)
    with solver(spec) as s:
        s.set_state([ub, V, X, Y])
        s.forward_euler(tau)
        a = s.get_state()
        s.set_state([ub.T.copy(), V.T.copy(), Y.T.copy(), X.T.copy()])
        s.forward_euler(tau)
        b = s.get_state()
    for x, y in [(b[0], a[0].T), (b[1], a[1].T), (b[2], a[3].T), (b[3], a[2].T)]:
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-14)


def test_shift_equivariance_bitwise_gpu():
    spec = ai.config2(96)
    st = np_state(ai.random_state_2d(spec, seed=8, lo=-1, hi=1))
    sh = lambda z: np.roll(np.roll(z, 32, axis=1), -8, axis=0)   # whole tiles: same arithmetic
    with solver(spec) as s:
        s.set_state(st)
        s.step(1e-4)
        a = s.get_state()
        s.set_state([sh(z) for z in st])
        s.step(1e-4)
        b = s.get_state()
    for x, y in zip(a, b):
        assert np.array_equal(sh(x), y)


# ----------------------------------------------------------------------------------
# full-size workloads: sampled cells against the oracle on local periodic windows

def _window(arrs, j, i, r):
    ny, nx = arrs[0].shape
    jj = (np.arange(j - r, j + r + 1) % ny)[:, None]
    ii = (np.arange(i - r, i + r + 1) % nx)[None, :]
    return [a[jj, ii] for a in arrs]


def _sampled_step_check(spec, st, dt, got, rk, samples, rng, r=8, tol=TOL64):
    """Compare sampled cells of one full RK step with the oracle on (2r+1)^2 windows.
    One stage reads +-2 (+-3 with blend) cells, so an SSP-RK3 step depends on +-9 at most;
    the window size makes the periodic wrap of the window invisible at its centre."""
    ny, nx = st[0].shape
    worst = 0.0
    sub = ai.Spec(**{**spec.__dict__, "nx": 2 * r + 1, "ny": 2 * r + 1,
                     "x1": spec.x0 + (2 * r + 1) * spec.dx, "y1": spec.y0 + (2 * r + 1) * spec.dy})
    scale = max(np.max(np.abs(a)) for a in st)
    u = st[0]
    rough = np.argwhere((u != np.roll(u, 1, 0)) | (u != np.roll(u, 1, 1)) | (u != np.roll(u, -1, 0)) |
                        (u != np.roll(u, -1, 1)))
    for k in range(samples):
        if k % 2 == 0 and len(rough):
            j, i = (int(v) for v in rough[rng.integers(len(rough))])
        else:
            j, i = int(rng.integers(ny)), int(rng.integers(nx))
        win = _window(st, j, i, r)
        out, _ = oracle.step(sub, rk, win, dt)
        for a_ref, a_got in zip(out, got):
            worst = max(worst, abs(a_ref[r, r] - a_got[j, i]) / scale)
    assert worst <= tol


@pytest.mark.parametrize("prec", ["fp64"])
def test_config2_full_size_sampled(prec):
    spec = ai.config2(1024)
    st = np_state(ai.initial_state(spec, device="cuda"))
    with solver(spec, prec) as s:
        s.set_state(st)
        dt = s.dt_cfl()
        assert dt == pytest.approx(oracle.dt_cfl(spec, st[0]), rel=1e-14)
        s.step(dt)
        got = s.get_state()
        lo, hi = s.bounds()
    assert lo >= -1.0 and hi <= 1.0
    rng = np.random.default_rng(0)
    # half the samples on the disc edges, where the limiter acts
    _sampled_step_check(spec, st, dt, got, 3, 60, rng, r=10)


@pytest.mark.parametrize("pattern", ["checker", "stripes_x", "stripes_y"])
def test_device_cfl_step_interior_extrema(pattern):
    """Buckley-Leverett: |f_l'| vanishes at u = 0 and u = 1, so on a 0/1 pattern every
    face's interval wave speed comes from the interior extrema of f_l' (the flagged
    path of the reduction); stripes exercise one direction at a time."""
    spec = spec2d("bl_cubic", 40, 24)
    j, i = np.meshgrid(np.arange(spec.ny), np.arange(spec.nx), indexing="ij")
    ub = {"checker": (i + j) % 2, "stripes_x": i % 2, "stripes_y": j % 2}[pattern].astype(np.float64)
    st = [ub, np.zeros_like(ub), np.zeros_like(ub), np.zeros_like(ub)]
    with solver(spec) as s:
        s.set_state(st)
        assert s.dt_cfl() == pytest.approx(oracle.dt_cfl(spec, ub), rel=1e-14)


def test_forward_euler_tall_mesh():
    """A mesh with more than 65535 tile rows (8 x 600000 cells): the stage grid is linear
    in the tile index, so any aspect ratio launches."""
    spec = spec2d("burgers_pwl", 8, 600000, x1=0.05, y1=600.0)
    st = np_state(ai.random_state_2d(spec, seed=11))
    tau = oracle.dt_cfl(spec, st[0])
    want = oracle.fe(spec, st, tau)
    with solver(spec) as s:
        s.set_state(st)
        s.forward_euler(tau)
        got = s.get_state()
    assert relerr(got, want) <= TOL64


def test_run_is_idempotent_at_its_end_time():
    """af_run issues steps in chunks and clips on the device: a second run to the same
    time takes no step and leaves the state unchanged; a later end time continues."""
    spec = ai.config2(40)
    st = np_state(ai.initial_state(spec))
    with solver(spec) as s:
        s.set_state(st)
        n1 = s.run(0.02)
        a = s.get_state()
        assert s.run(0.02) == 0
        b = s.get_state()
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
        n2 = s.run(0.03)
        assert n1 > 0 and n2 > 0 and s.time() == pytest.approx(0.03, rel=1e-14)
        assert s.stats()["errors"] == 0
