"""Parity of the 3D CUDA path with the FP64 oracle (Section 4's 3D DoFs, Section 5.2
with d = 3), through the C ABI's array-form state calls.

FP64: relative max-norm difference <= 1e-12 on all 8 arrays, on meshes from 4^3 to
odd, unequal sizes spanning several 256-thread blocks; forward Euler, SSP-RK3 and
SSP-RK(5,4) steps, the device CFL step, and a porous-medium run from the 3D Barenblatt
profile (mass conserved, bounds exact).
"""
import numpy as np
import pytest

import af_inputs as ai
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_11527_gb300 import build
    build.build()


def solver(spec, rk=3, prec="fp64", **kw):
    from paper_2510_11527_gb300 import Solver
    return Solver(spec, precision=prec, rk=rk, **kw)


def relerr(a, b):
    a = [np.asarray(x, dtype=np.float64) for x in a]
    b = [np.asarray(x, dtype=np.float64) for x in b]
    assert all(x.shape == y.shape for x, y in zip(a, b))
    scale = max(max(np.max(np.abs(x)) for x in b), 1e-300)
    return max(np.max(np.abs(x - y)) for x, y in zip(a, b)) / scale


MODELS = {
    "burgers_pwl": dict(flux=("burgers", (0.5,)), diff=("pwl", (0.05, 0.25, 0.05, 0.75))),
    "linear_const": dict(flux=("linear", (1.0, -0.6, 0.3)), diff=("const", (0.01,))),
    "pme": dict(flux=("zero", ()), diff=("pme", (2,))),
    "burgers_ramp": dict(flux=("burgers", (0.5,)), diff=("ramp", (0.05, 0.4, 0.2))),
    # pure convection: face limiter factor 2d = 6
    "burgers_none": dict(flux=("burgers", (0.5,)), diff=("none", ())),
}


def box(name, n, limiter=True, blend="off"):
    return ai.Spec(dim=3, nx=n[0], ny=n[1], nz=n[2], x0=0.0, x1=1.3, y0=0.0, y1=0.9, z0=0.0, z1=0.7, umin=0.0,
                   umax=1.0, limiter=limiter, blend=blend, **MODELS[name])


@pytest.mark.parametrize("n", [(4, 4, 4), (5, 3, 7), (9, 8, 6), (17, 16, 3)])
@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("limiter,blend", [(True, "off"), (False, "off"), (True, "plain")])
def test_forward_euler_3d(n, name, limiter, blend):
    spec = box(name, n, limiter, blend)
    st = [a.numpy() for a in ai.random_state_3d(spec, seed=sum(n))]
    tau = oracle.dt_cfl(spec, st[0])
    want = oracle.fe(spec, st, tau)
    with solver(spec) as s:
        s.set_state(st)
        s.forward_euler(tau)
        got = s.get_state()
    assert relerr(got, want) <= TOL64


@pytest.mark.parametrize("rk", [3, 54])
@pytest.mark.parametrize("name,blend", [("burgers_pwl", "plain"), ("linear_const", "off")])
def test_rk_steps_3d(rk, name, blend):
    spec = box(name, (12, 10, 9), blend=blend)
    spec.rk = rk
    st = [a.numpy() for a in ai.random_state_3d(spec, seed=3)]
    ref = [a.copy() for a in st]
    with solver(spec, rk=rk) as s:
        s.set_state(st)
        for _ in range(3):
            dt = oracle.dt_cfl(spec, ref[0])
            ref, stats = oracle.step(spec, rk, ref, dt)
            assert stats["error"] == 0
            s.step(dt)
        got = s.get_state()
        assert s.stats()["errors"] == 0
    assert relerr(got, ref) <= TOL64


@pytest.mark.parametrize("name", ["burgers_pwl", "linear_const"])
def test_device_cfl_3d(name):
    spec = box(name, (11, 7, 5))
    st = [a.numpy() for a in ai.random_state_3d(spec, seed=5)]
    with solver(spec) as s:
        s.set_state(st)
        assert s.dt_cfl() == pytest.approx(oracle.dt_cfl(spec, st[0]), rel=1e-14)


def test_pme_3d_barenblatt_run():
    spec = ai.pme_3d(24)
    st = [a.numpy() for a in ai.initial_state(spec, sub=2, order=3)]
    ref, nref, stats = oracle.run(spec, 3, st, 0.05)
    assert stats["error"] == 0
    with solver(spec) as s:
        s.set_state(st)
        n = s.run(0.05)
        got = s.get_state()
        lo, hi = s.bounds()
        mass = s.mass()
    assert n == nref
    assert relerr(got, ref) <= TOL64
    assert lo >= 0.0 and hi <= 1.0
    assert mass == pytest.approx(float(np.sum(st[0])) * spec.dx * spec.dy * spec.dz, rel=1e-13)


def test_state_io_3d():
    spec = box("burgers_pwl", (6, 5, 4))
    st = [a.numpy() for a in ai.random_state_3d(spec, seed=8, lo=0.2, hi=0.7)]
    st[5][1, 2, 3], st[7][3, 4, 5] = 0.1, 0.9
    with solver(spec) as s:
        s.set_state(st)
        got = s.get_state()
        assert all(np.array_equal(a, b) for a, b in zip(got, st))
        assert s.bounds() == (0.1, 0.9)
        views = s.device_tensors()
        assert len(views) == 8 and all(tuple(v.shape) == (4, 5, 6) for v in views)


def test_3d_rejects_what_it_does_not_support():
    from paper_2510_11527_gb300 import AfError, Solver
    bad = [dict(flux=("bl", (5.0,))), dict(blend="external"), dict(diffusion_form="nodc"), dict(bc="outflow")]
    for kw in bad:
        spec = box("burgers_pwl", (6, 6, 6))
        for k, v in kw.items():
            setattr(spec, k, v)
        with pytest.raises(AfError):
            solver(spec)


@pytest.mark.parametrize("name,blend", [("burgers_pwl", "plain"), ("linear_const", "off"), ("pme", "off")])
def test_fp32_mixed_3d_vs_oracle(name, blend):
    spec = box(name, (13, 9, 6), blend=blend)
    st = [a.numpy() for a in ai.random_state_3d(spec, seed=11)]
    tau = oracle.dt_cfl(spec, st[0])
    want = oracle.fe(spec, st, tau)
    with solver(spec, prec="fp32_mixed") as s:
        s.set_state(st)
        s.forward_euler(tau)
        got = s.get_state()
        lo, hi = s.bounds()
    assert max(np.max(np.abs(g - w)) for g, w in zip(got, want)) <= 1e-5
    assert max(np.mean(np.abs(g - w)) for g, w in zip(got, want)) <= 1e-6
    assert lo >= 0.0 and hi <= 1.0


def test_fp32_mixed_3d_run_vs_fp64():
    spec = ai.pme_3d(20)
    st = [a.numpy() for a in ai.initial_state(spec, sub=2, order=3)]
    res = {}
    for prec in ("fp64", "fp32_mixed"):
        with solver(spec, prec=prec) as s:
            s.set_state(st)
            s.run(0.03)
            res[prec] = (s.get_state(), s.mass(), s.bounds(), s.stats())
    (g64, m64, _, _), (g32, m32, (lo, hi), stats) = res["fp64"], res["fp32_mixed"]
    assert stats["errors"] == 0 and lo >= 0.0 and hi <= 1.0
    assert m32 == pytest.approx(float(np.sum(st[0])) * spec.dx * spec.dy * spec.dz, rel=1e-12)
    assert max(np.mean(np.abs(a - b)) for a, b in zip(g32, g64)) < 1e-6


def test_fp32_mixed_3d_state_io():
    spec = box("burgers_pwl", (6, 5, 4))
    st = [a.numpy() for a in ai.random_state_3d(spec, seed=8)]
    with solver(spec, prec="fp32_mixed") as s:
        s.set_state(st)
        got = s.get_state()
        views = s.device_tensors()
    assert np.array_equal(got[0], st[0])
    for a, b in zip(got[1:], st[1:]):
        assert np.array_equal(a, b.astype(np.float32).astype(np.float64))
    assert str(views[0].dtype) == "torch.float64" and str(views[1].dtype) == "torch.float32"
