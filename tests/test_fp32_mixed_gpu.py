"""FP32-mixed form: FP32 point values and stencil/limiter arithmetic, FP64 cell
averages and update. Its results are stated as L1 / L-infinity differences from the FP64
path (itself parity-checked against the oracle); the MPP bounds must hold exactly and
mass stays conserved to FP64 round-off because the cell-average update and its
telescoping flux differences are formed in FP64."""
import numpy as np
import pytest

import af_inputs as ai
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_11527_gb300 import build
    build.build()


def solver(spec, prec, rk=3):
    from paper_2510_11527_gb300 import Solver
    return Solver(spec, precision=prec, rk=rk)


def l1(a, b):
    return max(float(np.mean(np.abs(np.asarray(x) - np.asarray(y)))) for x, y in zip(a, b))


def linf(a, b):
    return max(float(np.max(np.abs(np.asarray(x) - np.asarray(y)))) for x, y in zip(a, b))


@pytest.mark.parametrize("name,flux,diff,lo,hi,blend", [
    ("burgers", ("burgers", (0.5,)), ("pwl", (0.0, 0.0, 0.1, 0.5)), -1.0, 1.0, "off"),
    ("bl", ("bl", (5.0,)), ("cubic", (0.0, 0.02, -0.04 / 3)), 0.0, 1.0, "plain"),
    ("pme", ("zero", ()), ("pme", (2,)), 0.0, 1.0, "off"),
])
def test_fp32_forward_euler_vs_oracle(name, flux, diff, lo, hi, blend):
    spec = ai.Spec(dim=2, nx=70, ny=45, x0=0, x1=1.3, y0=0, y1=0.9, flux=flux, diff=diff, umin=lo, umax=hi,
                   limiter=True, blend=blend)
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=7)]
    tau = oracle.dt_cfl(spec, st[0])
    want = oracle.fe(spec, st, tau)
    with solver(spec, "fp32_mixed") as s:
        s.set_state(st)
        s.forward_euler(tau)
        got = s.get_state()
    scale = max(abs(lo), abs(hi))
    assert linf(got, want) <= 1e-5 * scale
    assert l1(got, want) <= 1e-6 * scale


def test_fp32_config2_1024_l1_vs_fp64_and_bounds():
    """Target of the FP32 form: L1 difference <= 1e-5 from FP64 at 1024^2."""
    spec = ai.config2(1024)
    st = [a.cpu().numpy() for a in ai.initial_state(spec, device="cuda")]
    res = {}
    for prec in ("fp64", "fp32_mixed"):
        with solver(spec, prec) as s:
            s.set_state(st)
            m0 = s.mass()
            for _ in range(10):
                s.step(0.0)
            res[prec] = s.get_state()
            lo, hi = s.bounds()
            assert lo >= -1.0 and hi <= 1.0
            stats = s.stats()
            assert stats["errors"] == 0
            scale = np.sum(np.abs(st[0])) * spec.dx * spec.dy
            # conservation holds to FP64 round-off plus the (counted) mass the safeguard
            # clamps of cell averages moved
            assert abs(s.mass() - m0) <= 1e-13 * scale + stats["mass_adjust"]
    e1 = l1(res["fp32_mixed"], res["fp64"])
    assert e1 <= 1e-5, e1


def test_fp32_1d_config1_accuracy():
    spec = ai.config1(128)
    st = [a.numpy() for a in ai.sine_1d_state(spec)]
    dt = ai.config1_dt(spec)
    with solver(spec, "fp32_mixed") as s:
        s.set_state(st)
        t = 0.0
        while t < 1.0 - 1e-14:
            d = min(dt, 1.0 - t)
            s.step(d)
            t += d
        got = s.get_state()
    i = np.arange(128)
    ex = np.exp(-0.01) * np.sin((i + 1.0) * spec.dx - 1.0)
    assert np.max(np.abs(got[1] - ex)) < 1e-4


@pytest.mark.parametrize("rk", [3, 54])
def test_fp32_rk_steps_vs_oracle(rk):
    """Three limited SSP-RK3 / SSP-RK(5,4) steps of the FP32-mixed form on a rough
    Burgers state against the FP64 oracle: within the FP32 tolerance, bounds exact."""
    spec = ai.Spec(dim=2, nx=48, ny=40, x0=0, x1=1.2, y0=0, y1=1.0, flux=("burgers", (0.5,)),
                   diff=("pwl", (0.0, 0.0, 0.1, 0.5)), umin=-1.0, umax=1.0, limiter=True)
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=21)]
    ref = [np.array(a) for a in st]
    with solver(spec, "fp32_mixed", rk=rk) as s:
        s.set_state(st)
        for _ in range(3):
            dt = oracle.dt_cfl(spec, ref[0])
            ref, _ = oracle.step(spec, rk, ref, dt)
            s.step(dt)
        got = s.get_state()
        lo, hi = s.bounds()
        assert s.stats()["errors"] == 0
    assert lo >= -1.0 and hi <= 1.0
    assert linf(got, ref) <= 1e-5
    assert l1(got, ref) <= 1e-6
