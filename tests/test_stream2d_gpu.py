"""The column-marching FP32-mixed stage (periodic meshes) against the FP64
oracle: one forward-Euler evaluation and SSP-RK3 / SSP-RK(5,4) steps, on meshes that
exercise its band edges (28 output columns per warp, ragged last band, meshes narrower
than the halo) and strip edges (16-row strips with a 4-row warm-up, ragged last strip),
for every flux kind and every diffusion kind the kernel is compiled for, without and
with the smoothness blend. FP32 stencils: max difference <= 1e-5 and mean difference
<= 1e-6 of the bound scale, bounds exact, and mass conserved to FP64 round-off plus
what counted safeguard clamps of cell averages moved."""
import numpy as np
import pytest

import af_inputs as ai
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_11527_gb300 import build
    build.build()


MODELS = {
    "burgers_pwl": (("burgers", (0.5,)), ("pwl", (0.0, 0.0, 0.1, 0.5)), -1.0, 1.0),
    "burgers_band": (("burgers", (0.5,)), ("pwl", (0.03, 0.25, 0.03, 0.75)), 0.0, 1.0),
    "burgers_none": (("burgers", (0.5,)), ("none", ()), -1.0, 1.0),
    "bl_cubic": (("bl", (5.0,)), ("cubic", (0.0, 0.02, -0.04 / 3)), 0.0, 1.0),
    "bl_cubic01": (("bl", (5.0,)), ("cubic01", (0.0, 0.02, -0.04 / 3)), 0.0, 1.0),
    "pme2": (("zero", ()), ("pme", (2,)), 0.0, 1.0),
    "pme3": (("zero", ()), ("pme", (3,)), 0.0, 1.0),
    "linear_const": (("linear", (1.0, -0.6)), ("const", (0.01,)), -2.0, 2.0),
    "burgers_ramp": (("burgers", (0.5,)), ("ramp", (0.05, 0.4, 0.2)), 0.0, 1.0),
}
SHAPES = [(1, 1), (3, 2), (5, 9), (27, 5), (28, 16), (29, 17), (57, 33), (100, 3), (3, 100), (130, 75)]


def spec_of(name, nx, ny, limiter=True, blend="off"):
    flux, diff, lo, hi = MODELS[name]
    return ai.Spec(dim=2, nx=nx, ny=ny, x0=0, x1=0.02 * nx + 0.3, y0=0, y1=0.015 * ny + 0.2, flux=flux,
                   diff=diff, umin=lo, umax=hi, limiter=limiter, blend=blend)


def check(spec, got, want, stats, m0, m1, st):
    scale = max(abs(spec.umin), abs(spec.umax))
    got = [np.asarray(g, dtype=np.float64) for g in got]
    assert max(float(np.max(np.abs(g - w))) for g, w in zip(got, want)) <= 1e-5 * scale
    assert max(float(np.mean(np.abs(g - w))) for g, w in zip(got, want)) <= 1e-6 * scale
    assert stats["errors"] == 0
    if spec.limiter:
        assert min(float(g.min()) for g in got) >= spec.umin and max(float(g.max()) for g in got) <= spec.umax
    # mass is conserved to FP64 round-off plus what counted clamps of cell averages
    # moved (an FP32-rounding excess of less than an FP32 ulp of the bound)
    mscale = float(np.sum(np.abs(st[0]))) * spec.dx * spec.dy
    assert stats["avg_clamps"] <= stats["clamps"]
    assert abs(m1 - m0) <= 1e-13 * mscale + stats["mass_adjust"]


def run_gpu(spec, st, rk, tau, s_ext=None):
    from paper_2510_11527_gb300 import Solver
    with Solver(spec, precision="fp32_mixed", rk=(3 if rk == "fe" else rk)) as s:
        s.set_state(st)
        if s_ext is not None:
            s.set_indicator(s_ext)
        m0 = s.mass()
        if rk == "fe":
            s.forward_euler(tau)
        else:
            s.step(tau)
        return s.get_state(), s.stats(), m0, s.mass()


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("name", ["burgers_pwl", "bl_cubic", "pme2"])
@pytest.mark.parametrize("limiter", [True, False])
def test_forward_euler_shapes(nx, ny, name, limiter):
    spec = spec_of(name, nx, ny, limiter)
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=nx * 131 + ny)]
    tau = oracle.dt_cfl(spec, st[0])
    got, stats, m0, m1 = run_gpu(spec, st, "fe", tau)
    check(spec, got, oracle.fe(spec, st, tau), stats, m0, m1, st)


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("rk", [3, 54])
def test_rk_step_every_model(name, rk):
    spec = spec_of(name, 61, 47)
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=rk + len(name))]
    tau = oracle.dt_cfl(spec, st[0])
    want, _ = oracle.step(spec, rk, [a.copy() for a in st], tau)
    got, stats, m0, m1 = run_gpu(spec, st, rk, tau)
    check(spec, got, want, stats, m0, m1, st)


def test_several_strips_and_bands_multi_step():
    """Five SSP-RK3 steps of the degenerate Burgers data on 200 x 150 (8 bands, 10
    strips): every cell against the oracle."""
    import af_inputs
    spec = af_inputs.config2(200).with_size(200, 150)
    st = [a.numpy() for a in af_inputs.initial_state(spec)]
    ref = [a.copy() for a in st]
    from paper_2510_11527_gb300 import Solver
    with Solver(spec, precision="fp32_mixed") as s:
        s.set_state(st)
        m0 = s.mass()
        for _ in range(5):
            dt = oracle.dt_cfl(spec, ref[0])
            ref, _ = oracle.step(spec, 3, ref, dt)
            s.step(dt)
        got, stats, m1 = s.get_state(), s.stats(), s.mass()
    check(spec, got, ref, stats, m0, m1, st)


# ---- the smoothness blend (Section 5.1.3): the plain indicator, formed by its own pass,
# and an external indicator per cell

@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("name", ["burgers_pwl", "bl_cubic"])
@pytest.mark.parametrize("blend", ["plain", "external"])
def test_forward_euler_blend_shapes(nx, ny, name, blend):
    spec = spec_of(name, nx, ny, blend=blend)
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=nx * 17 + ny)]
    sx = np.random.default_rng(nx + 3 * ny).uniform(0, 2, size=(ny, nx)) if blend == "external" else None
    tau = oracle.dt_cfl(spec, st[0])
    got, stats, m0, m1 = run_gpu(spec, st, "fe", tau, sx)
    check(spec, got, oracle.fe(spec, st, tau, s_ext=sx), stats, m0, m1, st)


@pytest.mark.parametrize("name", ["burgers_pwl", "bl_cubic", "pme2", "linear_const", "burgers_none"])
@pytest.mark.parametrize("rk", [3, 54])
def test_rk_step_blend_every_flux(name, rk):
    spec = spec_of(name, 61, 47, blend="plain")
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=5 * rk + len(name))]
    tau = oracle.dt_cfl(spec, st[0])
    want, _ = oracle.step(spec, rk, [a.copy() for a in st], tau)
    got, stats, m0, m1 = run_gpu(spec, st, rk, tau)
    check(spec, got, want, stats, m0, m1, st)


def test_blend_several_strips_multi_step():
    """Three SSP-RK3 steps of the Buckley-Leverett disc with the plain blend on 200 x 150
    (8 bands, several strips): every cell against the oracle."""
    import af_inputs
    spec = af_inputs.config5(200).with_size(200, 150)
    st = [a.numpy() for a in af_inputs.initial_state(spec)]
    ref = [a.copy() for a in st]
    from paper_2510_11527_gb300 import Solver
    with Solver(spec, precision="fp32_mixed") as s:
        s.set_state(st)
        m0 = s.mass()
        for _ in range(3):
            dt = oracle.dt_cfl(spec, ref[0])
            ref, _ = oracle.step(spec, 3, ref, dt)
            s.step(dt)
        got, stats, m1 = s.get_state(), s.stats(), s.mass()
    check(spec, got, ref, stats, m0, m1, st)

