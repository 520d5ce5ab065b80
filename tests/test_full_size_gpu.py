"""Parity at the benchmark's full sizes, in the launch configurations bench.py times:
one SSP-RK3 step of the 4096^2 porous-medium and Buckley-Leverett workloads and of the
256-instance batch, checked on sampled cells against the oracle run on a window around
each sampled cell (a stage reads +-2 cells, +-3 with the blend, so a step depends on at
most +-9; the windows are wide enough that their own periodic wrap cannot reach the
centre). FP64 is held to the 1e-12 parity bound; FP32-mixed to its stated tolerance."""
import numpy as np
import pytest

import af_inputs as ai
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_11527_gb300 import build
    build.build()


def _window(st, j, i, r):
    ny, nx = st[0].shape
    jj = (np.arange(j - r, j + r + 1) % ny)[:, None]
    ii = (np.arange(i - r, i + r + 1) % nx)[None, :]
    return [np.ascontiguousarray(a[jj, ii]) for a in st]


def _sampled(spec, st, dt, got, rng, samples, r, tol):
    ny, nx = st[0].shape
    sub = ai.Spec(**{**spec.__dict__, "nx": 2 * r + 1, "ny": 2 * r + 1,
                     "x1": spec.x0 + (2 * r + 1) * spec.dx, "y1": spec.y0 + (2 * r + 1) * spec.dy})
    scale = max(abs(spec.umin), abs(spec.umax))
    u = st[0]
    rough = np.argwhere(np.abs(u - np.roll(u, 1, 1)) + np.abs(u - np.roll(u, 1, 0)) > 1e-3 * scale)
    worst = 0.0
    for k in range(samples):
        if k % 2 == 0 and len(rough):
            j, i = (int(v) for v in rough[rng.integers(len(rough))])
        else:
            j, i = int(rng.integers(ny)), int(rng.integers(nx))
        out, _ = oracle.step(sub, 3, _window(st, j, i, r), dt)
        for a_ref, a_got in zip(out, got):
            worst = max(worst, abs(a_ref[r, r] - float(a_got[j, i])) / scale)
    assert worst <= tol, worst


def _one_step(spec, st, prec):
    from paper_2510_11527_gb300 import Solver
    with Solver(spec, precision=prec, rk=3) as s:
        s.set_state(st)
        dt = s.dt_cfl()
        s.step(dt)
        got = s.get_state()
        lo, hi = s.bounds()
        assert s.stats()["errors"] == 0
    assert spec.umin <= lo and hi <= spec.umax
    return dt, got


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_mixed", 1e-5)])
def test_pme_4096_sampled(prec, tol):
    spec = ai.config3(4096)
    st = [a.cpu().numpy() for a in ai.state_2d(lambda x, y: ai.barenblatt(x, y, 1.0), spec, device="cuda",
                                                sub=2, order=3)]
    dt, got = _one_step(spec, st, prec)
    assert dt == pytest.approx(oracle.dt_cfl(spec, st[0]), rel=1e-14)
    _sampled(spec, st, dt, got, np.random.default_rng(1), 40, 10, tol)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_mixed", 1e-5)])
def test_bl_4096_plain_blend_sampled(prec, tol):
    spec = ai.config5(4096)
    spec.blend = "plain"
    st = [a.cpu().numpy() for a in ai.state_2d(ai.bl_disc_fn, spec, device="cuda", sub=2, order=3)]
    dt, got = _one_step(spec, st, prec)
    assert dt == pytest.approx(oracle.dt_cfl(spec, st[0]), rel=1e-14)
    _sampled(spec, st, dt, got, np.random.default_rng(2), 40, 12, tol)


def test_batch_256_fp32_sampled():
    """The full 256-instance batch (FP32-mixed, autotuned tile, graph replay): one step,
    then sampled cells of 12 instances against the oracle."""
    from paper_2510_11527_gb300 import capi
    inst = ai.batch_instances()
    specs = [s for s, _ in inst]
    grids, fl, df, bd = [], [], [], []
    for s in specs:
        grids.append(capi.af_grid(2, s.nx, s.ny, s.x0, s.x1, s.y0, s.y1))
        f = capi.af_flux()
        f.kind = capi.FLUX[s.flux[0]]
        f.p[0] = s.flux[1][0]
        d = capi.af_diff()
        d.kind = capi.DIFF[s.diff[0]]
        for k, v in enumerate(s.diff[1]):
            d.p[k] = v
        fl.append(f)
        df.append(d)
        bd.append(capi.af_bounds_t(s.umin, s.umax, 0))
    b = capi.af_batch_create(grids, fl, df, bd, capi.af_opts(capi.PREC["fp32_mixed"], 3, 0.0, 0.0, 1, 0, 1.0))
    rng = np.random.default_rng(3)
    pick = sorted(rng.choice(len(inst), size=12, replace=False).tolist())
    states = {}
    try:
        for i, (s, m) in enumerate(inst):
            st = [a.cpu().numpy() for a in ai.batch_state(s, m, device="cuda")]
            if i in pick:
                states[i] = st
            capi.af_batch_set_state(b, i, s.cells, *st)
        capi.af_batch_autotune(b)
        capi.af_batch_step(b, 1)
        capi.af_batch_sync(b)
        assert capi.af_batch_stats(b)["errors"] == 0
        for i in pick:
            s = specs[i]
            got = capi.af_batch_get_state(b, i, s.cells)
            dt = capi.af_batch_time(b, i)
            assert dt == pytest.approx(oracle.dt_cfl(s, states[i][0]), rel=1e-14)
            _sampled(s, states[i], dt, [np.asarray(a).reshape(s.ny, s.nx) for a in got], rng, 6, 10, 1e-5)
    finally:
        capi.af_batch_destroy(b)
