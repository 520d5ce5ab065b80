"""Failure detection on the host (no GPU fault is provoked) and checkpoint/resume."""
import numpy as np
import pytest

import af_inputs as ai

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_11527_gb300 import build
    build.build()


def test_invalid_arguments_rejected():
    from paper_2510_11527_gb300 import capi
    ok = dict(flux=capi.af_flux(), diff=capi.af_diff(), bounds=capi.af_bounds_t(0.0, 1.0, 0),
              opts=capi.af_opts(0, 3, 0.0, 0.0, 1, 0, 1.0))
    bad = [capi.af_grid(3, 8, 8, 0, 1, 0, 1), capi.af_grid(2, 0, 8, 0, 1, 0, 1), capi.af_grid(2, 8, 8, 1, 0, 0, 1)]
    for g in bad:
        with pytest.raises(capi.AfError) as ei:
            capi.af_create(g, ok["flux"], ok["diff"], ok["bounds"], ok["opts"])
        assert ei.value.status == capi.AF_E_ARG
    g = capi.af_grid(2, 8, 8, 0, 1, 0, 1)
    with pytest.raises(capi.AfError) as ei:
        capi.af_create(g, ok["flux"], ok["diff"], capi.af_bounds_t(1.0, 0.0, 0), ok["opts"])
    assert ei.value.status == capi.AF_E_ARG
    with pytest.raises(capi.AfError) as ei:
        capi.af_create(g, ok["flux"], ok["diff"], ok["bounds"], capi.af_opts(0, 7, 0.0, 0.0, 1, 0, 1.0))
    assert ei.value.status == capi.AF_E_ARG
    d = capi.af_diff()
    d.kind = capi.DIFF["pme"]
    d.p[0] = 2.5
    with pytest.raises(capi.AfError) as ei:
        capi.af_create(g, ok["flux"], d, ok["bounds"], ok["opts"])
    assert ei.value.status == capi.AF_E_ARG


def test_bad_states_rejected_and_context_stays_usable():
    from paper_2510_11527_gb300 import Solver, capi
    spec = ai.config2(16)
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=1, lo=-1, hi=1)]
    with Solver(spec) as s:
        s.set_state(st)
        bad = [a.copy() for a in st]
        bad[2][3, 4] = np.nan
        with pytest.raises(capi.AfError) as ei:
            s.set_state(bad)
        assert ei.value.status == capi.AF_E_STATE and "NaN" in str(ei.value)
        bad = [a.copy() for a in st]
        bad[0][0, 0] = 1.5
        with pytest.raises(capi.AfError) as ei:
            s.set_state(bad)
        assert ei.value.status == capi.AF_E_STATE
        # the previous state is untouched and stepping still works
        got = s.get_state()
        for a, b in zip(got, st):
            assert np.array_equal(a, b)
        s.step(0.0)
        with pytest.raises(capi.AfError):
            s.stage(7, 1e-3)


def test_bounds_from_initial_data():
    from paper_2510_11527_gb300 import Solver
    spec = ai.config2(24)
    st = [0.5 * a.numpy() for a in ai.random_state_2d(spec, seed=3, lo=-1, hi=1)]
    with Solver(spec, bounds_from_data=True) as s:
        s.set_state(st)
        lo0 = min(float(a.min()) for a in st)
        hi0 = max(float(a.max()) for a in st)
        for _ in range(3):
            s.step(0.0)
        lo, hi = s.bounds()
    assert lo >= lo0 and hi <= hi0


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_checkpoint_resume_is_bitwise(prec):
    """Run 6 steps; or run 3, read the state and time back, restart a fresh context from
    them and run 3 more: identical results."""
    from paper_2510_11527_gb300 import Solver
    spec = ai.config2(64)
    st = [a.numpy() for a in ai.initial_state(spec)]
    with Solver(spec, precision=prec) as a:
        a.set_state(st)
        for _ in range(6):
            a.step(0.0)
        full = a.get_state()
    with Solver(spec, precision=prec) as b:
        b.set_state(st)
        for _ in range(3):
            b.step(0.0)
        ck = b.get_state()
    with Solver(spec, precision=prec) as c:
        c.set_state(ck)
        for _ in range(3):
            c.step(0.0)
        resumed = c.get_state()
    for x, y in zip(full, resumed):
        assert np.array_equal(x, y)


def test_oversize_mesh_reports_oom_and_device_stays_usable():
    """A mesh far larger than device memory (1e6 x 1e6 cells, ~1e14 bytes) fails with
    AF_E_OOM at creation, without a fault; a normal context works afterwards."""
    from paper_2510_11527_gb300 import Solver, capi
    g = capi.af_grid(2, 1000000, 1000000, 0.0, 1.0, 0.0, 1.0)
    f, d = capi.af_flux(), capi.af_diff()
    with pytest.raises(capi.AfError) as ei:
        capi.af_create(g, f, d, capi.af_bounds_t(0.0, 1.0, 0), capi.af_opts(0, 3, 0.0, 0.0, 1, 0, 1.0))
    assert ei.value.status == capi.AF_E_OOM
    spec = ai.config2(16)
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=2, lo=-1, hi=1)]
    with Solver(spec) as s:
        s.set_state(st)
        s.step(0.0)
        assert s.stats()["errors"] == 0
