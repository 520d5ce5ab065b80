"""The 3D CUDA path reproduces what the paper prints for d = 3: Table 4's 3D Barenblatt
minima (Example 6.3) and fourth-order convergence of averages and point values for the
smooth linear problem (Example 6.1)."""
import math
import os

import numpy as np
import pytest

import af_inputs as ai

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_11527_gb300 import build
    build.build()


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append(line.split())
    return rows


def solver(spec, **kw):
    from paper_2510_11527_gb300 import Solver
    return Solver(spec, **kw)


def _barenblatt_spec(m, limiter):
    return ai.Spec(dim=3, nx=80, ny=80, nz=80, x0=-10, x1=10, y0=-10, y1=10, z0=-10, z1=10, flux=("zero", ()),
                   diff=("pme", (m,)), umin=0.0, umax=1.0, limiter=limiter)


@pytest.mark.parametrize("m", [2, 3, 5, 8])
def test_table4_barenblatt_minimum_3d(m):
    """3D Barenblatt, N = 80 on [-10, 10]^3, t: 1 -> 2, SSP-RK(5,4) at the default step
    (the diffusive cap binds). With limiting the minimum is exactly 0; without it, the
    scheme undershoots to the printed negative minimum."""
    rows = {int(r[0]): [float(v) for v in r[1:]] for r in _golden("table4_barenblatt_3d.txt")}
    spec = _barenblatt_spec(m, True)
    st = [a.numpy() for a in ai.state_3d(lambda x, y, z: ai.barenblatt_3d(x, y, z, 1.0, m=m), spec)]
    with solver(spec, rk=54) as s:
        s.set_state(st)
        s.run(1.0)
        lo, hi = s.bounds()
        assert s.stats()["errors"] == 0
    assert lo == 0.0 and hi <= 1.0
    with solver(_barenblatt_spec(m, False), rk=54) as s:
        s.set_state(st)
        s.run(1.0)
        lo, _ = s.bounds()
    print(f"m={m}: unlimited minimum {lo:.4e} (printed {rows[m][0]:.4e})")
    assert lo == pytest.approx(rows[m][0], rel=TOL_TABLE4_3D)


def _order(e):
    return [math.log2(e[k] / e[k + 1]) for k in range(len(e) - 1)]


def _exact_3d(spec, t, k=2 * math.pi, c=1.0, k0=0.01):
    """Example 6.1 with d = 3: 1 + exp(-3 k^2 k0 t) sin(k (x + y + z - 3 c t)), as cell
    averages (product of the three averaging factors) and point values by kind."""
    out = ai.mode_3d_state(spec, k)
    ph = -3 * k * c * t
    dec = math.exp(-3 * k * k * k0 * t)
    fac = 1.0
    for h in (spec.dx, spec.dy, spec.dz):
        fac *= math.sin(k * h / 2) / (k * h / 2)
    i = np.arange(spec.nx)
    res = []
    for s_, (sx, sy, sz) in enumerate(ai.kind_offsets_3d()):
        x = spec.x0 + (i + 0.5 + 0.5 * sx) * spec.dx
        y = spec.y0 + (np.arange(spec.ny) + 0.5 + 0.5 * sy) * spec.dy
        z = spec.z0 + (np.arange(spec.nz) + 0.5 + 0.5 * sz) * spec.dz
        w = k * (x[None, None, :] + y[None, :, None] + z[:, None, None]) + ph
        res.append(1.0 + dec * (fac if s_ == 0 else 1.0) * np.sin(w))
    return [a.numpy() for a in out], res


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_fourth_order_3d_gpu(prec):
    """Example 6.1, d = 3: f_l = u, a = 0.01 u on [0, 1]^3 to T = 0.2, SSP-RK(5,4) at
    dt = 0.05 / (1/h + k0/h^2); L1 errors of the averages and of the 7 point kinds."""
    T = 0.2
    eb, ep = [], []
    for n in (16, 32, 64):
        spec = ai.Spec(dim=3, nx=n, ny=n, nz=n, x0=0, x1=1, y0=0, y1=1, z0=0, z1=1,
                       flux=("linear", (1.0, 1.0, 1.0)), diff=("const", (0.01,)), umin=-10, umax=10, limiter=False)
        st, _ = _exact_3d(spec, 0.0)
        _, ex = _exact_3d(spec, T)
        dt = 0.05 / (1.0 / spec.dx + 0.01 / spec.dx ** 2)
        with solver(spec, precision=prec, rk=54) as s:
            s.set_state(st)
            t = 0.0
            while t < T - 1e-14:
                d = min(dt, T - t)
                s.step(d)
                t += d
            got = s.get_state()
        eb.append(float(np.mean(np.abs(got[0] - ex[0]))))
        ep.append(max(float(np.mean(np.abs(g - e))) for g, e in zip(got[1:], ex[1:])))
    print(f"{prec}: averages {eb} orders {_order(eb)}; points {ep} orders {_order(ep)}")
    if prec == "fp64":
        assert min(_order(eb)) > 3.8
        assert min(_order(ep)) > 3.8
    else:
        # 64^3: discretisation error ~7e-7 plus the FP32 point round-off
        assert eb[-1] < 1.5e-6 and ep[-1] < 1.5e-6


# the paper does not state the step of the unlimited runs; the undershoot is a spatial
# effect and varies little with it
TOL_TABLE4_3D = 0.05
