"""Pins of the oracle for Example 6.6 (1D Buckley-Leverett with Dirichlet ends, without
and with gravity) against what the paper and the mathematics fix:

  * the 1D flux is f1 = u^2/(u^2+(1-u)^2), times 1 - 5(1-u)^2 with gravity, and the
    diffusion potential is eps (2u^2 - 4u^3/3) on [0, 1], constant outside, kappa_max =
    eps; the wave speed over [0, 1] is the brute-force maximum of |f'|;
  * the AF method on 100 cells stays in [0, 1] and matches the first-order 2000-cell
    reference (the kind of reference the paper uses for its 1D examples), and moves
    closer to it on 200 cells.
"""
import os

import numpy as np
import pytest

import af_inputs as ai
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = 0.01


def _golden_column(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return np.array([float(line) for line in f if line.strip() and not line.startswith("#")])


def _ref(problem, gravity, n):
    col = _golden_column(f"buckley_leverett_{problem}_{'gravity' if gravity else 'nogravity'}_first_order_2000.txt")
    return col.reshape(n, 2000 // n).mean(axis=1)


@pytest.mark.parametrize("gravity", [False, True])
def test_example_6_6_model_functions(gravity):
    sp = ai.buckley_leverett_1d(100, gravity)
    g = 5.0 if gravity else 0.0
    for u in (0.0, 0.2, 0.5, 0.77, 1.0):
        f1 = u * u / (u * u + (1 - u) ** 2)
        f, d, a = oracle.point_funcs(sp, 0, u)
        assert f == pytest.approx(f1 * (1 - g * (1 - u) ** 2), rel=1e-14, abs=1e-16)
        assert a == pytest.approx(EPS * (2 * u * u - 4 * u ** 3 / 3), rel=1e-14, abs=1e-18)
        h = 1e-6
        fp, _, _ = oracle.point_funcs(sp, 0, u + h)
        fm, _, _ = oracle.point_funcs(sp, 0, u - h)
        assert d == pytest.approx((fp - fm) / (2 * h), rel=1e-7, abs=1e-9)
    # a is constant outside [0, 1]
    assert oracle.point_funcs(sp, 0, -0.3)[2] == 0.0
    assert oracle.point_funcs(sp, 0, 1.4)[2] == pytest.approx(2 * EPS / 3, rel=1e-15)
    assert oracle.kappa_max(sp) == pytest.approx(EPS, rel=1e-12)
    wide = ai.Spec(dim=1, nx=4, diff=sp.diff, umin=-1.0, umax=2.0)
    assert oracle.kappa_max(wide) == pytest.approx(EPS, rel=1e-12)
    # the interval wave speed over [0, 1]: brute force over a dense grid
    u = np.linspace(0.0, 1.0, 2_000_001)
    v = 1 - u
    D = u * u + v * v
    f1 = u * u / D
    d1 = 2 * u * v / D ** 2
    dd = d1 * (1 - g * v * v) + f1 * 2 * g * v
    assert oracle.alpha_interval(sp, 0, 0.0, 1.0) == pytest.approx(np.max(np.abs(dd)), abs=1e-10)
    assert oracle.alpha_interval(sp, 0, 0.0, 1.0) == pytest.approx(3.3105 if gravity else 2.0, abs=1e-4)


@pytest.mark.parametrize("gravity", [False, True])
@pytest.mark.parametrize("problem", ["ibvp", "rp"])
def test_example_6_6_matches_first_order_reference(problem, gravity):
    sp = ai.buckley_leverett_1d(100, gravity, problem)
    st = [a.numpy() for a in ai.initial_state(sp)]
    out, _, stats = oracle.run_native(sp, 3, st, sp.T)
    assert stats["error"] == 0 and stats["clamps"] == 0
    assert min(out[0].min(), out[1].min()) >= 0.0 and max(out[0].max(), out[1].max()) <= 1.0
    assert out[1][0] == sp.bc_values[0] and out[1][-1] == sp.bc_values[1]
    e100 = np.abs(out[0] - _ref(problem, gravity, 100)).sum() * sp.dx
    assert e100 < 4e-3
    sp2 = ai.buckley_leverett_1d(200, gravity, problem)
    out2, _, _ = oracle.run_native(sp2, 3, [a.numpy() for a in ai.initial_state(sp2)], sp2.T)
    e200 = np.abs(out2[0] - _ref(problem, gravity, 200)).sum() * sp2.dx
    assert e200 < e100
