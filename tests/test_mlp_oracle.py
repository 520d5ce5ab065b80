"""Pins of the FP64 indicator-network reference (oracle/mlp.py)."""
import numpy as np
import pytest
import torch

import af_inputs as ai
from oracle import mlp


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(0).normal(0, 3, 20000)
    x = np.concatenate([x, [0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, 65504.0, 1e-30]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    p = mlp.init_params(3)
    x = rng.normal(0, 0.5, (64, mlp.NIN))
    y = rng.uniform(0, 1, 64)
    loss, g = mlp.loss_and_grad(p, x, y, quantize=False)
    flat, gflat = mlp.pack(p), mlp.pack(g)
    idx = rng.choice(mlp.NPARAM, 80, replace=False)
    h = 1e-6
    for k in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[k] += h
        fm[k] -= h
        lp, _ = mlp.loss_and_grad(mlp.unpack(fp), x, y, quantize=False)
        lm, _ = mlp.loss_and_grad(mlp.unpack(fm), x, y, quantize=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[k]) <= 1e-6 * max(1e-3, abs(fd))


def test_features_and_label_by_brute_force():
    rng = np.random.default_rng(2)
    ny, nx = 6, 7
    ub, V, X, Y = (rng.uniform(-1, 1, (ny, nx)) for _ in range(4))
    F = mlp.features(ub, V, X, Y).reshape(ny, nx, mlp.NIN)
    L = mlp.plain_label(ub).reshape(ny, nx)
    for j in range(ny):
        for i in range(nx):
            u = lambda a, b: ub[(j + b) % ny, (i + a) % nx]
            vals = [u(a, b) for a, b in mlp.PATCH_UB]
            vals += [V[(j - 1) % ny, (i - 1) % nx], V[(j - 1) % ny, i], V[j, (i - 1) % nx], V[j, i],
                     X[j, (i - 1) % nx], X[j, i], Y[(j - 1) % ny, i], Y[j, i]]
            sc = max(abs(v) for v in vals) + 1e-13
            np.testing.assert_allclose(F[j, i], [(v - ub[j, i]) / sc for v in vals], rtol=0, atol=1e-15)

            def st(um, uc, up):
                return abs(um - 2 * uc + up) / (abs(um) + 2 * abs(uc) + abs(up) + 1e-13)

            s1 = (st(u(-2, 0), u(-1, 0), u(0, 0)) + 4 * st(u(-1, 0), u(0, 0), u(1, 0)) +
                  st(u(0, 0), u(1, 0), u(2, 0))) / 6
            s2 = (st(u(0, -2), u(0, -1), u(0, 0)) + 4 * st(u(0, -1), u(0, 0), u(0, 1)) +
                  st(u(0, 0), u(0, 1), u(0, 2))) / 6
            assert L[j, i] == pytest.approx(max(s1, s2), rel=1e-14, abs=1e-16)


def test_label_is_zero_on_constant_and_linear_fields_and_large_at_jumps():
    spec = ai.Spec(dim=2, nx=16, ny=16)
    ub = np.full((16, 16), 0.4)
    assert np.max(mlp.plain_label(ub)) == 0.0
    ub2 = np.where(np.arange(16)[None, :] < 8, 1.0, 0.0) * np.ones((16, 1))
    assert np.max(mlp.plain_label(ub2)) > 0.1


def test_adam_step_definition():
    p = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    m = np.zeros(2)
    v = np.zeros(2)
    p1, m1, v1 = mlp.adam(p, g, m, v, 1, 1e-3)
    # first Adam step moves every parameter by lr * sign(g) (up to eps)
    np.testing.assert_allclose(p1, p - 1e-3 * np.sign(g), rtol=0, atol=1e-10)
