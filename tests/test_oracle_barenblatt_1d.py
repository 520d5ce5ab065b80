"""Pins of the oracle on the 1D case of Example 6.3 (Barenblatt, 80 cells on [-6, 6],
t from 1 to 2, m = 2, 3, 5, 8): with the MPP limiting the minimum is exactly 0, without
it the scheme undershoots below 0 (the paper's enlarged 1D views); the peak at t = 2
is the closed form B_m(0, 2) = 2^(-1/(m+1)), and the L1 error against the exact cell
averages is small."""
import dataclasses

import numpy as np
import pytest
import torch

import af_inputs as ai
import oracle


def barenblatt_1d_spec(m, limiter=True):
    return ai.Spec(dim=1, nx=80, x0=-6.0, x1=6.0, flux=("zero", ()), diff=("pme", (m,)), umin=0.0, umax=1.0,
                   limiter=limiter)


def barenblatt_1d_state(spec, m, t=1.0):
    return [a.numpy() for a in ai.state_1d(lambda x: ai.barenblatt(x, torch.zeros_like(x), t, m=m, d=1), spec)]


@pytest.mark.parametrize("m", [2, 3, 5, 8])
def test_barenblatt_1d_limiting(m):
    sp = barenblatt_1d_spec(m)
    st = barenblatt_1d_state(sp, m)
    out, _, stats = oracle.run_native(sp, 54, st, 1.0)
    lo, hi = oracle.bounds(out)
    assert stats["error"] == 0 and lo == 0.0
    # the peak within the discretisation error at h = 0.15 (measured 1.5e-6 to 1.7e-5)
    assert hi == pytest.approx(2.0 ** (-1.0 / (m + 1)), abs=1e-4)
    ex = ai.cell_average_1d(lambda x: ai.barenblatt(x, torch.zeros_like(x), 2.0, m=m, d=1), sp).numpy()
    assert np.abs(out[0] - ex).sum() * sp.dx < 1e-2
    un, _, _ = oracle.run_native(dataclasses.replace(sp, limiter=False), 54, st, 1.0)
    assert oracle.bounds(un)[0] < 0.0
