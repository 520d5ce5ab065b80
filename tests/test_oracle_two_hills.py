"""Pins of the oracle on Example 6.4 (collision of two hills, u_t = Lap(u^2) on the
periodic [-10, 10]^2) against what the paper states and the mathematics fixes: with the
MPP limiting the solution stays in [0, max u0]; without it negative values appear; the
hills diffuse and merge; mass is conserved; the data and the equation are symmetric
under (x, y) -> (-x, -y) and (x, y) -> (-y, -x), and so is the solution."""
import dataclasses

import numpy as np

import af_inputs as ai
import oracle


def _state(sp):
    return [a.numpy() for a in ai.initial_state(sp)]


def test_two_hills_limiting_keeps_nonnegative_and_unlimited_does_not():
    sp = ai.two_hills(100)
    st = _state(sp)
    assert max(a.max() for a in st) == sp.umax and min(a.min() for a in st) == 0.0
    out, _, stats = oracle.run_native(sp, 3, st, 0.5)
    lo, hi = oracle.bounds(out)
    assert stats["error"] == 0 and lo == 0.0 and hi <= sp.umax
    un, _, _ = oracle.run_native(dataclasses.replace(sp, limiter=False), 3, st, 0.5)
    assert oracle.bounds(un)[0] < -1e-4


def test_two_hills_merge_conserve_mass_and_stay_symmetric():
    sp = ai.two_hills(50)
    st = _state(sp)
    out, _, stats = oracle.run_native(sp, 3, st, sp.T)
    assert stats["error"] == 0 and oracle.bounds(out)[0] == 0.0
    ub = out[0]
    # the two cells on the diagonal y = x that touch the origin lie outside both initial
    # supports; by T = 4 the hills have merged over them
    mid = [(24, 24), (25, 25)]
    assert all(st[0][c] == 0.0 for c in mid)
    assert all(ub[c] > 0.2 for c in mid)
    assert abs(ub.sum() - st[0].sum()) <= 1e-12 * st[0].sum()
    assert np.max(np.abs(ub - ub[::-1, ::-1])) < 1e-14
    assert np.max(np.abs(ub - ub.T[::-1, ::-1])) < 1e-14
