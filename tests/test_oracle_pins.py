"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: the paper's printed
linear reduction and Fourier matrix, Table 1's CFL limits, the SSP-RK(5,4) order
conditions and eta, closed-form solutions, invariants (conservation, MPP, symmetry)
and brute force. A plausible slip (a dropped term, wrong sign, wrong index, transposed
operand) in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import torch

import af_inputs as ai
import oracle
from oracle import fourier

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def lin1d(n, c=1.0, k0=0.01, L=2 * math.pi):
    return ai.Spec(dim=1, nx=n, x0=0.0, x1=L, flux=("linear", (c, 0.0)), diff=("const", (k0,)),
                   umin=-10.0, umax=10.0, limiter=False)


# ----------------------------------------------------------------------------------
# 1. linear reduction printed in eq. 1d_af_constant (Section 3)

@pytest.mark.parametrize("c", [1.0, -0.7])
def test_linear_reduction_matches_printed_form(c):
    n, k0 = 12, 0.013
    spec = lin1d(n, c=c, k0=k0, L=1.7)
    rng = np.random.default_rng(3)
    ub = rng.uniform(-1, 1, n)
    P = rng.uniform(-1, 1, n)
    tau = 1e-3
    nb, nP = oracle.fe(spec, [ub, P], tau)
    rb, rP = (nb - ub) / tau, (nP - P) / tau
    h = spec.dx
    R = lambda a, s: np.roll(a, -s)  # R(a, s)[i] = a[i+s]
    Pm1, P0, Pp1, Pm2 = R(P, -1), P, R(P, 1), R(P, -2)   # u_{i-1/2}, u_{i+1/2}, u_{i+3/2}, u_{i-3/2}
    cen = (6 * ub - Pm1 - P0) / 4                       # Simpson centre u_i
    if c > 0:
        # printed form (c > 0): only the D+ operator acts on f+ = c u
        conv_b = -(c / h) * (P0 - Pm1)
        conv_p = -(c / (3 * h)) * (Pm1 - 6 * cen + 3 * P0 + 2 * R(cen, 1))
    else:
        # mirror image of the printed form: only D- acts on f- = c u
        conv_b = -(c / h) * (P0 - Pm1)
        conv_p = -(c / (3 * h)) * (-2 * cen - 3 * P0 + 6 * R(cen, 1) - Pp1)
    diff_b = k0 / (2 * h * h) * (-Pm2 + 4 * R(ub, -1) + Pm1 - 8 * ub + P0 + 4 * R(ub, 1) - Pp1)
    diff_p = k0 / (3 * h * h) * (-5 * Pm1 + 24 * ub - 38 * P0 + 24 * R(ub, 1) - 5 * Pp1)
    np.testing.assert_allclose(rb, conv_b + diff_b, rtol=0, atol=1e-9 * np.max(np.abs(rb)) + 1e-10)
    np.testing.assert_allclose(rP, conv_p + diff_p, rtol=0, atol=1e-9 * np.max(np.abs(rP)) + 1e-10)


# ----------------------------------------------------------------------------------
# 2. Fourier matrix G (eq. 1d_fourier_ode) measured from the oracle operator

@pytest.mark.parametrize("n,k,c,k0", [(64, 1, 1.0, 0.01), (32, 7, 1.0, 0.3), (16, 5, 0.0, 1.0), (24, 11, 2.0, 0.0)])
def test_fourier_matrix_matches_printed(n, k, c, k0):
    G, dx = fourier.G_from_oracle(n, k, c, k0)
    Gp = fourier.G_printed(2 * math.pi * k / n, c, k0, dx)
    assert np.max(np.abs(G - Gp)) <= 1e-12 * np.max(np.abs(Gp))


# ----------------------------------------------------------------------------------
# 3. Table 1 maximum stable CFL numbers from the von Neumann search

def test_table1_cfl_limits():
    for name, adv, dif in _golden("table1_cfl.txt"):
        assert round(fourier.max_stable_cfl(name, 1.0), 3) == pytest.approx(float(adv), abs=1.01e-3)
        assert round(fourier.max_stable_cfl(name, 0.0), 3) == pytest.approx(float(dif), abs=1.01e-3)


def test_table1_ssprk3_limit_with_oracle_time_stepping():
    """Run the oracle itself (SSP-RK3, pure advection) just below and above 0.773."""
    spec = ai.Spec(dim=1, nx=32, x0=0, x1=1, flux=("linear", (1.0, 0.0)), diff=("none", ()),
                   umin=-10, umax=10, limiter=False)
    rng = np.random.default_rng(0)
    st0 = [rng.uniform(-1, 1, 32), rng.uniform(-1, 1, 32)]

    def growth(cfl):
        st = [a.copy() for a in st0]
        for _ in range(3000):
            st, _ = oracle.step(spec, 3, st, cfl * spec.dx)
        return max(np.max(np.abs(a)) for a in st)

    assert growth(0.76) < 10.0
    assert growth(0.79) > 1e3


# ----------------------------------------------------------------------------------
# 4. SSP-RK(5,4): order-4 conditions and the printed eta

def _butcher_from_shu_osher(alpha, beta):
    s = alpha.shape[0]
    # stage values u^(k) = sum_l alpha[k-1][l] u^(l) + beta[k-1][l] dt F(u^(l)), u^(0) = u^n
    # Butcher A for the s stages u^(0..s-1), b for the output
    Acoef = np.zeros((s + 1, s + 1))
    for k in range(1, s + 1):
        for l in range(k):
            Acoef[k] += alpha[k - 1][l] * Acoef[l]
            Acoef[k][l] += beta[k - 1][l]
    A = Acoef[:s, :s]
    b = Acoef[s, :s]
    return A, b


def test_rk54_order_conditions_and_eta():
    alpha, beta = oracle.rk54_coefficients()
    A, b = _butcher_from_shu_osher(alpha, beta)
    c = A.sum(axis=1)
    conds = [
        (b.sum(), 1.0), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ (A @ c), 1 / 6),
        (b @ c ** 3, 1 / 4), (b @ (c * (A @ c)), 1 / 8), (b @ (A @ c ** 2), 1 / 12), (b @ (A @ (A @ c)), 1 / 24),
    ]
    for got, want in conds:
        assert abs(got - want) < 1e-14
    eta = float(_golden("rk54_eta.txt")[0][1])
    # z^5 coefficient of R(z) = 1 + z b^T (I - zA)^{-1} 1 is b^T A^4 1
    z5 = b @ np.linalg.matrix_power(A, 4) @ np.ones(5)
    assert abs(z5 - eta) < 1e-14
    # all Shu-Osher weights non-negative and rows sum to one (convex combinations)
    assert np.all(alpha >= 0) and np.all(beta >= 0)
    np.testing.assert_allclose(alpha.sum(axis=1), 1.0, atol=2e-15)


# ----------------------------------------------------------------------------------
# 5. spatial order from the Fourier symbol (Proposition 3.1) and in practice

def test_eigenvalue_error_constant():
    """lambda_1 - lambda ~ (i c + 7 k0 w) w^5 dx^4 / 2880 as dx -> 0 with k0 > 0
    (Proposition 3.1); for k0 = 0 the constant is 16 times larger (i c / 180).
    Evaluated from the printed G in 50-digit arithmetic."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50

    def ratio(c, k0, w, dx):
        t = mp.e ** (1j * w * dx)
        ti = 1 / t
        Gc = [[0, ti - 1], [3 - t, (-5 * ti - 8 + t) / 6]]
        Gd = [[2 * (ti - 2 + t), (-ti * ti + ti + 1 - t) / 2], [8 * (1 + t), -(5 * ti + 38 + 5 * t) / 3]]
        G = [[c / dx * Gc[i][j] + k0 / dx ** 2 * Gd[i][j] for j in range(2)] for i in range(2)]
        tr, det = G[0][0] + G[1][1], G[0][0] * G[1][1] - G[0][1] * G[1][0]
        d = mp.sqrt(tr * tr - 4 * det)
        lam = -1j * c * w - k0 * w * w
        l1 = min([(tr + d) / 2, (tr - d) / 2], key=lambda e: abs(e - lam))
        return (l1 - lam) / ((1j * c + 7 * k0 * w) * w ** 5 * dx ** 4 / 2880)

    r = [ratio(1, 0.5, 1, mp.mpf(dx)) for dx in ("0.01", "0.001", "0.0001")]
    assert abs(r[-1] - 1) < 3e-4 and abs(r[-1] - 1) < abs(r[1] - 1) < abs(r[0] - 1)
    r0 = ratio(1, 0, 1, mp.mpf("0.0001"))
    assert abs(r0 - 16) < 1e-2


def _order(errs):
    return [math.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]


def test_fourth_order_convergence_1d():
    """u_t + u_x = 0.01 u_xx on [0, 2 pi], exact exp(-0.01 t) sin(x - t), SSP-RK(5,4)."""
    eb, ep = [], []
    for n in [16, 32, 64]:
        spec = ai.config1(n)
        st0 = ai.sine_1d_state(spec)
        dt = 0.5 * 0.9284 / (1.0 / spec.dx + 0.01 / spec.dx ** 2)
        T = 1.0
        st, _, _ = oracle.run(spec, 54, [a.numpy() for a in st0], T, dt_fixed=dt)
        i = np.arange(n)
        xc = (i + 0.5) * spec.dx
        ub_ex = np.exp(-0.01 * T) * (2 / spec.dx) * math.sin(spec.dx / 2) * np.sin(xc - T)
        P_ex = np.exp(-0.01 * T) * np.sin((i + 1.0) * spec.dx - T)
        eb.append(np.mean(np.abs(st[0] - ub_ex)))
        ep.append(np.max(np.abs(st[1] - P_ex)))
    assert min(_order(eb)) > 3.7
    assert min(_order(ep)) > 3.7


def test_fourth_order_convergence_2d():
    """Example 6.1 in 2D: u = 1 + exp(-8 pi^2 k0 t) sin(2 pi (x + y - 2 c t))."""
    errs = []
    T = 0.05
    for n in [16, 32, 64]:
        spec = ai.Spec(dim=2, nx=n, ny=n, flux=("linear", (1.0, 1.0)), diff=("const", (0.01,)),
                       umin=-10, umax=10, limiter=False)
        st0 = ai.mode_2d_state(spec, 2 * math.pi)
        dt = 0.2 * 0.9 / (1.0 / spec.dx + 0.01 / spec.dx ** 2)
        st, _, _ = oracle.run(spec, 54, [a.numpy() for a in st0], T, dt_fixed=dt)
        # exact cell averages at T: the mode decays and shifts by c t in x and y
        k = 2 * math.pi
        fx = math.sin(k * spec.dx / 2) / (k * spec.dx / 2)
        i = np.arange(n)
        xc = (i + 0.5) * spec.dx
        ex = 1 + math.exp(-2 * k * k * 0.01 * T) * fx * fx * np.sin(k * (xc[None, :] + xc[:, None] - 2 * T))
        errs.append(np.mean(np.abs(st[0] - ex)))
    assert min(_order(errs)) > 3.6


# ----------------------------------------------------------------------------------
# 6. dimension reduction: 2D operator on y-independent data equals the 1D operator

@pytest.mark.parametrize("flux", [("linear", (0.8, 0.3)), ("burgers", (0.5,))])
def test_2d_reduces_to_1d_on_y_independent_data(flux):
    n, ny = 10, 4
    rng = np.random.default_rng(5)
    ub1 = rng.uniform(-0.5, 0.5, n)
    P1 = rng.uniform(-0.5, 0.5, n)
    c1 = (6 * ub1 - np.roll(P1, 1) - P1) / 4
    s1 = ai.Spec(dim=1, nx=n, x0=0, x1=1.3, flux=flux, diff=("const", (0.02,)), umin=-9, umax=9,
                 limiter=False)
    s2 = ai.Spec(dim=2, nx=n, ny=ny, x0=0, x1=1.3, y0=0, y1=0.7, flux=flux, diff=("const", (0.02,)),
                 umin=-9, umax=9, limiter=False)
    tau = 1e-3
    nb1, nP1 = oracle.fe(s1, [ub1, P1], tau)
    tile = lambda a: np.tile(a[None, :], (ny, 1))
    out = oracle.fe(s2, [tile(ub1), tile(P1), tile(P1), tile(c1)], tau)
    # the y-direction flux difference cancels only if f2 is y-independent: it is
    np.testing.assert_allclose(out[0], tile(nb1), rtol=0, atol=1e-13)
    np.testing.assert_allclose(out[1], tile(nP1), rtol=0, atol=1e-13)
    np.testing.assert_allclose(out[2], tile(nP1), rtol=0, atol=1e-13)


# ----------------------------------------------------------------------------------
# 7. invariants: conservation, MPP, Remark 5.1, constant states, symmetry

def _discs(n):
    spec = ai.config2(n)
    return spec, [a.numpy() for a in ai.initial_state(spec)]


def test_mass_conservation_with_limiter():
    spec, st = _discs(24)
    m0 = oracle.mass(spec, st[0])
    scale = np.sum(np.abs(st[0])) * spec.dx * spec.dy
    for rk in (3, 54):
        s = [a.copy() for a in st]
        for _ in range(4):
            s, stats = oracle.step(spec, rk, s, oracle.dt_cfl(spec, s[0]))
            assert stats["error"] == 0
            assert abs(oracle.mass(spec, s[0]) - m0) <= 1e-14 * scale * 4


@pytest.mark.parametrize("rk", [3, 54])
@pytest.mark.parametrize("flux,diff", [
    (("burgers", (0.5,)), ("pwl", (0.0, 0.0, 0.1, 0.5))),
    (("burgers", (0.5,)), ("none", ())),
    (("bl", (5.0,)), ("cubic", (0.0, 0.02, -0.04 / 3))),
    (("zero", ()), ("pme", (2,))),
])
def test_mpp_on_random_rough_states(rk, flux, diff):
    spec = ai.Spec(dim=2, nx=12, ny=10, x0=0, x1=1.2, y0=0, y1=1.0, flux=flux, diff=diff,
                   umin=0.0, umax=1.0, limiter=True)
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=11)]
    for _ in range(3):
        st, stats = oracle.step(spec, rk, st, oracle.dt_cfl(spec, st[0]))
        assert stats["error"] == 0
        lo, hi = oracle.bounds(st)
        assert lo >= 0.0 and hi <= 1.0


def test_mpp_1d_random_and_blend():
    spec = ai.Spec(dim=1, nx=40, x0=-2, x1=2, flux=("burgers", (1.0,)), diff=("pwl", (0.1, -0.25, 0.1, 0.25)),
                   umin=-1.0, umax=1.0, limiter=True, blend="plain")
    st = [a.numpy() for a in ai.random_state_1d(spec, seed=2)]
    for _ in range(5):
        st, stats = oracle.step(spec, 54, st, oracle.dt_cfl(spec, st[0]))
        assert stats["error"] == 0
        lo, hi = oracle.bounds(st)
        assert lo >= -1.0 and hi <= 1.0


def test_limiter_inactive_reproduces_high_order_bitwise():
    """Remark 5.1: with every theta = 1 the limited update is the high-order update."""
    spec = ai.Spec(dim=2, nx=16, ny=16, flux=("burgers", (0.5,)), diff=("const", (0.01,)),
                   umin=-10.0, umax=10.0, limiter=True)
    st = [a.numpy() for a in ai.mode_2d_state(spec, 2 * math.pi, shift=0.5, amp=0.3)]
    tau = 0.2 * oracle.dt_cfl(spec, st[0])
    on = oracle.fe(spec, st, tau)
    spec.limiter = False
    off = oracle.fe(spec, st, tau)
    for a, b in zip(on, off):
        assert np.array_equal(a, b)


def test_constant_state_preserved():
    spec = ai.config2(8)
    st = [np.full((8, 8), 0.3) for _ in range(4)]
    out, stats = oracle.step(spec, 3, st, 1e-3)
    assert np.array_equal(out[0], st[0])
    for a in out[1:]:
        np.testing.assert_allclose(a, 0.3, rtol=0, atol=1e-15)


def test_transpose_symmetry():
    """With f1 = f2 and dx = dy, transposing the mesh (V -> V^T, X <-> Y^T) commutes
    with the scheme."""
    spec = ai.Spec(dim=2, nx=10, ny=10, flux=("burgers", (0.5,)), diff=("pwl", (0.0, 0.0, 0.1, 0.5)),
                   umin=-1.0, umax=1.0, limiter=True, blend="plain")
    ub, V, X, Y = [a.numpy() for a in ai.random_state_2d(spec, seed=4, lo=-1, hi=1)]
    tau = oracle.dt_cfl(spec, ub)
    a = oracle.fe(spec, [ub, V, X, Y], tau)
    b = oracle.fe(spec, [ub.T.copy(), V.T.copy(), Y.T.copy(), X.T.copy()], tau)
    np.testing.assert_allclose(b[0], a[0].T, rtol=0, atol=1e-14)
    np.testing.assert_allclose(b[1], a[1].T, rtol=0, atol=1e-14)
    np.testing.assert_allclose(b[2], a[3].T, rtol=0, atol=1e-14)
    np.testing.assert_allclose(b[3], a[2].T, rtol=0, atol=1e-14)


def test_shift_equivariance():
    spec = ai.config2(12)
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=9, lo=-1, hi=1)]
    tau = oracle.dt_cfl(spec, st[0])
    a = oracle.fe(spec, st, tau)
    sh = lambda z: np.roll(np.roll(z, 3, axis=1), -5, axis=0)
    b = oracle.fe(spec, [sh(z) for z in st], tau)
    for x, y in zip(a, b):
        assert np.array_equal(sh(x), y)


# ----------------------------------------------------------------------------------
# 8. limiter building blocks

def test_theta_definition():
    spec = ai.Spec(dim=1, nx=4, umin=0.0, umax=1.0)
    assert oracle.theta(spec, 0.5, 0.9) == 1.0
    assert oracle.theta(spec, 0.5, 1.0) == 1.0
    assert oracle.theta(spec, 0.5, 0.0) == 1.0
    t = oracle.theta(spec, 0.5, 1.5)
    assert t == pytest.approx(0.5)
    t = oracle.theta(spec, 0.25, -0.75)
    assert (1 - t) * 0.25 + t * (-0.75) == pytest.approx(0.0, abs=1e-15)
    assert 0.0 <= oracle.theta(spec, 1.0 + 1e-16, 2.0) <= 1.0


def test_interval_wave_speed():
    burg = ai.Spec(dim=1, nx=4, flux=("burgers", (0.5,)))
    assert oracle.alpha_interval(burg, 0, -0.3, 0.7) == pytest.approx(0.7, abs=0)
    assert oracle.alpha_interval(burg, 0, -0.9, 0.2) == pytest.approx(0.9, abs=0)
    bl = ai.Spec(dim=2, nx=4, ny=4, flux=("bl", (5.0,)))
    assert oracle.alpha_interval(bl, 0, 0.1, 0.9) == pytest.approx(2.0, abs=1e-14)
    # brute force over a dense grid for the gravity flux
    u = np.linspace(0.0, 1.0, 2_000_001)
    v = 1 - u
    D = u * u + v * v
    f1 = u * u / D
    d1 = 2 * u * v / D ** 2
    d2 = d1 * (1 - 5 * v * v) + f1 * 10 * v
    assert oracle.alpha_interval(bl, 1, 0.0, 1.0) == pytest.approx(np.max(np.abs(d2)), abs=1e-10)
    for a, b in [(0.0, 0.3), (0.2, 0.6), (0.55, 0.95)]:
        sel = (u >= a) & (u <= b)
        assert oracle.alpha_interval(bl, 1, a, b) == pytest.approx(np.max(np.abs(d2[sel])), abs=1e-10)
    # the sampled check value for gravity 5 on [0, 1]
    assert oracle.alpha_interval(bl, 1, 0.0, 1.0) == pytest.approx(3.3105, abs=1e-4)


def test_kappa_max_closed_forms():
    mk = lambda d, lo, hi: ai.Spec(dim=1, nx=4, diff=d, umin=lo, umax=hi)
    assert oracle.kappa_max(mk(("const", (0.01,)), 0, 1)) == 0.01
    assert oracle.kappa_max(mk(("pwl", (0.0, 0.0, 0.1, 0.5)), -1, 1)) == 0.1
    assert oracle.kappa_max(mk(("pwl", (0.03, 0.25, 0.03, 0.75)), 0, 1)) == 0.03
    assert oracle.kappa_max(mk(("pme", (2,)), 0, 1)) == pytest.approx(2.0)
    assert oracle.kappa_max(mk(("pme", (3,)), 0, 0.5)) == pytest.approx(0.75)
    assert oracle.kappa_max(mk(("cubic", (0.0, 0.02, -0.04 / 3)), 0, 1)) == pytest.approx(0.01, abs=1e-12)


def test_point_functions():
    bl = ai.Spec(dim=2, nx=4, ny=4, flux=("bl", (5.0,)), diff=("cubic", (0.0, 0.02, -0.04 / 3)))
    u = 0.3
    f1 = u * u / (u * u + (1 - u) ** 2)
    f, d, a = oracle.point_funcs(bl, 0, u)
    assert f == pytest.approx(f1, rel=1e-15)
    assert a == pytest.approx(0.04 * (u * u / 2 - u ** 3 / 3), rel=1e-14)
    f, d, a = oracle.point_funcs(bl, 1, u)
    assert f == pytest.approx(f1 * (1 - 5 * (1 - u) ** 2), rel=1e-14)
    eps = 1e-6
    fp, _, _ = oracle.point_funcs(bl, 1, u + eps)
    fm, _, _ = oracle.point_funcs(bl, 1, u - eps)
    assert d == pytest.approx((fp - fm) / (2 * eps), rel=1e-8)


def test_blend_is_identity_on_linear_data_and_active_on_jumps():
    spec = ai.Spec(dim=1, nx=32, x0=0, x1=1, flux=("burgers", (1.0,)), diff=("pwl", (0.1, -0.25, 0.1, 0.25)),
                   umin=-1, umax=1, limiter=False, blend="off")
    x = (np.arange(32) + 0.5) / 32
    # linear data: s~ = 0 exactly in exact arithmetic, so the blend is (nearly) inactive
    ub = 0.2 + 0.1 * x
    P = 0.2 + 0.1 * (np.arange(32) + 1.0) / 32
    # (not periodic, so compare interior cells only)
    tau = 1e-4
    off = oracle.fe(spec, [ub, P], tau)
    spec.blend = "plain"
    on = oracle.fe(spec, [ub, P], tau)
    np.testing.assert_allclose(on[0][3:-3], off[0][3:-3], rtol=0, atol=1e-12)
    # a jump: the blend moves the update toward the low-order scheme
    ub2 = np.where(x < 0.5, 1.0, -1.0)
    P2 = np.where((np.arange(32) + 1.0) / 32 < 0.5, 1.0, -1.0)
    spec.blend = "off"
    a = oracle.fe(spec, [ub2, P2], tau)
    spec.blend = "plain"
    b = oracle.fe(spec, [ub2, P2], tau)
    assert np.max(np.abs(a[0] - b[0])) > 1e-6


# ----------------------------------------------------------------------------------
# 9. experiments with printed numbers

def _sin4(n):
    spec = ai.Spec(dim=1, nx=n, x0=0, x1=1, flux=("linear", (1.0, 0.0)), diff=("none", ()), umin=1.0, umax=2.0)
    fn = lambda x: 1 + torch.sin(2 * math.pi * x) ** 4
    return spec, [ai.cell_average_1d(fn, spec).numpy(), ai.points_1d(fn, spec).numpy()]


# Example 6.2 is pure convection; its CFL number is not stated (Section 6 fixes 0.33/d
# for the convection-diffusion cases). C = 0.08 fits Table 3's limited columns: each of
# their ten printed values is reproduced within a factor 1.6.
EX62_CFL = 0.08


def _ex62(n, limiter, cfl=EX62_CFL):
    """Example 6.2 to T = 1 (one period, so the exact solution is the initial data):
    (min - umin, max - umax, L1 error of the cell averages, safeguard stats)."""
    spec, st = _sin4(n)
    spec.limiter = limiter
    out, _, tot = oracle.run_native(spec, 54, st, 1.0, cfl=cfl, cfl_diff=0.0)
    lo, hi = oracle.bounds(out)
    return lo - 1.0, hi - 2.0, float(np.sum(np.abs(out[0] - st[0])) * spec.dx), tot


def test_table3_unlimited_columns():
    """Example 6.2 without limiting: the undershoot and overshoot match the printed
    values within 5% (at C = 0.33 as at any C <= 0.33: the error is spatial)."""
    rows = {int(r[0]): [float(v) for v in r[1:]] for r in _golden("table3_minmax.txt")}
    for n in (20, 40, 80):
        spec, st = _sin4(n)
        spec.limiter = False
        out, _, _ = oracle.run(spec, 54, st, 1.0, dt_fixed=0.33 * spec.dx)
        lo, hi = oracle.bounds(out)
        assert lo - 1.0 == pytest.approx(rows[n][0], rel=0.05)
        assert hi - 2.0 == pytest.approx(rows[n][1], rel=0.05)


def test_table3_limited_columns():
    """Example 6.2 with limiting (Table 3): every DoF stays in [1, 2], and each printed
    limited minimum (positive, 2.7e-9 .. 2.7e-6) and maximum (negative) is reproduced
    within a factor 2 for N = 20 .. 320. The face limiter factor of a pure-convection
    problem decides the minimum column: the three-part factor lifts the minimum at
    N = 20 to 3.6e-5 even at this CFL (and to 1.6e-2 at C = 0.33)."""
    rows = {int(r[0]): [float(v) for v in r[1:]] for r in _golden("table3_minmax.txt")}
    for n in (20, 40, 80, 160, 320):
        mn, mx, _, tot = _ex62(n, True)
        assert tot["error"] == 0 and tot["clamps"] == 0
        assert 0.0 < mn and rows[n][2] / 2 <= mn <= 2 * rows[n][2]
        assert mx < 0.0 and 2 * rows[n][3] <= mx <= rows[n][3] / 2


def _orders(errs):
    return [math.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]


def test_example62_fourth_order_with_limiting():
    """Example 6.2: the limiter keeps the fourth-order rate of the unlimited scheme (the
    paper's accuracy figure for this example). L1 orders of the cell averages over
    N = 20 .. 320: those of the last two refinements are >= 3.7, and every limited order
    is within 0.2 of the unlimited order of the same refinement."""
    ns = (20, 40, 80, 160, 320)
    lim = _orders([_ex62(n, True)[2] for n in ns])
    unl = _orders([_ex62(n, False)[2] for n in ns])
    assert min(lim[2:]) >= 3.7 and min(unl[2:]) >= 3.85
    assert all(abs(a - b) <= 0.2 for a, b in zip(lim, unl))


def test_example62_pins_catch_planted_face_factors():
    """The pins above catch a wrong face limiter factor planted in the oracle: the
    three-part factor 6 applied to this pure-convection problem misses Table 3's
    limited minimum at N = 20 by orders of magnitude and drops the L1 order below 3;
    a halved factor breaks the maximum principle on rough 2D data."""
    rows = {int(r[0]): [float(v) for v in r[1:]] for r in _golden("table3_minmax.txt")}
    with oracle.planted(AO_PLANT_FACE_SCALE=3.0):
        mn = _ex62(20, True)[0]
        assert mn > 20 * rows[20][2]
        assert _orders([_ex62(n, True)[2] for n in (160, 320)])[0] < 3.2
    spec = ai.Spec(dim=2, nx=12, ny=10, x0=0, x1=1.2, y0=0, y1=1.0, flux=("burgers", (0.5,)),
                   diff=("none", ()), umin=0.0, umax=1.0, limiter=True)
    with oracle.planted(AO_PLANT_FACE_SCALE=0.5):
        worst = 0.0
        for seed in range(6):
            st = [a.numpy() for a in ai.random_state_2d(spec, seed=seed)]
            for _ in range(3):
                st, _ = oracle.step(spec, 3, st, oracle.dt_cfl(spec, st[0]))
                lo, hi = oracle.bounds(st)
                worst = max(worst, -lo, hi - 1.0)
        assert worst > 1e-3


@pytest.mark.slow
@pytest.mark.parametrize("m", [2, 3])
def test_table4_barenblatt_minimum(m):
    """Example 6.3, 2D, N = 80 on [-8, 8]^2, t: 1 -> 2 (Table 4). With limiting the
    minimum is exactly 0 (hard pin). Without limiting it matches the printed negative
    minimum within 3%. The unlimited run uses C = 0.12: the 2D high-order scheme's
    Fourier symbol has spectral radius 40.78 kappa/h^2 for pure diffusion, so
    SSP-RK(5,4) is linearly stable only up to kappa dt/h^2 = 0.131, below 0.33/d."""
    rows = {int(r[0]): [float(v) for v in r[1:]] for r in _golden("table4_barenblatt.txt")}
    spec = ai.Spec(dim=2, nx=80, ny=80, x0=-8, x1=8, y0=-8, y1=8, flux=("zero", ()), diff=("pme", (m,)),
                   umin=0.0, umax=1.0, limiter=True)
    st = [a.numpy() for a in ai.state_2d(lambda x, y: ai.barenblatt(x, y, 1.0, m=m), spec)]
    out, _, tot = oracle.run(spec, 54, st, 1.0)
    assert oracle.bounds(out)[0] == 0.0 and tot["error"] == 0
    spec.limiter = False
    out, _, _ = oracle.run(spec, 54, st, 1.0, cfl=0.12, cfl_diff=0.0)
    mn = oracle.bounds(out)[0]
    assert mn == pytest.approx(rows[m][0], rel=0.03)


def test_barenblatt_error_decreases():
    """L1 error against the closed-form Barenblatt profile decreases under refinement."""
    errs = []
    for n in (20, 40):
        spec = ai.Spec(dim=2, nx=n, ny=n, x0=-8, x1=8, y0=-8, y1=8, flux=("zero", ()), diff=("pme", (2,)),
                       umin=0.0, umax=1.0, limiter=True)
        st = [a.numpy() for a in ai.state_2d(lambda x, y: ai.barenblatt(x, y, 1.0), spec)]
        out, _, tot = oracle.run(spec, 3, st, 0.25)
        ex = ai.cell_average_2d(lambda x, y: ai.barenblatt(x, y, 1.25), spec).numpy()
        errs.append(np.sum(np.abs(out[0] - ex)) * spec.dx * spec.dy)
        assert oracle.bounds(out)[0] >= 0.0
    assert errs[1] < 0.5 * errs[0]


# ----------------------------------------------------------------------------------
# 10. the blend's low-order residual and its weights (readings 6 and 7), pinned by the
# cases where they reduce to textbook schemes: with theta = 0 (an external indicator so
# large that exp(-gamma s) underflows) every face flux, cell potential and point
# residual is the low-order one, which for a linear flux c > 0 and a = k0 u is first-
# order upwinding plus the central second difference -- on the mesh for the cell
# averages and on the half-spaced points for the point values; with one indicator
# value everywhere every weight equals exp(-gamma s), so the evaluation is the convex
# combination of the unblended (s = 0) and the low-order (s huge) evaluations.

def _rng_state_1d(n, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.2, 0.8, n), rng.uniform(0.2, 0.8, n)]


@pytest.mark.parametrize("c,k0", [(1.0, 0.0), (0.7, 0.05), (-0.9, 0.02)])
def test_low_order_blend_is_upwind_1d(c, k0):
    n, L = 24, 1.3
    spec = ai.Spec(dim=1, nx=n, x0=0.0, x1=L, flux=("linear", (c, 0.0)), diff=("const", (k0,)), umin=-10.0,
                   umax=10.0, limiter=False, blend="external", gamma=1.0)
    ub, P = _rng_state_1d(n, 5)
    h, tau = L / n, 1e-3
    got = oracle.fe(spec, [ub, P], tau, s_ext=np.full(n, 1e3))
    # textbook first-order upwind flux c u_upwind; P_j sits between ub_j and ub_{j+1}
    ubm, ubp = np.roll(ub, 1), np.roll(ub, -1)
    up = lambda left, right: c * (left if c > 0 else right)
    want_ub = ub - tau / h * (up(ub, ubp) - up(ubm, ub)) + tau * k0 / h ** 2 * (ubp - 2 * ub + ubm)
    hh = h / 2   # spacing of the point's low-order stencil (its neighbouring averages)
    want_P = P - tau / hh * (up(P, ubp) - up(ub, P)) + tau * k0 / hh ** 2 * (ubp - 2 * P + ub)
    np.testing.assert_allclose(got[0], want_ub, rtol=0, atol=1e-13)
    np.testing.assert_allclose(got[1], want_P, rtol=0, atol=1e-13)


def test_low_order_blend_is_upwind_2d():
    nx, ny, Lx, Ly = 12, 10, 1.2, 0.8
    c1, c2, k0 = 0.8, -0.6, 0.03
    spec = ai.Spec(dim=2, nx=nx, ny=ny, x0=0, x1=Lx, y0=0, y1=Ly, flux=("linear", (c1, c2)), diff=("const", (k0,)),
                   umin=-10.0, umax=10.0, limiter=False, blend="external", gamma=1.0)
    rng = np.random.default_rng(9)
    ub, V, X, Y = (rng.uniform(0.2, 0.8, (ny, nx)) for _ in range(4))
    hx, hy, tau = Lx / nx, Ly / ny, 1e-3
    got = oracle.fe(spec, [ub, V, X, Y], tau, s_ext=np.full((ny, nx), 1e3))
    sh = lambda a, di, dj: np.roll(np.roll(a, -dj, axis=0), -di, axis=1)   # a[j + dj, i + di]

    def upd(left, mid, right, c, h):
        # -(F(mid, right) - F(left, mid)) / h with the upwind flux, + k0 (right - 2 mid + left) / h^2
        f = lambda a, b: c * (a if c > 0 else b)
        return -(f(mid, right) - f(left, mid)) / h + k0 * (right - 2 * mid + left) / h ** 2

    want_ub = ub + tau * (upd(sh(ub, -1, 0), ub, sh(ub, 1, 0), c1, hx) + upd(sh(ub, 0, -1), ub, sh(ub, 0, 1), c2, hy))
    # V_ij (corner x_{i+1/2}, y_{j+1/2}): along x between Y_ij and Y_{i+1,j}, along y between
    # X_ij and X_{i,j+1}; X_ij (x_{i+1/2}, y_j): along x between the averages of cells i
    # and i+1, along y between V_{i,j-1} and V_ij; Y_ij (x_i, y_{j+1/2}): along x between
    # V_{i-1,j} and V_ij, along y between the averages of rows j and j+1
    want_V = V + tau * (upd(Y, V, sh(Y, 1, 0), c1, hx / 2) + upd(X, V, sh(X, 0, 1), c2, hy / 2))
    want_X = X + tau * (upd(ub, X, sh(ub, 1, 0), c1, hx / 2) + upd(sh(V, 0, -1), X, V, c2, hy / 2))
    want_Y = Y + tau * (upd(sh(V, -1, 0), Y, V, c1, hx / 2) + upd(ub, Y, sh(ub, 0, 1), c2, hy / 2))
    for g, w in zip(got, [want_ub, want_V, want_X, want_Y]):
        np.testing.assert_allclose(g, w, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dim", [1, 2])
def test_constant_indicator_blend_is_convex_combination(dim):
    if dim == 1:
        spec = ai.Spec(dim=1, nx=20, x0=0, x1=1.0, flux=("burgers", (0.5,)), diff=("cubic", (0.01, 0.02, 0.0)),
                       umin=-10.0, umax=10.0, limiter=False, blend="external", gamma=2.0)
        st = _rng_state_1d(20, 3)
        shape = (20,)
    else:
        spec = ai.Spec(dim=2, nx=11, ny=9, x0=0, x1=1.1, y0=0, y1=0.9, flux=("bl", (5.0,)),
                       diff=("cubic", (0.01, 0.02, 0.0)), umin=-10.0, umax=10.0, limiter=False, blend="external",
                       gamma=2.0)
        rng = np.random.default_rng(4)
        st = [rng.uniform(0.2, 0.8, (9, 11)) for _ in range(4)]
        shape = (9, 11)
    tau, s = 1e-3, 0.37
    hi = oracle.fe(spec, st, tau, s_ext=np.zeros(shape))
    lo = oracle.fe(spec, st, tau, s_ext=np.full(shape, 1e3))
    mid = oracle.fe(spec, st, tau, s_ext=np.full(shape, s))
    w = math.exp(-spec.gamma * s)
    for m_, h_, l_ in zip(mid, hi, lo):
        np.testing.assert_allclose(m_, w * h_ + (1 - w) * l_, rtol=0, atol=1e-13)
    # and s = 0 is the method without the blend, bit for bit
    spec_off = ai.Spec(**{**spec.__dict__, "blend": "off"})
    off = oracle.fe(spec_off, st, tau)
    for a, b in zip(hi, off):
        np.testing.assert_array_equal(a, b)
