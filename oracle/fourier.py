"""Fourier and von Neumann analysis of the 1D linear AF scheme (Section 3).

Test infrastructure only. ``G_printed`` is the semi-discrete Fourier matrix exactly as
the paper prints it (eq. 1d_fourier_ode, Section 3.1); ``G_from_oracle`` measures the
same matrix by applying the oracle's forward-Euler operator to discrete Fourier modes, so
the tests can check one against the other. ``max_stable_cfl`` is the grid search of
Section 3.2 over xi for the stability polynomials R(z) of SSP-RK3, RK4 and SSP-RK(5,4).
"""
import math

import numpy as np

ETA_RK54 = 0.004477718303076   # z^5 coefficient of the SSP-RK(5,4) polynomial (Section 3.2)


def G_parts_printed(xi: float):
    """(G_c, G_d) of eq. 1d_fourier_ode with t_x = exp(i xi)."""
    t = np.exp(1j * xi)
    ti = 1.0 / t
    Gc = np.array([[0.0, ti - 1.0],
                   [3.0 - t, (-5.0 * ti - 8.0 + t) / 6.0]], dtype=complex)
    Gd = np.array([[2.0 * (ti - 2.0 + t), 0.5 * (-ti * ti + ti + 1.0 - t)],
                   [8.0 * (1.0 + t), -(5.0 * ti + 38.0 + 5.0 * t) / 3.0]], dtype=complex)
    return Gc, Gd


def G_printed(xi: float, c: float, k0: float, dx: float):
    Gc, Gd = G_parts_printed(xi)
    return (c / dx) * Gc + (k0 / dx ** 2) * Gd


def G_from_oracle(n: int, k: int, c: float, k0: float, length: float = 2 * math.pi):
    """Measure G at xi = 2 pi k / n from the oracle: apply the semi-discrete operator
    (FE(u, tau) - u) / tau, which is exact for a linear scheme, to the real and
    imaginary parts of the modes (1,0) exp(i w x_i) and (0,1) exp(i w x_i)."""
    import af_inputs
    import oracle

    spec = af_inputs.Spec(dim=1, nx=n, x0=0.0, x1=length, flux=("linear", (c, 0.0)),
                          diff=("const", (k0,)), umin=-10.0, umax=10.0, limiter=False)
    dx = spec.dx
    w = 2 * math.pi * k / length
    xc = (np.arange(n) + 0.5) * dx
    ph = np.exp(1j * w * xc)
    tau = 1.0  # the scheme is linear, so (FE - u)/tau is independent of tau

    def apply(u_hat):
        # complex mode -> real and imaginary parts separately
        out = np.zeros((2, n), dtype=complex)
        for part, fac in ((np.real, 1.0), (np.imag, 1j)):
            ub = part(u_hat[0] * ph)
            P = part(u_hat[1] * ph)
            nb, nP = oracle.fe(spec, [ub, P], tau)
            out[0] += fac * (nb - ub) / tau
            out[1] += fac * (nP - P) / tau
        return out

    G = np.zeros((2, 2), dtype=complex)
    for col, uh in enumerate(([1.0, 0.0], [0.0, 1.0])):
        r = apply(np.array(uh, dtype=complex))
        # read the coefficient at cell 0 (every cell gives the same value)
        G[0, col] = r[0][0] / ph[0]
        G[1, col] = r[1][0] / ph[0]
    return G, dx


def R_poly(name: str):
    """Stability polynomial coefficients (ascending powers)."""
    base = [1.0, 1.0, 0.5, 1.0 / 6.0]
    if name == "ssprk3":
        return base
    if name == "rk4":
        return base + [1.0 / 24.0]
    if name == "ssprk54":
        return base + [1.0 / 24.0, ETA_RK54]
    raise KeyError(name)


def amplification_radius(M: np.ndarray, coefs) -> float:
    """Spectral radius of R(M) for a 2x2 matrix M."""
    ev = np.linalg.eigvals(M)
    vals = [abs(sum(cf * z ** p for p, cf in enumerate(coefs))) for z in ev]
    return max(vals)


def max_stable_cfl(rk: str, r: float, nxi: int = 721, hi: float = 2.0, tol: float = 1e-10) -> float:
    """Largest C_CFL with spectral radius of R(C [r G_c + (1-r) G_d]) <= 1 for all xi on a
    uniform grid of [-pi, pi] (Section 3.2), by bisection on C."""
    coefs = R_poly(rk)
    xis = np.linspace(-math.pi, math.pi, nxi)
    mats = []
    for xi in xis:
        Gc, Gd = G_parts_printed(xi)
        mats.append(r * Gc + (1.0 - r) * Gd)

    def stable(C):
        return all(amplification_radius(C * M, coefs) <= 1.0 + 1e-12 for M in mats)

    lo = 0.0
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return lo
