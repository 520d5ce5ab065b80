"""Seeded synthetic problem descriptions and initial data.

This module holds problem set-up only -- mesh geometry, initial functions, their cell
averages by quadrature and their point values -- and none of the numerical method's
arithmetic. Both the CUDA path's tests/benchmark and the CPU oracle consume the arrays
it produces, so the two sides always start from identical inputs.

Layout of a 2D state (periodic, row-major [ny][nx], i fastest):
  ub[j,i] cell average, V[j,i] at (x_{i+1/2}, y_{j+1/2}), X[j,i] at (x_{i+1/2}, y_j),
  Y[j,i] at (x_i, y_{j+1/2}).  A 1D state is (ub[i], P[i] = u(x_{i+1/2})); on a 1D
  interval with Dirichlet or outflow ends P has nx+1 entries, P[k] = u(x0 + k dx). A 2D
  rectangle with outflow ends has V [ny+1][nx+1] at (x0 + k dx, y0 + l dy), X [ny][nx+1]
  at (x0 + k dx, y_j) and Y [ny+1][nx] at (x_i, y0 + l dy).

Cell averages use a tensor Gauss-Legendre rule on sub-cells (exact closed forms for
single Fourier modes); point values are exact evaluations. Disc indicators use the
strict inequality.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Sequence, Tuple

import numpy as np
import torch


@dataclasses.dataclass
class Spec:
    """Problem description: mesh, flux, diffusion potential, bounds, options.

    flux: ("zero", ()), ("linear", (cx, cy)), ("burgers", (coef,)) for f = coef*u^2 in
          every direction, ("bl", (g,)) for f1 = u^2/(u^2+(1-u)^2), f2 = f1*(1-g(1-u)^2)
          (in 1D, f = f1*(1-g(1-u)^2)).
    diff: ("none", ()), ("const", (k0,)) for a = k0*u,
          ("pwl", (klo, lo, khi, hi)) for a = klo*min(u-lo,0) + khi*max(u-hi,0),
          ("pme", (m,)) for a = u^m, ("cubic", (c1, c2, c3)) for a = c1 u + c2 u^2 + c3 u^3,
          ("ramp", (k, lo, w)) for a = 0 (u <= lo), k (u-lo)^2/(2w) (lo < u < lo+w),
          k (u - lo - w/2) (u >= lo+w), ("cubic01", (c1, c2, c3)) for the cubic at
          min(max(u, 0), 1).
    blend: "off", "plain" (smoothness indicator) or "external" (per-cell indicator input).
    bc: "periodic", "outflow" (1D or 2D), or in 1D "dirichlet" (end values bc_values).
    diffusion_form: "dc" (doubly conservative) or, in 1D, "nodc" (the diffusion
          discretization without double conservation of Appendix A).
    """
    dim: int
    nx: int
    ny: int = 1
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    flux: Tuple[str, Sequence[float]] = ("zero", ())
    diff: Tuple[str, Sequence[float]] = ("none", ())
    umin: float = 0.0
    umax: float = 1.0
    limiter: bool = True
    blend: str = "off"
    gamma: float = 1.0
    rk: int = 3
    cfl: float = 0.0          # 0 -> 0.33/d (the paper's experiments)
    T: float = 0.0
    name: str = ""
    bc: str = "periodic"
    bc_values: Tuple[float, float] = (0.0, 0.0)
    diffusion_form: str = "dc"
    nz: int = 1
    z0: float = 0.0
    z1: float = 1.0

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny if self.dim >= 2 else 1.0

    @property
    def dz(self) -> float:
        return (self.z1 - self.z0) / self.nz if self.dim == 3 else 1.0

    @property
    def cells(self) -> int:
        return self.nx * (self.ny if self.dim >= 2 else 1) * (self.nz if self.dim == 3 else 1)

    def with_size(self, nx: int, ny: int | None = None, nz: int | None = None) -> "Spec":
        return dataclasses.replace(self, nx=nx, ny=(ny if ny is not None else (nx if self.dim >= 2 else 1)),
                                   nz=(nz if nz is not None else (nx if self.dim == 3 else 1)))


# ----------------------------------------------------------------------------------
# quadrature

def _gauss(order: int):
    x, w = np.polynomial.legendre.leggauss(order)
    return x, w


def cell_average_2d(func: Callable, spec: Spec, sub: int = 4, order: int = 5,
                    device="cpu", row_chunk: int = 64) -> torch.Tensor:
    """Cell averages of func(x, y) by a tensor Gauss rule on sub x sub sub-cells."""
    gx, gw = _gauss(order)
    # local offsets inside a unit cell [0,1]
    offs = []
    wts = []
    for s in range(sub):
        for q in range(order):
            offs.append((s + 0.5 + 0.5 * gx[q]) / sub)
            wts.append(gw[q] / (2 * sub))
    offs = torch.tensor(offs, dtype=torch.float64, device=device)
    wts = torch.tensor(wts, dtype=torch.float64, device=device)
    nx, ny = spec.nx, spec.ny
    dx, dy = spec.dx, spec.dy
    out = torch.empty((ny, nx), dtype=torch.float64, device=device)
    xs = spec.x0 + (torch.arange(nx, dtype=torch.float64, device=device)[:, None] + offs[None, :]) * dx
    for j0 in range(0, ny, row_chunk):
        j1 = min(ny, j0 + row_chunk)
        ys = spec.y0 + (torch.arange(j0, j1, dtype=torch.float64, device=device)[:, None] + offs[None, :]) * dy
        # shape (rows, qy, nx, qx)
        Xg = xs[None, None, :, :]
        Yg = ys[:, :, None, None]
        vals = func(Xg, Yg)
        avg = torch.einsum("rqnp,q,p->rn", vals, wts, wts)
        out[j0:j1] = avg
    return out


def cell_average_1d(func: Callable, spec: Spec, sub: int = 4, order: int = 5, device="cpu") -> torch.Tensor:
    gx, gw = _gauss(order)
    offs, wts = [], []
    for s in range(sub):
        for q in range(order):
            offs.append((s + 0.5 + 0.5 * gx[q]) / sub)
            wts.append(gw[q] / (2 * sub))
    offs = torch.tensor(offs, dtype=torch.float64, device=device)
    wts = torch.tensor(wts, dtype=torch.float64, device=device)
    xs = spec.x0 + (torch.arange(spec.nx, dtype=torch.float64, device=device)[:, None] + offs[None, :]) * spec.dx
    return (func(xs) * wts[None, :]).sum(dim=1)


def points_2d(func: Callable, spec: Spec, device="cpu"):
    """Exact point values (V, X, Y) of func(x, y) (a rectangle with ends also holds the
    values on its left and bottom sides)."""
    i = torch.arange(spec.nx, dtype=torch.float64, device=device)
    j = torch.arange(spec.ny, dtype=torch.float64, device=device)
    xc = spec.x0 + (i + 0.5) * spec.dx   # x_i
    xf = spec.x0 + (i + 1.0) * spec.dx   # x_{i+1/2}
    yc = spec.y0 + (j + 0.5) * spec.dy
    yf = spec.y0 + (j + 1.0) * spec.dy
    if spec.bc != "periodic":
        xf = spec.x0 + torch.arange(spec.nx + 1, dtype=torch.float64, device=device) * spec.dx
        yf = spec.y0 + torch.arange(spec.ny + 1, dtype=torch.float64, device=device) * spec.dy
    V = func(xf[None, :], yf[:, None])
    X = func(xf[None, :], yc[:, None])
    Y = func(xc[None, :], yf[:, None])
    return V, X, Y


def points_1d(func: Callable, spec: Spec, device="cpu"):
    """Point values u(x_{i+1/2}), i = 0..nx-1 (periodic), or u(x0 + k dx), k = 0..nx
    (an interval with boundary conditions)."""
    if spec.bc != "periodic":
        k = torch.arange(spec.nx + 1, dtype=torch.float64, device=device)
        return func(spec.x0 + k * spec.dx)
    i = torch.arange(spec.nx, dtype=torch.float64, device=device)
    return func(spec.x0 + (i + 1.0) * spec.dx)


def state_1d(func: Callable, spec: Spec, device="cpu", sub: int = 4, order: int = 5) -> List[torch.Tensor]:
    return [cell_average_1d(func, spec, sub=sub, order=order, device=device).contiguous(),
            points_1d(func, spec, device=device).contiguous()]


def state_2d(func: Callable, spec: Spec, device="cpu", sub: int = 4, order: int = 5) -> List[torch.Tensor]:
    ub = cell_average_2d(func, spec, sub=sub, order=order, device=device)
    V, X, Y = points_2d(func, spec, device=device)
    return [ub.contiguous(), V.contiguous(), X.contiguous(), Y.contiguous()]


# ----------------------------------------------------------------------------------
# initial functions

def sine_1d_state(spec: Spec, device="cpu"):
    """u0 = sin(x): closed-form cell averages (2/dx) sin(dx/2) sin(x_i)."""
    i = torch.arange(spec.nx, dtype=torch.float64, device=device)
    xc = spec.x0 + (i + 0.5) * spec.dx
    ub = (2.0 / spec.dx) * math.sin(spec.dx / 2) * torch.sin(xc)
    P = torch.sin(spec.x0 + (i + 1.0) * spec.dx)
    return [ub, P]


def mode_1d_state(spec: Spec, k: float, shift: float = 1.0, amp: float = 1.0, device="cpu"):
    """u0 = shift + amp*sin(k x) with closed-form cell averages."""
    i = torch.arange(spec.nx, dtype=torch.float64, device=device)
    xc = spec.x0 + (i + 0.5) * spec.dx
    fac = math.sin(k * spec.dx / 2) / (k * spec.dx / 2)
    ub = shift + amp * fac * torch.sin(k * xc)
    P = shift + amp * torch.sin(k * (spec.x0 + (i + 1.0) * spec.dx))
    return [ub, P]


def mode_2d_state(spec: Spec, k: float, shift: float = 1.0, amp: float = 1.0, device="cpu"):
    """u0 = shift + amp*sin(k (x + y)) (Example 6.1 in 2D) with closed-form averages."""
    i = torch.arange(spec.nx, dtype=torch.float64, device=device)
    j = torch.arange(spec.ny, dtype=torch.float64, device=device)
    xc = spec.x0 + (i + 0.5) * spec.dx
    yc = spec.y0 + (j + 0.5) * spec.dy
    fx = math.sin(k * spec.dx / 2) / (k * spec.dx / 2)
    fy = math.sin(k * spec.dy / 2) / (k * spec.dy / 2)
    ub = shift + amp * fx * fy * torch.sin(k * (xc[None, :] + yc[:, None]))
    f = lambda x, y: shift + amp * torch.sin(k * (x + y))
    V, X, Y = points_2d(f, spec, device=device)
    return [ub.contiguous(), V.contiguous(), X.contiguous(), Y.contiguous()]


def discs_fn(x, y):
    """+1 on the disc r<0.35 about (-0.5,-0.5), -1 on the disc r<0.35 about (0.5,0.5)."""
    r1 = (x + 0.5) ** 2 + (y + 0.5) ** 2
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2
    return (r1 < 0.35 ** 2).to(torch.float64) - (r2 < 0.35 ** 2).to(torch.float64)


def barenblatt(x, y, t: float, m: int = 2, d: int = 2):
    """Barenblatt profile B_m(x, t) (Example 6.3)."""
    alpha = 1.0 / (m - 1 + 2.0 / d)
    r2 = x * x + y * y
    core = 1.0 - alpha * (m - 1) / (2.0 * d * m) * r2 / (t ** (2 * alpha / d))
    return t ** (-alpha) * torch.clamp(core, min=0.0) ** (1.0 / (m - 1))


def two_hills_fn(x, y):
    """Example 6.4: exp(-1/(6 - r^2)) inside r^2 < 6 about (2, -2) and about (-2, 2), 0
    elsewhere (the two supports are disjoint)."""
    out = torch.zeros(torch.broadcast_shapes(x.shape, y.shape), dtype=torch.float64, device=x.device)
    for cx, cy in ((2.0, -2.0), (-2.0, 2.0)):
        r2 = (x - cx) ** 2 + (y - cy) ** 2
        inside = r2 < 6.0
        out = out + torch.where(inside, torch.exp(-1.0 / torch.where(inside, 6.0 - r2, 1.0)), torch.zeros_like(out))
    return out


def two_hills(n: int = 100, limiter: bool = True) -> Spec:
    """Example 6.4 (collision of two hills): u_t = Lap(u^2) on the periodic [-10, 10]^2,
    T = 4; bounds [0, exp(-1/6)], the range of the initial data."""
    return Spec(dim=2, nx=n, ny=n, x0=-10.0, x1=10.0, y0=-10.0, y1=10.0, flux=("zero", ()), diff=("pme", (2,)),
                umin=0.0, umax=math.exp(-1.0 / 6.0), limiter=limiter, rk=3, T=4.0, name="two_hills")


def bl_disc_fn(x, y, radius: float = 0.5):
    return ((x * x + y * y) < radius * radius).to(torch.float64)


def fourier8_fn(A, p, q, phi):
    """clip(0.5 + sum_k A_k sin(2 pi (p_k x + q_k y) + phi_k), 0, 1)."""
    def f(x, y):
        s = torch.full(torch.broadcast_shapes(x.shape, y.shape), 0.5, dtype=torch.float64, device=x.device)
        for k in range(len(A)):
            s = s + A[k] * torch.sin(2 * math.pi * (p[k] * x + q[k] * y) + phi[k])
        return torch.clamp(s, 0.0, 1.0)
    return f


# ----------------------------------------------------------------------------------
# the five benchmark workloads

def config1(n: int = 128) -> Spec:
    """1D linear u_t + u_x = 0.01 u_xx on [0, 2 pi], SSP-RK3, limiter off, T = 1."""
    return Spec(dim=1, nx=n, x0=0.0, x1=2 * math.pi, flux=("linear", (1.0, 0.0)), diff=("const", (0.01,)),
                umin=-1.0, umax=1.0, limiter=False, rk=3, T=1.0, name="linear1d")


def config1_dt(spec: Spec, frac: float = 0.9, cfl_limit: float = 0.5611) -> float:
    """dt with dt*(c/dx + k0/dx^2) = frac * (SSP-RK3 von Neumann limit at this Peclet number)."""
    c, k0 = spec.flux[1][0], spec.diff[1][0]
    return frac * cfl_limit / (c / spec.dx + k0 / spec.dx ** 2)


def evje_karlsen(n: int = 200, diffusion_form: str = "dc") -> Spec:
    """Example 6.5 (Evje and Karlsen): f = u^2/4, a = 0 (u <= 0.5), 5(2u-1)^2/4
    (0.5 < u < 0.6), u - 11/20 (u >= 0.6) on [-1, 1], Dirichlet u(-1) = 1, u(1) = 0,
    MPP limiting, T = 1."""
    return Spec(dim=1, nx=n, x0=-1.0, x1=1.0, flux=("burgers", (0.25,)), diff=("ramp", (1.0, 0.5, 0.1)),
                umin=0.0, umax=1.0, limiter=True, rk=3, T=1.0, name="evje_karlsen", bc="dirichlet",
                bc_values=(1.0, 0.0), diffusion_form=diffusion_form)


def evje_karlsen_fn(x):
    """1 on [-1, -0.4), -2.5 x on [-0.4, 0), 0 otherwise."""
    return torch.where(x < -0.4, torch.ones_like(x), torch.where(x < 0.0, -2.5 * x, torch.zeros_like(x)))


def strongly_degenerate_1d(n: int = 100, blend: str = "plain", limiter: bool = True,
                           diffusion_form: str = "dc") -> Spec:
    """Example 6.8: f = u^2, a = 0.1 (u + 0.25) (u <= -0.25), 0.1 (u - 0.25) (u >= 0.25),
    0 otherwise, on [-2, 2] with outflow ends, T = 0.7, bounds [-1, 1]."""
    return Spec(dim=1, nx=n, x0=-2.0, x1=2.0, flux=("burgers", (1.0,)), diff=("pwl", (0.1, -0.25, 0.1, 0.25)),
                umin=-1.0, umax=1.0, limiter=limiter, blend=blend, gamma=1.0, rk=3, T=0.7,
                name="strongly_degenerate1d", bc="outflow", diffusion_form=diffusion_form)


def strongly_degenerate_fn(x):
    """1 where |x + 1/sqrt(2)| < 0.4, -1 where |x - 1/sqrt(2)| < 0.4, 0 otherwise."""
    r = 1.0 / math.sqrt(2.0)
    one = torch.ones_like(x)
    return torch.where((x + r).abs() < 0.4, one, torch.where((x - r).abs() < 0.4, -one, torch.zeros_like(x)))


def buckley_leverett_1d(n: int = 100, gravity: bool = False, problem: str = "ibvp") -> Spec:
    """Example 6.6: f = u^2/(u^2+(1-u)^2), times 1 - 5(1-u)^2 with gravity; a = eps
    (2u^2 - 4u^3/3) on [0, 1] (0 below, 2 eps/3 above), eps = 0.01; [0, 1] with Dirichlet
    ends, MPP limiting, T = 1. problem "ibvp": u0 = 1 - 3x on [0, 1/3), 0 otherwise, ends
    u(0) = 1, u(1) = 0. "rp": u0 = 0 on [0, 1 - 1/sqrt(2)), 1 otherwise; its ends hold the
    initial data's end values 0 and 1."""
    eps = 0.01
    return Spec(dim=1, nx=n, x0=0.0, x1=1.0, flux=("bl", (5.0 if gravity else 0.0,)),
                diff=("cubic01", (0.0, 2.0 * eps, -4.0 * eps / 3.0)), umin=0.0, umax=1.0, limiter=True, rk=3,
                T=1.0, name=f"buckley_leverett1d_{problem}", bc="dirichlet",
                bc_values=(1.0, 0.0) if problem == "ibvp" else (0.0, 1.0))


def bl1d_ibvp_fn(x):
    """1 - 3x on [0, 1/3), 0 otherwise"""
    return torch.where(x < 1.0 / 3.0, 1.0 - 3.0 * x, torch.zeros_like(x))


def bl1d_rp_fn(x):
    """0 on [0, 1 - 1/sqrt(2)), 1 otherwise"""
    return torch.where(x < 1.0 - 1.0 / math.sqrt(2.0), torch.zeros_like(x), torch.ones_like(x))


def buckley_leverett_2d_outflow(n: int = 100, limiter: bool = True) -> Spec:
    """Example 6.7: f = u^2/(u^2+(1-u)^2), g = f (1 - 5(1-u)^2), a = 0.01 u on
    [-1.5, 1.5]^2 with outflow ends, u0 = 1 on x^2 + y^2 < 1/2, T = 0.5."""
    return Spec(dim=2, nx=n, ny=n, x0=-1.5, x1=1.5, y0=-1.5, y1=1.5, flux=("bl", (5.0,)), diff=("const", (0.01,)),
                umin=0.0, umax=1.0, limiter=limiter, rk=3, T=0.5, name="buckley_leverett2d_outflow", bc="outflow")


def strongly_degenerate_2d(n: int = 100, blend: str = "plain") -> Spec:
    """Example 6.9: f = g = u^2, a = 0.1 (u - 1/4) (u > 1/4), 0.1 (u + 1/4) (u < -1/4), 0
    otherwise, on [-1.5, 1.5]^2 with outflow ends, discs +-1 of radius 2/5 about
    (-1/2, -1/2) / (1/2, 1/2), T = 0.5."""
    return Spec(dim=2, nx=n, ny=n, x0=-1.5, x1=1.5, y0=-1.5, y1=1.5, flux=("burgers", (1.0,)),
                diff=("pwl", (0.1, -0.25, 0.1, 0.25)), umin=-1.0, umax=1.0, limiter=True, blend=blend, gamma=1.0,
                rk=3, T=0.5, name="strongly_degenerate2d", bc="outflow")


def strongly_degenerate_2d_fn(x, y):
    r1 = (x + 0.5) ** 2 + (y + 0.5) ** 2
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2
    return (r1 < 4.0 / 25.0).to(torch.float64) - (r2 < 4.0 / 25.0).to(torch.float64)


def config2(n: int = 1024) -> Spec:
    """2D strongly degenerate Burgers: f = u^2/2, kappa = 0.1 [u > 0.5], discs +-1."""
    return Spec(dim=2, nx=n, ny=n, x0=-1.5, x1=1.5, y0=-1.5, y1=1.5, flux=("burgers", (0.5,)),
                diff=("pwl", (0.0, 0.0, 0.1, 0.5)), umin=-1.0, umax=1.0, limiter=True, rk=3, T=0.5,
                name="degenerate_burgers2d")


def config3(n: int = 4096) -> Spec:
    """2D porous medium u_t = Lap(u^2) on [-10, 10]^2 from Barenblatt t=1 to t=2."""
    return Spec(dim=2, nx=n, ny=n, x0=-10.0, x1=10.0, y0=-10.0, y1=10.0, flux=("zero", ()), diff=("pme", (2,)),
                umin=0.0, umax=1.0, limiter=True, rk=3, T=1.0, name="pme2d")


def config5(n: int = 4096) -> Spec:
    """2D Buckley-Leverett with gravity, kappa = 0.04 u (1-u), u0 = 1 in r < 0.5."""
    return Spec(dim=2, nx=n, ny=n, x0=-1.5, x1=1.5, y0=-1.5, y1=1.5, flux=("bl", (5.0,)),
                diff=("cubic", (0.0, 0.02, -0.04 / 3.0)), umin=0.0, umax=1.0, limiter=True, blend="plain",
                rk=3, T=0.5, name="buckley_leverett2d")


def initial_state(spec: Spec, device="cpu", sub: int = 4, order: int = 5):
    """Initial DoFs for the named workloads."""
    if spec.name == "linear1d":
        return sine_1d_state(spec, device=device)
    if spec.name == "pme3d":
        return state_3d(lambda x, y, z: barenblatt_3d(x, y, z, 1.0), spec, sub=sub, order=order)
    if spec.name == "evje_karlsen":
        return state_1d(evje_karlsen_fn, spec, device=device, sub=sub, order=order)
    if spec.name == "buckley_leverett1d_ibvp":
        return state_1d(bl1d_ibvp_fn, spec, device=device, sub=sub, order=order)
    if spec.name == "buckley_leverett1d_rp":
        return state_1d(bl1d_rp_fn, spec, device=device, sub=sub, order=order)
    if spec.name == "strongly_degenerate1d":
        return state_1d(strongly_degenerate_fn, spec, device=device, sub=sub, order=order)
    if spec.name == "degenerate_burgers2d":
        return state_2d(discs_fn, spec, device=device, sub=sub, order=order)
    if spec.name == "pme2d":
        return state_2d(lambda x, y: barenblatt(x, y, 1.0), spec, device=device, sub=sub, order=order)
    if spec.name == "two_hills":
        return state_2d(two_hills_fn, spec, device=device, sub=sub, order=order)
    if spec.name == "buckley_leverett2d":
        return state_2d(bl_disc_fn, spec, device=device, sub=sub, order=order)
    if spec.name == "buckley_leverett2d_outflow":
        return state_2d(lambda x, y: bl_disc_fn(x, y, math.sqrt(0.5)), spec, device=device, sub=sub, order=order)
    if spec.name == "strongly_degenerate2d":
        return state_2d(strongly_degenerate_2d_fn, spec, device=device, sub=sub, order=order)
    raise KeyError(spec.name)


def batch_instances(count: int = 256, seed: int = 20251011, nmin: int = 64, nmax: int = 1024):
    """Seeded batch of periodic 2D instances on [0,1]^2: Burgers f = u^2/2 and
    kappa = eps * 1[|u - 0.5| > 0.25] with eps ~ U[0.005, 0.05]; u0 a clipped 8-mode
    Fourier series. Returns a list of (Spec, (A, p, q, phi))."""
    rng = np.random.default_rng(seed)
    out = []
    modes = [(a, b) for a in range(-4, 5) for b in range(-4, 5) if (a, b) != (0, 0)]
    for k in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        eps = float(rng.uniform(0.005, 0.05))
        idx = rng.choice(len(modes), size=8, replace=False)
        p = [modes[t][0] for t in idx]
        q = [modes[t][1] for t in idx]
        A = rng.uniform(0.0, 0.25, size=8).tolist()
        phi = rng.uniform(0.0, 2 * math.pi, size=8).tolist()
        spec = Spec(dim=2, nx=n, ny=n, flux=("burgers", (0.5,)), diff=("pwl", (eps, 0.25, eps, 0.75)),
                    umin=0.0, umax=1.0, limiter=True, rk=3, name=f"batch{k}")
        out.append((spec, (A, p, q, phi)))
    return out


def batch_state(spec: Spec, modes, device="cpu", sub: int = 2, order: int = 3):
    A, p, q, phi = modes
    return state_2d(fourier8_fn(A, p, q, phi), spec, device=device, sub=sub, order=order)


def random_piecewise(spec: Spec, seed: int, nshapes: int = 6, device="cpu", sub: int = 2, order: int = 3):
    """Random piecewise-constant field on the mesh: a seeded union of rectangles and discs
    with values in [0, 1] painted over a random background (indicator-network data)."""
    rng = np.random.default_rng(seed)
    bg = float(rng.uniform(0, 1))
    shapes = []
    for _ in range(nshapes):
        kind = int(rng.integers(0, 2))
        cx = float(rng.uniform(spec.x0, spec.x1))
        cy = float(rng.uniform(spec.y0, spec.y1))
        sz = float(rng.uniform(0.05, 0.3)) * (spec.x1 - spec.x0)
        sz2 = float(rng.uniform(0.05, 0.3)) * (spec.y1 - spec.y0)
        val = float(rng.uniform(0, 1))
        shapes.append((kind, cx, cy, sz, sz2, val))

    def f(x, y):
        out = torch.full(torch.broadcast_shapes(x.shape, y.shape), bg, dtype=torch.float64, device=x.device)
        for kind, cx, cy, sz, sz2, val in shapes:
            if kind == 0:
                m = ((x - cx).abs() < sz / 2) & ((y - cy).abs() < sz2 / 2)
            else:
                m = ((x - cx) ** 2 + (y - cy) ** 2) < (sz / 2) ** 2
            out = torch.where(m, torch.full_like(out, val), out)
        return out

    return state_2d(f, spec, device=device, sub=sub, order=order)


def random_state_2d(spec: Spec, seed: int, lo: float | None = None, hi: float | None = None, device="cpu"):
    """Uniform random DoFs in [lo, hi] (defaults to the spec's bounds): a rough state
    that exercises every branch of the limiter."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    lo = spec.umin if lo is None else lo
    hi = spec.umax if hi is None else hi
    shapes = [(spec.ny, spec.nx)] * 4
    if spec.bc != "periodic":
        shapes = [(spec.ny, spec.nx), (spec.ny + 1, spec.nx + 1), (spec.ny, spec.nx + 1), (spec.ny + 1, spec.nx)]
    return [(lo + (hi - lo) * torch.rand(sh, generator=g, dtype=torch.float64)).to(device) for sh in shapes]


# 3D (periodic, [nz][ny][nx]): 8 arrays ordered by kind s = sx + 2 sy + 4 sz of the location
# (i + sx/2, j + sy/2, k + sz/2): ub, x-face, y-face, xy-edge, z-face, xz-edge, yz-edge,
# corner.
def kind_offsets_3d():
    return [((s >> 0) & 1, (s >> 1) & 1, (s >> 2) & 1) for s in range(8)]


def random_state_3d(spec: Spec, seed: int, lo: float | None = None, hi: float | None = None):
    g = torch.Generator(device="cpu").manual_seed(seed)
    lo = spec.umin if lo is None else lo
    hi = spec.umax if hi is None else hi
    shape = (spec.nz, spec.ny, spec.nx)
    return [lo + (hi - lo) * torch.rand(shape, generator=g, dtype=torch.float64) for _ in range(8)]


def mode_3d_state(spec: Spec, k: float, shift: float = 1.0, amp: float = 1.0):
    """u0 = shift + amp sin(k (x + y + z)): closed-form cell averages (the product of the
    three 1D averaging factors) and exact point values at every kind's location."""
    i = torch.arange(spec.nx, dtype=torch.float64)
    j = torch.arange(spec.ny, dtype=torch.float64)
    kk = torch.arange(spec.nz, dtype=torch.float64)
    fac = 1.0
    for h in (spec.dx, spec.dy, spec.dz):
        fac *= math.sin(k * h / 2) / (k * h / 2)
    out = []
    for s, (sx, sy, sz) in enumerate(kind_offsets_3d()):
        x = spec.x0 + (i + 0.5 + 0.5 * sx) * spec.dx
        y = spec.y0 + (j + 0.5 + 0.5 * sy) * spec.dy
        z = spec.z0 + (kk + 0.5 + 0.5 * sz) * spec.dz
        ph = k * (x[None, None, :] + y[None, :, None] + z[:, None, None])
        out.append(shift + amp * (fac if s == 0 else 1.0) * torch.sin(ph))
    return out


def state_3d(func: Callable, spec: Spec, sub: int = 2, order: int = 3) -> List[torch.Tensor]:
    """Cell averages of func(x, y, z) by a tensor Gauss-Legendre rule on sub^3 sub-cells and
    exact point values at every kind's location (8 arrays by kind, [nz][ny][nx])."""
    gx, gw = _gauss(order)
    offs, wts = [], []
    for s_ in range(sub):
        for q in range(order):
            offs.append((s_ + 0.5 + 0.5 * gx[q]) / sub)
            wts.append(gw[q] / (2 * sub))
    i = torch.arange(spec.nx, dtype=torch.float64)
    j = torch.arange(spec.ny, dtype=torch.float64)
    k = torch.arange(spec.nz, dtype=torch.float64)
    ub = torch.zeros((spec.nz, spec.ny, spec.nx), dtype=torch.float64)
    for oz, wz in zip(offs, wts):
        z = spec.z0 + (k + oz) * spec.dz
        for oy, wy in zip(offs, wts):
            y = spec.y0 + (j + oy) * spec.dy
            for ox, wx in zip(offs, wts):
                x = spec.x0 + (i + ox) * spec.dx
                ub += wx * wy * wz * func(x[None, None, :], y[None, :, None], z[:, None, None])
    out = [ub]
    for s_, (sx, sy, sz) in enumerate(kind_offsets_3d()):
        if s_ == 0:
            continue
        x = spec.x0 + (i + 0.5 + 0.5 * sx) * spec.dx
        y = spec.y0 + (j + 0.5 + 0.5 * sy) * spec.dy
        z = spec.z0 + (k + 0.5 + 0.5 * sz) * spec.dz
        out.append(func(x[None, None, :], y[None, :, None], z[:, None, None]).expand(spec.nz, spec.ny, spec.nx).clone())
    return out


def barenblatt_3d(x, y, z, t: float, m: int = 2):
    """Barenblatt solution of u_t = Lap(u^m) in 3D (Example 6.3 with d = 3); for m = 2,
    t^(-3/5) max(0, 1 - |x|^2 t^(-2/5) / 20)."""
    alpha = 1.0 / (m - 1 + 2.0 / 3.0)
    r2 = x * x + y * y + z * z
    core = 1.0 - alpha * (m - 1) / (6.0 * m) * r2 / (t ** (2 * alpha / 3))
    return t ** (-alpha) * torch.clamp(core, min=0.0) ** (1.0 / (m - 1))


def pme_3d(n: int = 32) -> Spec:
    """Porous medium a = u^2 in 3D on [-6, 6]^3 (periodic; the Barenblatt support stays
    inside), from the Barenblatt profile at t = 1."""
    return Spec(dim=3, nx=n, ny=n, nz=n, x0=-6.0, x1=6.0, y0=-6.0, y1=6.0, z0=-6.0, z1=6.0, flux=("zero", ()),
                diff=("pme", (2,)), umin=0.0, umax=1.0, limiter=True, rk=3, name="pme3d")


def random_state_1d(spec: Spec, seed: int, lo: float | None = None, hi: float | None = None):
    g = torch.Generator(device="cpu").manual_seed(seed)
    lo = spec.umin if lo is None else lo
    hi = spec.umax if hi is None else hi
    npts = spec.nx + (1 if spec.bc != "periodic" else 0)
    out = [lo + (hi - lo) * torch.rand((n,), generator=g, dtype=torch.float64) for n in (spec.nx, npts)]
    if spec.bc == "dirichlet":
        out[1][0], out[1][-1] = spec.bc_values
    return out


# ----------------------------------------------------------------------------------
# learned indicator: seeded initial parameters (flat FP32, layout W1[32][21], b1[32],
# W2[32][32], b2[32], w3[32], b3) -- He-normal hidden layers, output bias -2

MLP_NIN, MLP_NH = 21, 32


def mlp_init_params(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, math.sqrt(2.0 / MLP_NIN), MLP_NH * MLP_NIN), np.zeros(MLP_NH),
             rng.normal(0, math.sqrt(2.0 / MLP_NH), MLP_NH * MLP_NH), np.zeros(MLP_NH),
             rng.normal(0, math.sqrt(1.0 / MLP_NH), MLP_NH), np.array([-2.0])]
    return np.concatenate(parts).astype(np.float32)
