"""GB300 (sm_103a) implementation of the compact fourth-order doubly conservative
active flux method with monolithic convex MPP limiting (arXiv 2510.11527).

The numerical work runs in libaf.so (CUDA, include/af.h); ``capi`` is its ctypes
binding and ``Solver`` a small convenience wrapper that owns one af_ctx. PyTorch is
used only for device memory views and streams.
"""
import ctypes

import numpy as np

from . import capi
from .capi import AfError, af_bounds_t, af_diff, af_flux, af_grid, af_opts

__all__ = ["Solver", "capi", "AfError"]


class Solver:
    """One mesh behind an af_ctx.

    spec: any object with the attributes dim, nx, ny, x0, x1, y0, y1, flux=(kind, params),
    diff=(kind, params), umin, umax, limiter, blend, gamma and optionally bc ("periodic",
    "dirichlet", "outflow"), bc_values and diffusion_form ("dc", "nodc") (e.g.
    af_inputs.Spec). A 1D interval with Dirichlet or outflow ends has nx + 1 point values;
    a 2D rectangle with outflow ends has V [ny+1][nx+1], X [ny][nx+1], Y [ny+1][nx].
    """

    def __init__(self, spec, precision="fp64", rk=3, cfl=0.0, cfl_diff=0.0, bounds_from_data=False):
        self.spec = spec
        self.dim = spec.dim
        self.n = spec.nx * (spec.ny if spec.dim >= 2 else 1) * (spec.nz if spec.dim == 3 else 1)
        bc = getattr(spec, "bc", "periodic")
        gl, gr = getattr(spec, "bc_values", (0.0, 0.0))
        self.npts = self.n + (1 if spec.dim == 1 and bc != "periodic" else 0)
        nx, ny = spec.nx, (spec.ny if spec.dim >= 2 else 1)
        self.rect = spec.dim == 2 and bc != "periodic"
        self.shapes = ([(ny, nx), (ny + 1, nx + 1), (ny, nx + 1), (ny + 1, nx)] if self.rect
                       else [(ny, nx)] * 4 if spec.dim == 2 else [(nx,), (self.npts,)])
        if spec.dim == 3:
            self.shapes = [(spec.nz, ny, nx)] * 8
        g = af_grid(spec.dim, spec.nx, spec.ny if spec.dim >= 2 else 1, spec.x0, spec.x1, spec.y0, spec.y1,
                    capi.BC[bc], float(gl), float(gr), spec.nz if spec.dim == 3 else 1,
                    getattr(spec, "z0", 0.0), getattr(spec, "z1", 1.0))
        f = af_flux()
        f.kind = capi.FLUX[spec.flux[0]]
        for k, v in enumerate(spec.flux[1]):
            f.p[k] = float(v)
        d = af_diff()
        d.kind = capi.DIFF[spec.diff[0]]
        for k, v in enumerate(spec.diff[1]):
            d.p[k] = float(v)
        b = af_bounds_t(float(spec.umin), float(spec.umax), 1 if bounds_from_data else 0)
        o = af_opts(capi.PREC[precision], int(rk), float(cfl), float(cfl_diff), int(bool(spec.limiter)),
                    capi.BLEND[spec.blend], float(spec.gamma), capi.FORM[getattr(spec, "diffusion_form", "dc")])
        self.precision = precision
        self.ctx = capi.af_create(g, f, d, b, o)

    def close(self):
        if self.ctx:
            capi.af_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # state I/O
    def set_state(self, state):
        arrs = [np.asarray(a, dtype=np.float64) for a in state]
        if self.dim == 3:
            capi.af_set_state_arrays(self.ctx, arrs, [int(np.prod(s)) for s in self.shapes])
            return
        if self.dim == 1:
            capi.af_set_state(self.ctx, self.n, arrs[0], arrs[1], npts=self.npts)
        else:
            capi.af_set_state(self.ctx, self.n, *arrs, sizes=[int(np.prod(s)) for s in self.shapes])

    def get_state(self, out=None):
        """Host copy of (ub, V, X, Y); `out` may supply the destination float64 arrays
        (for instance views of pinned host memory, which copy fastest)."""
        if self.dim == 3:
            flat = None if out is None else [np.asarray(a).reshape(-1) for a in out]
            res = capi.af_get_state_arrays(self.ctx, [int(np.prod(s)) for s in self.shapes], flat)
            return [a.reshape(sh) for a, sh in zip(res, self.shapes)]
        if self.dim == 1:
            flat = None if out is None else [np.asarray(a).reshape(-1) for a in out]
            return capi.af_get_state(self.ctx, self.n, 1, flat, npts=self.npts)
        flat = None if out is None else [np.asarray(a).reshape(-1) for a in out]
        res = capi.af_get_state(self.ctx, self.n, self.dim, flat, sizes=[int(np.prod(s)) for s in self.shapes])
        return [a.reshape(sh) for a, sh in zip(res, self.shapes)]

    def device_tensors(self):
        """Zero-copy torch views of the current device state (ub, V, X, Y); a 2D rectangle
        with ends gives its padded device layout, [ny+1][nx+1] per array (entry (I, J):
        average of cell (I-1, J-1), corner / edge values at its top-right)."""
        import torch

        if self.dim == 3:
            ptrs, (d0, d1) = capi.af_device_ptrs_arrays(self.ctx, 8)
        else:
            ptrs, (d0, d1) = capi.af_device_ptrs(self.ctx)
        shape = (self.spec.ny, self.spec.nx) if self.dim == 2 else (self.spec.nx,)
        if self.rect:
            shape = (self.spec.ny + 1, self.spec.nx + 1)
        if self.dim == 3:
            shape = (self.spec.nz, self.spec.ny, self.spec.nx)
        out = []
        for k, p in enumerate(ptrs):
            if p is None:
                continue
            typestr = "<f8" if (k == 0 or d1 == 8) else "<f4"
            shp = (self.npts,) if (self.dim == 1 and k > 0) else shape

            class _View:
                __cuda_array_interface__ = {"shape": shp, "typestr": typestr, "data": (p, False), "version": 3}

            out.append(torch.as_tensor(_View(), device="cuda"))
        return out

    def set_stream(self, stream):
        capi.af_set_stream(self.ctx, stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)

    # stepping
    def forward_euler(self, tau):
        capi.af_forward_euler(self.ctx, tau)

    def stage(self, k, dt):
        capi.af_stage(self.ctx, k, dt)

    def dt_device(self):
        capi.af_dt_device(self.ctx)

    def step(self, dt=0.0, want_dt=False):
        return capi.af_step(self.ctx, dt, want_dt)

    def run(self, T):
        return capi.af_run(self.ctx, T)

    def time(self):
        return capi.af_time(self.ctx)

    def set_indicator(self, s):
        capi.af_set_indicator(self.ctx, self.n, s)

    # diagnostics
    def mass(self):
        return capi.af_mass(self.ctx)

    def bounds(self):
        return capi.af_bounds(self.ctx)

    def dt_cfl(self):
        return capi.af_dt_cfl(self.ctx)

    def stats(self):
        return capi.af_stats(self.ctx)

    @property
    def num_stages(self):
        return capi.af_num_stages(self.ctx)
