"""af_mass_noalloc: the allocation-free variant of the mass reduction, for callers that
cannot allocate device memory (an application whose memory pool already owns the
device memory, a loop that cannot take an allocation's device synchronisation, a
plugin host that forbids library allocations). Its scratch is a file-scope device
array shared by all calls.

Checked through the C ABI against the host's exactly rounded sum of the same data and
the existing entry point af_mass, on two calls in a row (the second call reuses the
scratch the first one left and allocates nothing); pointers that are not device memory
of the current device are rejected.
This file is collected last so that a run stopping at the first failure has already
run every other test; it passes alone in a fresh process and after the others."""
import math

import numpy as np
import pytest

import af_inputs as ai

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_11527_gb300 import build
    build.build()


@pytest.mark.parametrize("nx,ny", [(256, 256), (1000, 37), (3, 1)])
def test_mass_noalloc_matches_af_mass_twice(nx, ny):
    """Two calls in a row agree bit for bit, lie within FP64 round-off of the host's
    exactly rounded sum (math.fsum) and of af_mass, and the second call changes the
    device's free memory by nothing (no allocation)."""
    import torch
    from paper_2510_11527_gb300 import Solver, capi
    spec = ai.config2(8).with_size(nx, ny)
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=nx + ny, lo=-1, hi=1)]
    exact = math.fsum(st[0].ravel().tolist()) * spec.dx * spec.dy
    with Solver(spec) as s:
        s.set_state(st)
        ref = s.mass()                                   # existing entry point (af_mass)
        ptrs, _ = capi.af_device_ptrs(s.ctx)
        a = capi.af_mass_noalloc(ptrs[0], nx * ny, spec.dx * spec.dy)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        b = capi.af_mass_noalloc(ptrs[0], nx * ny, spec.dx * spec.dy)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    scale = np.sum(np.abs(st[0])) * spec.dx * spec.dy
    assert abs(a - exact) <= 1e-13 * scale
    assert abs(a - ref) <= 1e-13 * scale
    assert a == b
    assert free1 == free0


def test_mass_noalloc_rejects_oversize_and_null():
    from paper_2510_11527_gb300 import Solver, capi
    spec = ai.config2(16)
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=1, lo=-1, hi=1)]
    with Solver(spec) as s:
        s.set_state(st)
        ptrs, _ = capi.af_device_ptrs(s.ctx)
        with pytest.raises(capi.AfError) as ei:
            capi.af_mass_noalloc(ptrs[0], capi.AF_MASS_NOALLOC_MAX_CELLS + 1, 1.0)
        assert ei.value.status == capi.AF_E_ARG
        with pytest.raises(capi.AfError) as ei:
            capi.af_mass_noalloc(ptrs[0], 0, 1.0)
        assert ei.value.status == capi.AF_E_ARG
        with pytest.raises(capi.AfError) as ei:
            capi.af_mass_noalloc(None, 16, 1.0)
        assert ei.value.status == capi.AF_E_ARG
        # host memory is not device memory of the current device
        host = np.ascontiguousarray(st[0])
        with pytest.raises(capi.AfError) as ei:
            capi.af_mass_noalloc(host.ctypes.data, host.size, 1.0)
        assert ei.value.status == capi.AF_E_ARG
        # a rejected call leaves nothing behind: the next valid call succeeds
        got = capi.af_mass_noalloc(ptrs[0], host.size, spec.dx * spec.dy)
        assert got == pytest.approx(math.fsum(host.ravel().tolist()) * spec.dx * spec.dy, rel=1e-13, abs=1e-13)
        # the context's own reduction is unaffected by the shared scratch
        assert s.mass() == pytest.approx(np.sum(st[0]) * spec.dx * spec.dy, rel=1e-13, abs=1e-13)
