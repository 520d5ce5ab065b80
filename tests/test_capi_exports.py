"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/af.h declares. No compute calls: this runs without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(af_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libaf():
    from paper_2510_11527_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libaf):
    names = _declared("af.h")
    assert "af_create" in names and "af_step" in names and "af_run" in names
    for n in names:
        assert hasattr(libaf, n), n


def test_binding_covers_header():
    from paper_2510_11527_gb300 import capi
    assert sorted(capi.exported_symbols()) == _declared("af.h")


def test_create_without_gpu_is_unsupported_or_ok(libaf):
    import torch
    from paper_2510_11527_gb300 import capi
    g = capi.af_grid(2, 8, 8, 0.0, 1.0, 0.0, 1.0)
    f = capi.af_flux()
    d = capi.af_diff()
    b = capi.af_bounds_t(0.0, 1.0, 0)
    o = capi.af_opts(0, 3, 0.0, 0.0, 1, 0, 1.0)
    if torch.cuda.is_available():
        pytest.skip("GPU present: covered by the gpu tests")
    with pytest.raises(capi.AfError) as ei:
        capi.af_create(g, f, d, b, o)
    assert ei.value.status == capi.AF_E_UNSUPPORTED


def test_invalid_arguments_rejected_before_device_use(libaf):
    from paper_2510_11527_gb300 import capi
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present: covered by the gpu tests")
    # without a device every create fails; the argument checks are exercised on the GPU
    assert capi.lib().af_num_stages(None) == 0
