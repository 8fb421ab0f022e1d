"""mls_bands_noalloc, the iso-band entry point that allocates no device
memory, against mls_bands on the same fields: equal labels on two calls in
a row (the second with fewer levels, so the first call's levels are still
in the shared static array), NaN pixels included, and oversize requests
rejected before any device work."""
import ctypes

import numpy as np
import pytest

from paper_1408_0677_gb300 import _abi, inputs

pytestmark = pytest.mark.gpu

G = inputs.WEIGHT_GAUSS


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return _abi.load()


def _field_and_reference(wl, precision, levels):
    """A rendered field (with one NaN pixel per dimension) and mls_bands' labels of it."""
    import torch

    from paper_1408_0677_gb300 import Renderer
    r = Renderer(torch.from_numpy(wl.xy).cuda(), torch.from_numpy(wl.F).cuda(), degree=wl.degree,
                 weight=wl.weight, h=wl.h, precision=precision)
    field = r.render(wl.W, wl.H)["field"].clone()
    field[:, 0, 0] = float("nan")
    ref = r.bands(field, levels, wl.W, wl.H)
    r.sync()
    r.close()
    return field, ref


def _noalloc(field, levels):
    import torch
    D, H, W = field.shape
    lev = np.ascontiguousarray(levels, dtype=np.float64)
    out = torch.full((D, H, W), 77, dtype=torch.uint8, device=field.device)
    _abi.mls_bands_noalloc(D, W, H, field.data_ptr(), field.dtype == torch.float64, lev.ctypes.data, lev.shape[1],
                           out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_bands_equal_mls_bands_on_two_calls(lib, precision):
    import torch
    wl1 = inputs.small_random(41, 150, 6, 67, 41, 2, G, 0.1, L=12)    # 72 levels
    wl2 = inputs.small_random(42, 90, 3, 50, 29, 1, G, 0.12, L=5)     # 15 levels
    f1, ref1 = _field_and_reference(wl1, precision, wl1.levels)
    f2, ref2 = _field_and_reference(wl2, precision, wl2.levels)
    out1 = _noalloc(f1, wl1.levels)
    out2 = _noalloc(f2, wl2.levels)
    assert torch.equal(out1, ref1)
    assert torch.equal(out2, ref2)
    assert (out1[:, 0, 0] == 255).all() and (out2[:, 0, 0] == 255).all()
    # labels actually vary over the raster
    assert len(torch.unique(out1)) > 3


def test_noalloc_rejects_oversize_and_null_arguments(lib):
    lev = np.zeros((64, 65))
    st = lib.mls_bands_noalloc(64, 8, 8, ctypes.c_void_p(16), 0, lev.ctypes.data_as(ctypes.c_void_p), 65,
                               ctypes.c_void_p(16), None)
    assert st == _abi.MLS_E_INVAL
    assert b"exceeds" in _abi.load().mls_last_error()
    st = lib.mls_bands_noalloc(2, 8, 8, None, 0, lev.ctypes.data_as(ctypes.c_void_p), 4, ctypes.c_void_p(16), None)
    assert st == _abi.MLS_E_INVAL
