"""The C ABI without a GPU: the library loads, exports every declared symbol,
its structs match the header, and argument errors return before any launch."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1408_0677_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mls.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.load()


def declared_functions():
    names = set()
    for hdr in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)
        names |= set(re.findall(r"\b(mls_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "mls_create" in names and "mls_render" in names and "mls_bands" in names and "mls_destroy" in names
    assert "mls_debug_wait_selftest" in names and "mls_debug_df_weight" in names
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mls_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in names:
        assert hasattr(lib, n)


def test_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "mls.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(mls_desc), offsetof(mls_desc, h),
         offsetof(mls_desc, cond_recompute), offsetof(mls_desc, variant), offsetof(mls_desc, support),
         sizeof(mls_view), sizeof(mls_stats), sizeof(mls_map_desc), offsetof(mls_map_desc, lo),
         offsetof(mls_map_desc, texture));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(x) for x in subprocess.check_output([exe]).split()]
    assert vals == [ctypes.sizeof(_abi.MlsDesc), _abi.MlsDesc.h.offset, _abi.MlsDesc.cond_recompute.offset,
                    _abi.MlsDesc.variant.offset, _abi.MlsDesc.support.offset,
                    ctypes.sizeof(_abi.MlsView), ctypes.sizeof(_abi.MlsStats), ctypes.sizeof(_abi.MlsMapDesc),
                    _abi.MlsMapDesc.lo.offset, _abi.MlsMapDesc.texture.offset]


def test_abi_version_and_defaults(lib):
    assert _abi.mls_abi_version() == 5
    d = _abi.mls_desc_default()
    assert d.cond_fp64 == 1e6 and d.rcond_degenerate == 1e-12 and d.precision == _abi.MLS_P_FP32
    assert d.variant == _abi.MLS_V_POLY and d.support == 0.0


def _desc(**kw):
    d = _abi.mls_desc_default()
    d.n, d.D, d.degree, d.h = 10, 2, 1, 0.1
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("kw,code", [
    (dict(n=0), _abi.MLS_E_INVAL),
    (dict(D=0), _abi.MLS_E_INVAL),
    (dict(D=257), _abi.MLS_E_INVAL),
    (dict(degree=3), _abi.MLS_E_INVAL),
    (dict(h=0.0), _abi.MLS_E_INVAL),
    (dict(h=float("nan")), _abi.MLS_E_INVAL),
    (dict(weight=7), _abi.MLS_E_INVAL),
    (dict(precision=9), _abi.MLS_E_INVAL),
    (dict(weight=_abi.MLS_W_INVDIST, alpha=-1.0), _abi.MLS_E_INVAL),
    (dict(rcond_degenerate=2.0), _abi.MLS_E_INVAL),
    (dict(weight_split=3), _abi.MLS_E_INVAL),
    (dict(support=-1.0), _abi.MLS_E_INVAL),
    (dict(support=float("nan")), _abi.MLS_E_INVAL),
    (dict(support=2e6), _abi.MLS_E_INVAL),
    (dict(support=3.0, weight=_abi.MLS_W_WENDLAND), _abi.MLS_E_INVAL),
    (dict(support=3.0, weight=_abi.MLS_W_INVDIST), _abi.MLS_E_INVAL),
    (dict(variant=3), _abi.MLS_E_INVAL),
    (dict(variant=_abi.MLS_V_RIGID, D=3), _abi.MLS_E_INVAL),
])
def test_create_rejects_bad_descriptors_before_any_launch(lib, kw, code):
    buf = (ctypes.c_double * 64)()
    with pytest.raises(_abi.MlsError) as e:
        _abi.mls_create(_desc(**kw), ctypes.addressof(buf), ctypes.addressof(buf), False)
    assert e.value.status == code
    assert _abi.mls_last_error() != ""


def test_null_arguments(lib):
    assert lib.mls_create(None, None, None, 0, None, None) == _abi.MLS_E_INVAL
    h = ctypes.c_void_p()
    d = _desc()
    assert lib.mls_create(ctypes.byref(d), None, None, 0, None, ctypes.byref(h)) == _abi.MLS_E_INVAL
    v = _abi.MlsView(4, 4, 0, 0, 1, 1)
    assert lib.mls_render(None, ctypes.byref(v), None, None, None, 0, None, 1, None) == _abi.MLS_E_INVAL
    assert lib.mls_bands(None, ctypes.byref(v), None, None, 0, None, 1, None) == _abi.MLS_E_INVAL
    assert lib.mls_sync(None, 1.0, None) == _abi.MLS_E_INVAL
    assert lib.mls_destroy(None) == _abi.MLS_OK
    assert lib.mls_batch_create(0, None, 0, ctypes.byref(h)) == _abi.MLS_E_INVAL
    assert lib.mls_batch_create(1, None, 0, None) == _abi.MLS_E_INVAL
    assert lib.mls_batch_render(None, None, None, None, None, None, None, None) == _abi.MLS_E_INVAL
    assert lib.mls_batch_sync(None, 1.0, None) == _abi.MLS_E_INVAL
    assert lib.mls_batch_destroy(None) == _abi.MLS_OK
    assert lib.mls_debug_df_weight(3, None, None, 1, None) == _abi.MLS_E_INVAL
    assert lib.mls_debug_df_weight(0, None, None, 4, None) == _abi.MLS_E_INVAL
    assert lib.mls_debug_df_weight(0, None, None, 0, None) == _abi.MLS_OK
    assert lib.mls_debug_handover_split(None, 0, 0) == _abi.MLS_E_INVAL
    assert lib.mls_debug_host_output(None, 1) == _abi.MLS_E_INVAL


def test_injected_allocation_failure_returns_nomem(lib, monkeypatch):
    """Host-side fault injection: the allocation fails before any CUDA call."""
    monkeypatch.setenv("MLS_INJECT_NOMEM", "1")
    buf = (ctypes.c_double * 64)()
    with pytest.raises(_abi.MlsError) as e:
        _abi.mls_create(_desc(), ctypes.addressof(buf), ctypes.addressof(buf), False)
    assert e.value.status == _abi.MLS_E_NOMEM


def _map_desc(**kw):
    d = _abi.MlsMapDesc()
    d.mode, d.ndim, d.line_width = _abi.MLS_MAP_LINES, 1, 1.0
    d.fade_lo, d.fade_hi, d.sublevels = 2.0, 6.0, 3
    d.lo[0], d.hi[0], d.lo[1], d.hi[1] = 0.0, 1.0, 0.0, 1.0
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("kw,D,L,levels", [
    (dict(mode=6), 1, 2, [0.0, 1.0]),
    (dict(ndim=3), 1, 2, [0.0, 1.0]),
    (dict(ndim=2), 1, 2, [0.0, 1.0]),                 # dim[1] = 1 is out of range for D = 1
    (dict(line_width=-1.0), 1, 2, [0.0, 1.0]),
    (dict(mode=_abi.MLS_MAP_ADAPTIVE, fade_lo=6.0, fade_hi=2.0), 1, 2, [0.0, 1.0]),
    (dict(mode=_abi.MLS_MAP_ADAPTIVE, sublevels=17), 1, 2, [0.0, 1.0]),
    (dict(mode=_abi.MLS_MAP_TEXTURE), 1, 2, [0.0, 1.0]),          # no texture
    (dict(mode=_abi.MLS_MAP_GRADIENT), 1, 2, [0.0, 1.0]),         # lo == hi set below
    (dict(), 1, 2, [1.0, 0.0]),                                   # levels descend
    (dict(), 1, 255, None),                                       # too many levels
])
def test_space_map_rejects_bad_arguments_before_any_launch(lib, kw, D, L, levels):
    d = _map_desc(**kw)
    if kw.get("mode") == _abi.MLS_MAP_GRADIENT:
        d.hi[0] = d.lo[0]
    if kw.get("ndim") == 2:
        d.dim[1] = 1                                   # out of range for D = 1
    lev = np.asarray(levels if levels is not None else np.arange(L), dtype=np.float64)
    buf = (ctypes.c_double * 64)()
    with pytest.raises(_abi.MlsError) as e:
        _abi.mls_space_map(d, D, 4, 4, ctypes.addressof(buf), False, lev.ctypes.data, L, ctypes.addressof(buf))
    assert e.value.status == _abi.MLS_E_INVAL


def test_host_outputs_are_checked_before_the_call():
    """render_host refuses caller-supplied outputs of the wrong shape, type or
    layout before anything reaches the library (page-locked outputs are
    written by the kernels, which cannot check them)."""
    import numpy as np

    from paper_1408_0677_gb300 import _check_host_out
    _check_host_out("field", None, (2, 3, 4), np.float32)
    _check_host_out("field", np.zeros((2, 3, 4), np.float32), (2, 3, 4), np.float32)
    bad = [np.zeros((2, 3, 5), np.float32), np.zeros((2, 3, 4), np.float64), np.zeros((2, 4, 3), np.float32).T,
           np.zeros((2, 3, 8), np.float32)[:, :, ::2], [[0.0]]]
    for a in bad:
        with pytest.raises(ValueError):
            _check_host_out("field", a, (2, 3, 4), np.float32)
    ro = np.zeros((3, 4), np.uint8)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        _check_host_out("status_out", ro, (3, 4), np.uint8)
