"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer (CPU).

compute-sanitizer is not available for the GPU runs, so the host halves are
checked here instead:

- the FP64 oracle (oracle/mls_oracle.c), compiled with
  -fsanitize=address,undefined -fno-sanitize-recover=all, runs every entry
  point over small cases (each weight and degree, the truncated Gaussian,
  the rounding-error bound, the rigid / mean mappings, the bands) in a child
  process with the sanitizer runtimes preloaded;
- the library's host code (the C ABI's validation of descriptors, views,
  levels and buffers), compiled the same way (build(sanitize=True)), runs
  the argument-error paths of every entry point, which return before any
  CUDA work and so need no GPU.

A sanitizer report aborts the child with a non-zero status.  The device
side has its own checked build (MLS_CHECKED, tests/test_checked_build_gpu.py).
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _runtimes():
    libs = []
    for name in ("libasan.so", "libubsan.so"):
        p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
        if not os.path.isabs(p) or not os.path.exists(p):
            pytest.skip(f"{name} not available")
        libs.append(os.path.realpath(p))
    return ":".join(libs)


def _run_child(code, extra_env=None, timeout=600):
    env = dict(os.environ)
    env["LD_PRELOAD"] = _runtimes()
    env["ASAN_OPTIONS"] = "detect_leaks=0:protect_shadow_gap=0:abort_on_error=0:halt_on_error=1"
    env["UBSAN_OPTIONS"] = "halt_on_error=1:print_stacktrace=1"
    env["PYTHONPATH"] = ROOT
    env["OMP_NUM_THREADS"] = "2"
    env.update(extra_env or {})
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=timeout, env=env,
                       cwd=ROOT)
    out = r.stdout + r.stderr
    assert r.returncode == 0 and "ERROR: AddressSanitizer" not in out and "runtime error:" not in out, out[-4000:]
    return r.stdout


ORACLE_CASES = r'''
import numpy as np
import oracle
from oracle import oracle as orc
lib = orc.load_library(LIB)
rng = np.random.default_rng(5)
xy = rng.random((40, 2)); F = rng.standard_normal((40, 3))
for weight, h in ((0, 0.15), (1, 0.3), (2, 0.2)):
    for deg in (0, 1, 2):
        r = oracle.mls(xy, F, deg, weight, h, 9, 7, lib=lib, ebound=True, view=(-0.2, 0.1, 1.1, 0.9))
        assert r.field.shape == (63, 3)
        oracle.mls(xy, F, deg, weight, h, 9, 7, lib=lib, pixels=np.array([0, 5, 62]))
oracle.mls(xy, F, 2, 0, 0.1, 9, 7, lib=lib, trunc=2.0, ebound=True)
oracle.mls(xy[:1], F[:1], 2, 1, 0.05, 5, 5, lib=lib, ebound=True)              # empty supports, NaN
xy2 = np.vstack([xy, [[0.5 / 9, 0.5 / 7]]]); F2 = np.vstack([F, [[1.0, 2.0, 3.0]]])
oracle.mls(xy2, F2, 1, 2, 0.2, 9, 7, lib=lib, ebound=True)                      # a point on a pixel centre
oracle.bands(np.array([[0.1, np.nan], [2.0, -1.0]]), np.array([[0.0, 1.0], [0.5, 0.6]]), lib=lib)
for v in (1, 2):
    for weight, h in ((0, 0.15), (1, 0.3), (2, 0.2)):
        oracle.mls_variant(xy, xy + 0.01 * F[:, :2], v, weight, h, 8, 6, lib=lib, aux=True)
try:
    oracle.mls(xy, F, 3, 0, 0.1, 4, 4, lib=lib)
except ValueError:
    pass
print("oracle ok")
'''


def test_oracle_under_address_and_undefined_behaviour_sanitizers():
    src = os.path.join(ROOT, "oracle", "mls_oracle.c")
    with tempfile.TemporaryDirectory() as d:
        lib = os.path.join(d, "libmls_oracle_asan.so")
        subprocess.check_call(["gcc", "-O1", "-g", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                               "-fno-omit-frame-pointer", "-o", lib, src, "-lm"])
        out = _run_child(f"LIB = {lib!r}\n" + ORACLE_CASES)
    assert "oracle ok" in out


ABI_CASES = r'''
import ctypes
import numpy as np
from paper_1408_0677_gb300 import _abi
lib = _abi.load(LIB)
P = ctypes.c_void_p
d = _abi.MlsDesc()
assert lib.mls_desc_default(ctypes.byref(d)) == 0
xy = np.zeros((4, 2)); F = np.zeros((4, 2))
out = P()
bad = []
for field, value in (("n", 0), ("D", 0), ("D", 100000), ("degree", 3), ("weight", 7), ("precision", 9),
                     ("h", 0.0), ("h", float("nan")), ("weight_split", 5), ("variant", 9), ("support", -1.0)):
    e = _abi.MlsDesc(); lib.mls_desc_default(ctypes.byref(e)); e.n = 4; e.D = 2
    setattr(e, field, value)
    bad.append(lib.mls_create(ctypes.byref(e), xy.ctypes.data, F.ctypes.data, 0, None, ctypes.byref(out)))
assert all(s != 0 for s in bad), bad
e = _abi.MlsDesc(); lib.mls_desc_default(ctypes.byref(e)); e.n = 4; e.D = 2
assert lib.mls_create(ctypes.byref(e), None, F.ctypes.data, 0, None, ctypes.byref(out)) != 0
assert lib.mls_create(None, xy.ctypes.data, F.ctypes.data, 0, None, ctypes.byref(out)) != 0
v = _abi.MlsView(8, 8, 0.0, 0.0, 1.0, 1.0)
assert lib.mls_render(None, ctypes.byref(v), None, None, None, 0, None, 1, None) != 0
assert lib.mls_bands(None, ctypes.byref(v), None, None, 0, None, 1, None) != 0
lev = np.array([[0.0, 1.0], [2.0, 1.0]])
assert lib.mls_bands_noalloc(2, 8, 8, None, 0, lev.ctypes.data, 2, None, None) != 0
assert lib.mls_bands_noalloc(2, 8, 8, P(16), 0, lev.ctypes.data, 2, P(16), None) != 0        # not ascending
big = np.zeros(5000); assert lib.mls_bands_noalloc(1, 8, 8, P(16), 0, big.ctypes.data, 300, P(16), None) != 0
assert lib.mls_destroy(None) == 0                       # destroying NULL is a no-op
assert lib.mls_sync(None, 1.0, None) != 0
assert len(lib.mls_last_error()) > 0
print("abi ok")
'''


@pytest.mark.slow
def test_library_host_code_under_address_and_undefined_behaviour_sanitizers():
    from paper_1408_0677_gb300 import build
    lib = build.build(sanitize=True)
    out = _run_child(f"LIB = {lib!r}\n" + ABI_CASES)
    assert "abi ok" in out
