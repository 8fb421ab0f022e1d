"""The checked build (MLS_CHECKED) on the GPU: every path, no index out of range.

build(checked=True) compiles the same kernels with every bin, tile, cell and
list index tested against its array's extent; a bad index is recorded in the
device error word (no trap), which mls_sync turns into an error.  A child
process loads that library (MLS_LIBRARY) and renders small cases through
every path: the tensor-core kernel in FP16 (two passes, split weights) and
BF16, the FP32 kernel in tile and pixel frames, the FP64 kernel, the
double-float hand-over and its FP64 tier, the FP64 emulation on the tensor
cores, Gaussian / Wendland / inverse distance / truncated Gaussian, the
rigid and mean mappings, host-pointer renders, standalone bands and the
batch.  Each render must leave the error
word at zero and match the oracle.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import dataclasses
import numpy as np
import torch
import oracle
from paper_1408_0677_gb300 import Batch, Renderer, _abi, inputs
from tests.gpu_util import compare, gpu_render, oracle_ref
assert _abi.load()._name.endswith("libmls_checked.so")
G, WD, ID = inputs.WEIGHT_GAUSS, inputs.WEIGHT_WENDLAND, inputs.WEIGHT_INVDIST
cases = [
    (inputs.fourier_mix(31, 10000, 8, 100, 75, 2, G, 0.02), ["fp16", "bf16", "fp32", "fp64"], {}),
    (inputs.fourier_mix(41, 3000, 8, 100, 75, 2, G, 0.03), ["fp16"], {"weight_split": 1}),
    (inputs.fourier_mix(34, 100000, 6, 90, 70, 2, WD, 0.02), ["fp16", "bf16", "fp32", "fp64"], {}),
    (inputs.fourier_mix(35, 100000, 48, 40, 36, 2, WD, 0.02), ["fp16"], {}),
    (dataclasses.replace(inputs.fourier_mix(51, 10000, 8, 100, 75, 2, G, 0.02), trunc=3.0), ["fp16", "fp32", "fp64"], {}),
    (inputs.fourier_mix(53, 3000, 4, 64, 48, 2, G, 0.008), ["fp16", "fp32"], {}),      # pixel frames
    (inputs.small_random(7, 50, 3, 29, 21, 1, ID, 0.2), ["fp32", "fp64"], {}),
    (inputs.small_random(4, 400, 4, 45, 38, 2, WD, 0.15), ["fp32", "fp64"], {}),
]
# the FP64 emulation on the tensor cores (zoom windows: 16 pixels span at most 4 h)
for seed, n, D, W, H, deg, wt, h, view in ((31, 10000, 8, 100, 75, 2, G, 0.02, (0.1, 0.2, 0.4, 0.425)),
                                           (34, 100000, 6, 90, 70, 2, WD, 0.02, (0.3, 0.2, 0.6, 0.45))):
    wl = inputs.fourier_mix(seed, n, D, W, H, deg, wt, h)
    wl.view = view
    ref = oracle_ref(wl)
    res = gpu_render(wl, "fp64tc")
    assert res["stats"].device_error == 0 and res["stats"].main_path == 5
    compare(wl, res, ref, "fp64tc", max_allow_frac=1.0)
    print("ok fp64tc", wl.name, flush=True)
for wl, precs, kw in cases:
    wl.view = (0.05, 0.1, 0.9, 0.85)
    ref = oracle_ref(wl)
    for prec in precs:
        res = gpu_render(wl, prec, **kw)
        assert res["stats"].device_error == 0, (wl.name, prec, res["stats"].device_error)
        compare(wl, res, ref, prec, max_allow_frac=1.0)
    print("ok", wl.name, precs, flush=True)
# host-pointer render, standalone bands
wl = inputs.small_random(24, 120, 3, 33, 27, 1, G, 0.1)
r = Renderer(wl.xy, wl.F, degree=1, weight=G, h=0.1, precision="fp16")
host = r.render_host(wl.W, wl.H, levels=wl.levels)
r.close()
r = Renderer(torch.from_numpy(wl.xy).cuda(), torch.from_numpy(wl.F).cuda(), degree=1, weight=G, h=0.1, precision="fp32")
out = r.render(wl.W, wl.H, levels=wl.levels)
b2 = r.bands(out["field"], wl.levels, wl.W, wl.H)
assert r.sync().device_error == 0
assert torch.equal(out["bands"], b2)
r.close()
# rigid and mean mappings
rng = np.random.default_rng(62)
q = rng.uniform(0.05, 0.95, (1500, 2))
p = q + 0.04 * np.stack([np.sin(2 * np.pi * q[:, 1]), np.cos(2 * np.pi * q[:, 0])], axis=1)
for variant in (1, 2):
    for w, h in ((G, 0.03), (WD, 0.06)):
        r = Renderer(torch.from_numpy(p).cuda(), torch.from_numpy(q).cuda(), degree=1, weight=w, h=h,
                     precision="fp32", variant=variant)
        r.render(60, 45)
        assert r.sync().device_error == 0
        r.close()
# a batch of two datasets in one graph
wls = [inputs.fourier_mix(71, 4000, 5, 96, 80, 2, G, 0.03), inputs.fourier_mix(72, 30000, 4, 80, 64, 2, WD, 0.03)]
rs = [Renderer(torch.from_numpy(w.xy).cuda(), torch.from_numpy(w.F).cuda(), degree=w.degree, weight=w.weight, h=w.h,
               precision="fp16") for w in wls]
b = Batch(rs)
outs = b.render([(w.W, w.H, (0.0, 0.0, 1.0, 1.0), w.levels) for w in wls])
st = b.sync()
assert st.device_error == 0
b.close()
for r in rs:
    r.close()
print("checked build: every path clean", flush=True)
'''


def test_checked_build_renders_every_path_without_an_index_error():
    from paper_1408_0677_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, MLS_LIBRARY=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, timeout=1200, env=env, cwd=ROOT)
    out = r.stdout + r.stderr
    assert r.returncode == 0 and "every path clean" in r.stdout, out[-6000:]
    print(r.stdout)
