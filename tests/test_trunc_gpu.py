"""GPU parity of the truncated Gaussian (weight zero outside the box
|dx|, |dy| < c h around each pixel; support count = points in the box)
against the FP64 oracle, through every path: the tensor-core kernel in FP16
and BF16 (binned point tiles, box-masked separable weights), the FP32 and
FP64 CUDA-core kernels, the hand-over of count-ambiguous and ill-conditioned
pixels, and the rigid / mean mappings."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1408_0677_gb300 import inputs
from tests.gpu_util import compare, gpu_render, oracle_ref

pytestmark = pytest.mark.gpu

G = inputs.WEIGHT_GAUSS
ALL_PREC = ["fp64", "fp32", "fp16", "bf16"]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _ref(wl, pixels=None):
    return oracle_ref(wl, pixels)


@pytest.mark.parametrize("precision", ALL_PREC)
def test_fourier_10k_truncated_sampled(precision):
    """The 10k-point workload (1024 x 1024, D = 32, quadratic, h = 0.02) with
    a box of half-width 4 h: full render, sampled pixels."""
    wl = dataclasses.replace(inputs.fourier_10k(), trunc=4.0)
    pix = inputs.sample_pixels(12, wl.W, wl.H, 2048 if precision != "fp64" else 512)
    res = gpu_render(wl, precision)
    err, npx = compare(wl, res, _ref(wl, pix), precision, pixels=pix)
    print(f"fourier-10k trunc 4: {precision} max err {err:.3g} over {npx} pixels")


STRUCTURED = [
    # seed, n, D, W, H, degree, h, c: clusters + background (empty boxes far
    # from the clusters when c h is small), several tiles and a ragged tail
    (51, 10000, 8, 100, 75, 2, 0.02, 3.0),
    (52, 3000, 5, 61, 47, 1, 0.02, 2.0),
    (53, 2000, 3, 48, 33, 0, 0.02, 1.5),
    (54, 10000, 40, 50, 20, 2, 0.02, 6.0),
]


@pytest.mark.parametrize("case", STRUCTURED, ids=[f"t{c[0]}" for c in STRUCTURED])
@pytest.mark.parametrize("precision", ALL_PREC)
def test_truncated_structured_ragged(case, precision):
    seed, n, D, W, H, degree, h, c = case
    wl = dataclasses.replace(inputs.fourier_mix(seed, n, D, W, H, degree, G, h), trunc=c)
    ref = _ref(wl)
    res = gpu_render(wl, precision)
    compare(wl, res, ref, precision)
    st = res["status"].reshape(-1)
    nan = np.isnan(ref.field[:, 0])
    assert np.array_equal(nan[ref.amb == 0], (st & 0x04).astype(bool)[ref.amb == 0])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_truncated_small_sparse(precision):
    """Few points, rough fields, boxes of one to a few points: empty boxes,
    counts below k and the degree policy's lowering."""
    wl = dataclasses.replace(inputs.small_random(61, 80, 3, 41, 29, 2, G, 0.05), trunc=2.0)
    ref = _ref(wl)
    assert np.isnan(ref.field[:, 0]).any() and (ref.deg_used == 0).any() and (ref.deg_used == 1).any()
    compare(wl, gpu_render(wl, precision), ref, precision)


@pytest.mark.parametrize("variant", [1, 2], ids=["rigid", "mean"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_truncated_mappings(variant, precision):
    import torch

    from paper_1408_0677_gb300 import Renderer
    rng = np.random.default_rng(62)
    q = rng.uniform(0.05, 0.95, (1500, 2))
    p = q + 0.04 * np.stack([np.sin(2 * np.pi * q[:, 1]), np.cos(2 * np.pi * q[:, 0])], axis=1)
    r = Renderer(torch.from_numpy(p).cuda(), torch.from_numpy(q).cuda(), degree=1, weight=G, h=0.03,
                 precision=precision, variant=variant, support=3.0)
    out = r.render(60, 45)
    r.sync()
    r.close()
    f = out["field"].double().cpu().numpy().reshape(2, -1).T
    ref, aux = oracle.mls_variant(p, q, variant, G, 0.03, 60, 45, aux=True, trunc=3.0)
    assert np.array_equal(np.isnan(ref), np.isnan(f))
    ok = ~np.isnan(ref[:, 0])
    tol, c = (1e-10, 1e-12) if precision == "fp64" else (1e-3, 1e-4)
    kappa = np.where(np.isfinite(aux[:, 3]), aux[:, 3], 0.0)
    bound = tol + c * kappa * aux[:, 2]
    err = np.abs(f - ref).max(axis=1)
    assert np.all(err[ok] <= bound[ok]), err[ok].max()
