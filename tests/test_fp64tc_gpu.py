"""FP64 emulation on the tensor cores (precision "fp64tc", MLS_P_FP64_TC)
against the FP64 oracle at the FP64 tolerance (1e-10 of the data range,
with the rounding-error allowance of ill-conditioned fits: tests/gpu_util).

The moments come from the FP16 tensor cores: weights and operands split
into ten exact FP16 digits, the digit products summed exactly in FP32 and
combined in FP64, then the FP64 policy and solve of the definition
(Section 3.3)."""
import numpy as np
import pytest

from paper_1408_0677_gb300 import inputs
from tests.gpu_util import compare, gpu_render, oracle_ref

pytestmark = pytest.mark.gpu

G, WD, ID = inputs.WEIGHT_GAUSS, inputs.WEIGHT_WENDLAND, inputs.WEIGHT_INVDIST


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


CASES = [
    # seed, n, D, W, H, degree, weight, h, view: several tiles and ragged tails,
    # every degree, both weights, D over several value passes (5 per pass
    # quadratic); zoom windows where 16 pixels would otherwise span more than 4 h
    (31, 10000, 8, 100, 75, 2, G, 0.02, (0.1, 0.2, 0.4, 0.425)),
    (32, 10000, 5, 61, 47, 1, G, 0.02, (0.2, 0.3, 0.4, 0.45)),
    (33, 10000, 3, 48, 33, 0, G, 0.02, (0.1, 0.1, 0.3, 0.25)),
    (34, 100000, 6, 90, 70, 2, WD, 0.02, (0.3, 0.2, 0.6, 0.45)),
    (36, 10000, 13, 50, 20, 1, G, 0.02, (0.0, 0.0, 0.2, 0.1)),
    (37, 60000, 11, 40, 36, 2, WD, 0.02, (0.45, 0.4, 0.6, 0.55)),
]


@pytest.mark.parametrize("case", CASES, ids=[f"c{c[0]}" for c in CASES])
def test_structured_cases(case):
    seed, n, D, W, H, degree, weight, h, view = case
    wl = inputs.fourier_mix(seed, n, D, W, H, degree, weight, h)
    wl.view = view
    res = gpu_render(wl, "fp64tc")
    assert res["stats"].main_path == 5          # the tensor-core kernel ran
    # the sparse Wendland window c37: 6% of its pixels have an allowance above
    # 1e-10 under the emulation's error model
    err, npx = compare(wl, res, oracle_ref(wl), "fp64tc", max_allow_frac=0.08 if seed == 37 else None)
    print(f"fp64tc {wl.name}: max err {err:.3g} of range over {npx} pixels")


def test_wide_tiles_take_the_fp64_kernel():
    """16 pixels spanning about 9 h: no shared moment frame suits the tile,
    and the render takes the FP64 kernel (each pixel in its own frame)."""
    wl = inputs.fourier_mix(34, 100000, 6, 90, 70, 2, WD, 0.02)
    res = gpu_render(wl, "fp64tc")
    assert res["stats"].main_path == 3
    compare(wl, res, oracle_ref(wl), "fp64tc")


def test_wine_shaped_full_grid():
    """Three clusters on 256 x 256 pixels over [0,1]^2 (h = 0.05, a tile spans
    1.25 h).  Far from the clusters the fit extrapolates from a few weights:
    the allowance of the emulation's error model exceeds 1e-10 of the range on
    about half the pixels there."""
    wl = inputs.wine_shaped()
    res = gpu_render(wl, "fp64tc")
    err, npx = compare(wl, res, oracle_ref(wl), "fp64tc", max_allow_frac=0.60)
    print(f"fp64tc wine-shaped: max err {err:.3g} of range over {npx} pixels")


def test_fourier_10k_sampled():
    """The 10k-point configuration (1024 x 1024, D = 32, quadratic, Gaussian
    h = 0.02): full render, 512 sampled pixels at the FP64 tolerance."""
    wl = inputs.fourier_10k()
    pix = inputs.sample_pixels(11, wl.W, wl.H, 512)
    res = gpu_render(wl, "fp64tc")
    err, npx = compare(wl, res, oracle_ref(wl, pix), "fp64tc", pixels=pix)
    print(f"fp64tc fourier-10k: max err {err:.3g} of range, main pass {res['stats'].main_kernel_ms:.2f} ms")


def test_unsupported_forms_are_refused():
    import torch

    from paper_1408_0677_gb300 import MlsError, Renderer
    wl = inputs.small_random(7, 50, 3, 29, 21, 1, ID, 0.2)
    with pytest.raises(MlsError) as e:
        Renderer(torch.from_numpy(wl.xy).cuda(), torch.from_numpy(wl.F).cuda(), degree=1, weight=ID, h=0.2,
                 precision="fp64tc")
    assert e.value.status == 5
    with pytest.raises(MlsError):
        Renderer(torch.from_numpy(wl.xy).cuda(), torch.from_numpy(wl.F).cuda(), degree=1, weight=G, h=0.2,
                 precision="fp64tc", support=3.0)
