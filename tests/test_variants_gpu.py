"""GPU parity of the paper's rigid (Section 3.3.3) and mean-displacement
(Section 3.3.1) mappings against the oracle's literal equations: points p_i
are distorted positions and the 2-D values q_i their original positions (the
paper's use), for every weight and precision."""
import numpy as np
import pytest

import oracle
from paper_1408_0677_gb300 import inputs

pytestmark = pytest.mark.gpu

VARIANTS = {"rigid": 1, "mean": 2}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _case(seed, n, weight, h):
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.05, 0.95, (n, 2))                  # original positions
    th = 0.3 * np.sin(3 * q[:, 0]) * np.cos(2 * q[:, 1])
    p = np.stack([q[:, 0] + 0.06 * np.sin(2 * np.pi * q[:, 1]) + 0.02 * np.cos(th),
                  q[:, 1] + 0.05 * np.cos(2 * np.pi * q[:, 0])], axis=1)   # distorted positions
    return p, q, weight, h


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("weight,h", [(0, 0.06), (1, 0.12), (2, 0.05)], ids=["gauss", "wendland", "idw"])
def test_variant_matches_oracle(variant, precision, weight, h):
    """Element by element within tol (1e-10 of the value range in FP64, 1e-3
    in FP32; FP16 renders take the FP32 kernel) plus, for the rigid form,
    c * kappa * |v - p*|: a relative error e in the moments turns the result
    by about e * kappa radians (kappa the oracle's conditioning of the
    rotation), c = 1e-12 / 1e-4 leaves a wide margin over FP64 / FP32
    rounding.  Everywhere |f - q*| = |v - p*| (a rotation keeps lengths)."""
    import torch

    from paper_1408_0677_gb300 import Renderer
    p, q, weight, h = _case(81 + weight, 1500, weight, h)
    W, H = 70, 53
    r = Renderer(torch.from_numpy(p).cuda(), torch.from_numpy(q).cuda(), degree=1, weight=weight, h=h,
                 precision=precision, variant=VARIANTS[variant])
    lev = inputs.default_levels(q, 12)
    out = r.render(W, H, levels=lev)
    r.sync()
    r.close()
    f = out["field"].double().cpu().numpy().reshape(2, -1).T
    ref, aux = oracle.mls_variant(p, q, VARIANTS[variant], weight, h, W, H, aux=True)
    scale = np.ptp(q, axis=0).max()
    nan_ref = np.isnan(ref)
    assert np.array_equal(nan_ref, np.isnan(f))
    ok = ~nan_ref[:, 0]
    tol, c = (1e-10, 1e-12) if precision == "fp64" else (1e-3, 1e-4)
    kappa = np.where(np.isfinite(aux[:, 3]), aux[:, 3], 0.0)
    bound = tol * scale + c * kappa * aux[:, 2]
    err = np.abs(f - ref).max(axis=1)
    assert np.all(err[ok] <= bound[ok]), (err[ok].max(), int(np.argmax(np.where(ok, err - bound, -np.inf))))
    rad = np.hypot(*(f - aux[:, :2]).T)
    assert np.all(np.abs(rad - aux[:, 2])[ok] <= tol * scale)
    # bands: exact away from the levels
    b = out["bands"].cpu().numpy().reshape(2, -1).T
    bo = oracle.bands(ref, lev)
    near = np.zeros_like(nan_ref)
    for j in range(lev.shape[1]):
        near |= np.abs(ref - lev[:, j][None, :]) <= bound[:, None]
    assert np.array_equal(b[~near], bo[~near])


def test_variant_needs_two_dimensions():
    import torch

    from paper_1408_0677_gb300 import MlsError, Renderer
    with pytest.raises(MlsError):
        Renderer(torch.zeros(10, 2, dtype=torch.float64).cuda(), torch.zeros(10, 3, dtype=torch.float64).cuda(),
                 variant=1)
