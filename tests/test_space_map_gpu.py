"""GPU space mappings (Section 3.4, mls_space_map) against the oracle's
float32 statement of them, byte for byte on the same field: every mode, one
and two planes, FP32 and FP64 fields with NaN holes on a raster that is not
a multiple of the block, repeated and unevenly spaced levels; then the
mapping of a field the GPU rendered."""
import numpy as np
import pytest

from oracle import space_map as SM
from paper_1408_0677_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _field(seed, D=3, H=77, W=101):
    rng = np.random.default_rng(seed)
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    F = []
    for d in range(D):
        a, b, c = rng.uniform(0.02, 0.12, 3)
        F.append(np.sin(a * u + 1.3 * d) * np.cos(b * v) + c * u + 0.3 * np.sin(0.05 * (u + v)))
    F = np.array(F)
    F[:, 30:34, 40:45] = np.nan
    F[1, 5, 7] = np.nan
    F[2, 0, :] = np.nan
    return F


def _levels(F, L=9):
    lo, hi = np.nanmin(F, axis=(1, 2)), np.nanmax(F, axis=(1, 2))
    lev = lo[:, None] + (hi - lo)[:, None] * (np.arange(1, L + 1) ** 1.3 / (L + 1) ** 1.3)[None, :]
    lev[1, 4] = lev[1, 3]                                   # a repeated level (zero spacing)
    return lev


MODES = [(SM.LINES, [0]), (SM.LINES, [0, 2]), (SM.DISCRETE, [1]), (SM.DISCRETE, [0, 1]),
         (SM.DISCRETE_LINES, [2]), (SM.ADAPTIVE, [0]), (SM.ADAPTIVE, [1, 2]), (SM.GRADIENT, [0]),
         (SM.GRADIENT, [0, 1]), (SM.TEXTURE, [2]), (SM.TEXTURE, [0, 1])]


@pytest.mark.parametrize("fp64", [False, True], ids=["f32", "f64"])
@pytest.mark.parametrize("mode,dims", MODES, ids=[f"m{m}-{'.'.join(map(str, d))}" for m, d in MODES])
def test_space_map_bytes_match_oracle(mode, dims, fp64):
    import torch

    from paper_1408_0677_gb300 import space_map
    F = _field(3)
    if not fp64:
        F = F.astype(np.float32)
    lev = _levels(F)
    lo = [float(np.nanmin(F[d])) for d in dims]
    hi = [float(np.nanmax(F[d])) for d in dims]
    tex = np.random.default_rng(4).integers(0, 256, (23, 37, 4), dtype=np.uint8)
    kw = dict(line_width=1.5, fade=(2.0, 6.0, 4), lo=lo, hi=hi)
    out = space_map(torch.from_numpy(F).cuda(), lev, dims, mode, texture=torch.from_numpy(tex).cuda(), **kw)
    torch.cuda.synchronize()
    ref = SM.space_map(F, lev, dims, mode, texture=tex, **kw)
    got = out.cpu().numpy()
    bad = np.argwhere(np.any(got != ref, axis=2))
    assert bad.size == 0, f"{len(bad)} pixels differ, first {bad[:3].tolist()}: {got[tuple(bad[0])]} vs {ref[tuple(bad[0])]}"


def test_space_map_without_levels():
    import torch

    from paper_1408_0677_gb300 import space_map
    F = _field(5).astype(np.float32)
    lev = np.zeros((3, 0))
    out = space_map(torch.from_numpy(F).cuda(), lev, [0, 1], SM.GRADIENT, lo=[-1, -1], hi=[2, 2])
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), SM.space_map(F, lev, [0, 1], SM.GRADIENT, lo=[-1, -1], hi=[2, 2]))


@pytest.mark.parametrize("mode", [SM.DISCRETE_LINES, SM.ADAPTIVE])
def test_space_map_of_a_rendered_field(mode):
    """The wine-shaped workload rendered on the GPU (FP32), then mapped there;
    the oracle maps the same downloaded field."""
    import torch

    from paper_1408_0677_gb300 import Renderer, space_map
    wl = inputs.wine_shaped()
    r = Renderer(torch.from_numpy(wl.xy).cuda(), torch.from_numpy(wl.F).cuda(), degree=wl.degree, weight=wl.weight,
                 h=wl.h, precision="fp32")
    res = r.render(wl.W, wl.H, levels=wl.levels)
    r.sync()
    img = space_map(res["field"], wl.levels, [4], mode, line_width=1.0)
    torch.cuda.synchronize()
    field = res["field"].cpu().numpy()
    r.close()
    assert np.array_equal(img.cpu().numpy(), SM.space_map(field, wl.levels, [4], mode, line_width=1.0))
