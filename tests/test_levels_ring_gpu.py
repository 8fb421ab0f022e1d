"""Level uploads of back-to-back renders: each render copies its iso-levels
through a ring of pinned host slots without waiting for its stream, so a
render enqueued before the previous one has run must still label its bands
with its own levels.  Renders with distinct levels (more of them than the
ring has slots) are enqueued on one stream with no synchronisation in
between, from one handle and from two, and each render's bands must be the
count #{t <= f} of its own levels on its own field (f in float32 against the
levels rounded up to float32, the rule the kernels use)."""
import numpy as np
import pytest

from paper_1408_0677_gb300 import inputs

pytestmark = pytest.mark.gpu

RENDERS = 20   # more than the ring's slots


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _levels_up(lev):
    """Levels rounded up to float32: for a float32 f, f >= t exactly when f >= t_up."""
    up = lev.astype(np.float32)
    low = up.astype(np.float64) < lev
    up[low] = np.nextafter(up[low], np.float32(np.inf))
    return up


def _expected_bands(field, lev):
    up = _levels_up(lev)
    f = field.astype(np.float32)
    b = np.zeros(f.shape, np.int64)
    for d in range(f.shape[0]):
        b[d] = (f[d][None, :, :] >= up[d][:, None, None]).sum(axis=0)
    b[np.isnan(f)] = 255
    return b.astype(np.uint8)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("handles", [1, 2])
def test_back_to_back_renders_use_their_own_levels(precision, handles):
    import torch

    from paper_1408_0677_gb300 import Renderer
    wl = inputs.small_random(7101, n=400, D=3, W=48, H=40, degree=2, weight=inputs.WEIGHT_GAUSS, h=0.06, L=9)
    xy, F = torch.from_numpy(wl.xy).cuda(), torch.from_numpy(wl.F).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    rs = [Renderer(xy, F, degree=wl.degree, weight=wl.weight, h=wl.h, precision=precision, stream=stream)
          for _ in range(handles)]
    base = np.asarray(wl.levels, np.float64)
    span = base[:, -1:] - base[:, :1]
    outs, levs = [], []
    for k in range(RENDERS):
        # distinct ascending levels per render: the set shifted by a fraction of its span
        lev = base + span * (0.013 * k - 0.1)
        out = rs[k % handles].render(wl.W, wl.H, levels=lev)
        outs.append(out)
        levs.append(lev)
    torch.cuda.synchronize()
    for r in rs:
        r.sync()
    for k, (out, lev) in enumerate(zip(outs, levs)):
        field = out["field"].cpu().numpy()
        bands = out["bands"].cpu().numpy()
        exp = _expected_bands(field, lev)
        bad = int((bands != exp).sum())
        assert bad == 0, f"render {k}: {bad} band labels differ from its own levels"
    for r in rs:
        r.close()
