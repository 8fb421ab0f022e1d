"""The hand-over's two forms.  Pixels that the reduced-precision passes hand
over are recomputed by four kernels (setup, double-float moments, degree
policy in double-float, double-float values; per-entry state in global
memory) for the first entries of a long list, up to a state capacity, and by
one fused kernel (a block per chunk of pixels, phases separated by block
barriers, degree policy in FP64) for short lists and for the entries past
that capacity.  The moments and values are the same arithmetic in both; the
policies differ in rounding only.  So whichever form takes an entry (the
default choice, all split, all fused, a mix) the same pixels are handed
over and passed on to FP64, with the same status wherever the oracle's
degree decision is not near its threshold, and every render matches
the oracle (the weighted least-squares fit of Section 3.3)."""
import numpy as np
import pytest

from paper_1408_0677_gb300 import inputs
from tests.gpu_util import compare, gpu_render, oracle_ref

pytestmark = pytest.mark.gpu

G, WEND = inputs.WEIGHT_GAUSS, inputs.WEIGHT_WENDLAND


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


CASES = [
    ("wine", "fp16", lambda: inputs.wine_shaped()),
    ("fourier_gauss", "bf16", lambda: inputs.fourier_mix(seed=21, n=3000, D=5, W=160, H=160, degree=2,
                                                          weight=G, h=0.03)),
    ("fourier_wendland", "fp16", lambda: inputs.fourier_mix(seed=22, n=4000, D=7, W=192, H=160, degree=2,
                                                             weight=WEND, h=0.04)),
    ("fourier_linear", "bf16", lambda: inputs.fourier_mix(seed=23, n=2500, D=3, W=128, H=144, degree=1,
                                                           weight=G, h=0.035)),
]


@pytest.mark.parametrize("name,precision,make", CASES, ids=[c[0] + "-" + c[1] for c in CASES])
def test_split_and_fused_handover_agree(name, precision, make):
    wl = make()
    split = gpu_render(wl, precision, handover_split=(-1, 0))
    n = split["stats"].recomputed
    assert n > 0, "the case must hand pixels over"
    default = gpu_render(wl, precision)
    fused = gpu_render(wl, precision, handover_split=(0, -1))
    mixed = gpu_render(wl, precision, handover_split=(max(1, n // 3), 0))
    ref = oracle_ref(wl)
    S = wl.F.max(0) - wl.F.min(0)
    for label, res in (("split", split), ("default", default), ("fused", fused), ("mixed", mixed)):
        assert res["stats"].recomputed == n
        assert res["stats"].recomputed_fp64 == split["stats"].recomputed_fp64
        clear = (ref.amb == 0).reshape(res["status"].shape)   # no degree decision near its threshold
        assert np.array_equal(res["status"][clear], split["status"][clear])
        err, npx = compare(wl, res, ref, precision)
        dmax = np.nanmax(np.abs(res["field"].astype(np.float64) - split["field"]) / S[:, None, None])
        print(f"{name} {precision} {label}: {n} pixels handed over ({res['stats'].recomputed_fp64} on to "
              f"FP64), max err {err:.3g} of range, {dmax:.2g} from the split form")
