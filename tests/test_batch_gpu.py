"""Batched rendering (mls_batch_*): one CUDA graph over many resident
datasets gives exactly the results of rendering each dataset alone, on the
capture, on replays and after a view change; with the autotuner the results
stay within the oracle tolerance."""
import numpy as np
import pytest

import oracle
from paper_1408_0677_gb300 import inputs
from tests.gpu_util import compare, oracle_ref

pytestmark = pytest.mark.gpu

PRECS = ["fp16", "fp32", "bf16", "fp64", "fp16", "fp32"]


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


def _datasets():
    return inputs.batch_datasets(seed=77, count=len(PRECS), n_range=(200, 4000), D_range=(3, 20),
                                 side_range=(40, 110))


def _renderers(wls, **kw):
    import torch

    from paper_1408_0677_gb300 import Renderer
    return [Renderer(torch.from_numpy(w.xy).cuda(), torch.from_numpy(w.F).cuda(), degree=w.degree, weight=w.weight,
                     h=w.h, precision=pr, **kw) for w, pr in zip(wls, PRECS)]


def _alone(r, W, H, view, lev):
    out = r.render(W, H, view=view, levels=lev)
    r.sync()
    return {k: (v.clone() if v is not None else None) for k, v in out.items()}


def _same(a, b):
    import torch
    assert torch.equal(torch.isnan(a["field"]), torch.isnan(b["field"]))
    assert torch.equal(torch.nan_to_num(a["field"]), torch.nan_to_num(b["field"]))
    assert torch.equal(a["status"], b["status"])
    assert torch.equal(a["bands"], b["bands"])


def test_batch_equals_renders_alone_capture_replay_recapture(built):
    from paper_1408_0677_gb300 import Batch
    wls = _datasets()
    rs = _renderers(wls)
    entries = [(w.W, w.H, (0.0, 0.0, 1.0, 1.0), w.levels) for w in wls]
    alone = [_alone(r, *e) for r, e in zip(rs, entries)]
    b = Batch(rs)
    for rep in range(2):
        outs = b.render(entries)
        st = b.sync()
        for a, o in zip(alone, outs):
            _same(a, o)
    assert st.captures == 1 and st.replays == 2 and st.datasets == len(rs) and st.launches > 0
    # a new view (zoom window) re-captures
    entries2 = [(w.W // 2 + 3, w.H, (0.2, 0.1, 0.7, 0.9), w.levels) for w in wls]
    alone2 = [_alone(r, *e) for r, e in zip(rs, entries2)]
    outs = b.render(entries2)
    st = b.sync()
    for a, o in zip(alone2, outs):
        _same(a, o)
    assert st.captures == 2 and st.replays == 3
    b.close()
    for r in rs:
        r.close()


def test_batch_with_autotune_matches_oracle(built):
    from paper_1408_0677_gb300 import Batch
    wls = _datasets()
    rs = _renderers(wls)
    b = Batch(rs, autotune=True)
    outs = b.render([(w.W, w.H, (0.0, 0.0, 1.0, 1.0), w.levels) for w in wls])
    b.sync()
    for w, pr, o in zip(wls, PRECS, outs):
        pix = inputs.sample_pixels(5, w.W, w.H, 300)
        ref = oracle_ref(w, pix)
        res = {k: (v.cpu().numpy() if v is not None else None) for k, v in o.items()}
        # h = 0.5 / sqrt(n) leaves most pixels of the sparse datasets with a
        # handful of effective points: the FP64 rounding bound exceeds 1e-10
        # of the range on most of them
        compare(w, res, ref, pr, pixels=pix, max_allow_frac=0.70 if pr == "fp64" else None)
    b.close()
    for r in rs:
        r.close()


def test_batch_argument_errors(built):
    from paper_1408_0677_gb300 import MlsError, _abi
    wls = _datasets()[:2]
    rs = _renderers(wls)
    with pytest.raises(MlsError):
        _abi.mls_batch_create([rs[0].handle, rs[0].handle])
    with pytest.raises(MlsError):
        _abi.mls_batch_create([])
    for r in rs:
        r.close()
