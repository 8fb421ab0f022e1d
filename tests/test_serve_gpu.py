"""Serving (mls_server_*): requests admitted by slots and device memory,
overlapping on the device, give each exactly the result of the same render
alone; the memory budget bounds what is in flight; oversized requests are
refused at submit."""
import time

import numpy as np
import pytest

from paper_1408_0677_gb300 import inputs

pytestmark = pytest.mark.gpu

G, WD = inputs.WEIGHT_GAUSS, inputs.WEIGHT_WENDLAND


@pytest.fixture(scope="module")
def datasets():
    import __graft_entry__
    __graft_entry__.build()
    import torch

    from paper_1408_0677_gb300 import Renderer
    specs = [(inputs.fourier_mix(61, 4000, 6, 96, 96, 2, G, 0.03), "fp16"),
             (inputs.fourier_mix(62, 30000, 5, 96, 96, 2, WD, 0.03), "fp32"),
             (inputs.fourier_mix(63, 3000, 4, 96, 96, 1, G, 0.04), "bf16")]
    rs = [(w, Renderer(torch.from_numpy(w.xy).cuda(), torch.from_numpy(w.F).cuda(), degree=w.degree,
                       weight=w.weight, h=w.h, precision=p)) for w, p in specs]
    yield rs
    for _, r in rs:
        r.close()


def _requests(rs, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        k = int(rng.integers(len(rs)))
        side = float(np.exp(rng.uniform(np.log(1 / 8), 0)))
        x0, y0 = rng.uniform(0, 1 - side, size=2)
        W, H = int(rng.integers(40, 150)), int(rng.integers(40, 150))
        out.append((k, W, H, (x0, y0, x0 + side, y0 + side)))
    return out


def _alone(w, r, W, H, view):
    o = r.render(W, H, view=view, levels=w.levels)
    r.sync()
    return {k: v.cpu().numpy() for k, v in o.items()}


def _check(req, ref):
    assert req.done.status == 0
    assert np.array_equal(req.bands.numpy(), ref["bands"])
    assert np.array_equal(req.status.numpy(), ref["status"])
    assert np.array_equal(req.field.numpy(), ref["field"], equal_nan=True)


def test_requests_in_the_mix_equal_requests_alone(datasets):
    from paper_1408_0677_gb300 import Server
    reqs = _requests(datasets, 30, 1)
    srv = Server(slots=4, mem_budget=2 << 30)
    subs = []
    for k, W, H, view in reqs:
        w, r = datasets[k]
        subs.append((srv.submit(r, W, H, view, levels=w.levels, field=True), k, W, H, view))
    st = srv.drain()
    done = {q.id: q for q in srv.poll()}
    assert st.completed == st.submitted == len(reqs) and st.failed == 0
    assert st.peak_inflight > 1            # requests overlapped on the device
    for q, k, W, H, view in subs:
        assert q.id in done and q.done.latency_ms >= q.done.queued_ms >= 0.0
        w, r = datasets[k]
        _check(q, _alone(w, r, W, H, view))
    srv.close()


def test_memory_budget_bounds_requests_in_flight(datasets):
    from paper_1408_0677_gb300 import Server
    reqs = _requests(datasets, 12, 2)
    srv = Server(slots=8, mem_budget=3 << 20)      # room for about one request
    subs = []
    for k, W, H, view in reqs:
        w, r = datasets[k]
        subs.append((srv.submit(r, W, H, view, levels=w.levels, field=True), k, W, H, view))
    st = srv.drain()
    srv.poll()
    assert st.completed == len(reqs) and st.failed == 0
    assert st.peak_bytes <= 3 << 20 and st.peak_inflight <= 8
    for q, k, W, H, view in subs:
        w, r = datasets[k]
        _check(q, _alone(w, r, W, H, view))
    srv.close()


def test_arrivals_while_busy_and_oversized_request(datasets):
    from paper_1408_0677_gb300 import MlsError, Server
    srv = Server(slots=3, mem_budget=64 << 20)
    w, r = datasets[0]
    with pytest.raises(MlsError) as e:
        srv.submit(r, 4096, 4096, levels=w.levels, field=True)
    assert e.value.status == 2
    subs = []
    for wave in range(3):                          # later waves arrive while earlier ones run
        for k, W, H, view in _requests(datasets, 6, 10 + wave):
            wk, rk = datasets[k]
            subs.append((srv.submit(rk, W, H, view, levels=wk.levels, field=True), k, W, H, view))
        time.sleep(0.002)
    srv.drain()
    srv.poll()
    for q, k, W, H, view in subs:
        wk, rk = datasets[k]
        _check(q, _alone(wk, rk, W, H, view))
    srv.close()


def test_served_results_match_the_oracle(datasets):
    """Served renders of zoom windows (side 1/8 to 1 of the square, ragged
    rasters) against the FP64 oracle on sampled pixels of every request: a
    mistake common to the served and the lone render would pass the tests
    above but not this one."""
    import dataclasses

    from paper_1408_0677_gb300 import Server
    from tests.gpu_util import compare, oracle_ref
    precs = ["fp16", "fp32", "bf16"]
    reqs = _requests(datasets, 18, 3)
    srv = Server(slots=4, mem_budget=2 << 30)
    subs = []
    for k, W, H, view in reqs:
        w, r = datasets[k]
        subs.append((srv.submit(r, W, H, view, levels=w.levels, field=True), k, W, H, view))
    st = srv.drain()
    srv.poll()
    assert st.completed == len(reqs) and st.failed == 0
    for i, (q, k, W, H, view) in enumerate(subs):
        w, _ = datasets[k]
        wl = dataclasses.replace(w, W=W, H=H, view=tuple(float(x) for x in view))
        pix = inputs.sample_pixels(100 + i, W, H, 400)
        res = {"field": q.field.numpy(), "status": q.status.numpy(), "bands": q.bands.numpy()}
        compare(wl, res, oracle_ref(wl, pix), precs[k], pixels=pix)
    srv.close()
