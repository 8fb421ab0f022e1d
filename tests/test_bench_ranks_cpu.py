"""The multi-process side of bench.py on CPU (gloo, world size 2): the
max-over-ranks timing and the reference arm under torchrun, where rank 0
alone prints one JSON line.  Each rank renders its own replica, so the data
path has no collective; only the timing reduction crosses ranks."""
import dataclasses
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    w, r, _ = bench._dist()
    got = bench.max_over_ranks(10.0 * (rank + 1), w, "cpu")
    q.put((r, w, got))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 20.0), (1, 2, 20.0)]


def test_reference_arm_under_torchrun_prints_one_line():
    import __graft_entry__
    __graft_entry__.build()
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    # every key of the one-line contract, with its type
    for key, typ in (("metric", str), ("value", float), ("unit", str), ("steps", int), ("warmup", int),
                     ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str), ("dtype", str),
                     ("data", str), ("config", dict), ("cpu_baseline", dict), ("e2e", dict)):
        assert isinstance(d[key], typ), (key, d.get(key))
    assert "vs_baseline" in d and d["warmup"] >= 3 and d["steps"] == 1
    assert d["e2e"]["unit"] == d["unit"] and d["cpu_baseline"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_pairs_in_boxes_equals_the_oracle_counts():
    """bench.py counts the truncated Gaussian's pixel-point pairs per point
    (the rectangle of pixels its box covers); the oracle counts them per
    pixel.  Both must agree exactly, including ragged rasters and zoomed
    views."""
    import dataclasses

    import oracle
    sys.path.insert(0, ROOT)
    import bench
    from paper_1408_0677_gb300 import inputs
    for wl, c in ((inputs.small_random(61, 80, 3, 41, 29, 2, 0, 0.05), 2.0),
                  (inputs.fourier_mix(51, 3000, 2, 77, 53, 1, 0, 0.02), 3.0)):
        for view in ((0.0, 0.0, 1.0, 1.0), (0.2, 0.1, 0.7, 0.45)):
            w = dataclasses.replace(wl, trunc=c, view=view)
            r = oracle.mls(w.xy, w.F, w.degree, w.weight, w.h, w.W, w.H, view=view, trunc=c)
            assert bench.pairs_in_boxes(w) == int(r.count.sum())


def test_pairs_in_discs_equals_the_oracle_counts():
    """bench.py counts the Wendland weight's in-support pairs per point (the
    pixel columns of each row inside its disc); the oracle counts them per
    pixel.  Both must agree exactly, including ragged rasters and zoomed
    views."""
    import oracle
    sys.path.insert(0, ROOT)
    import bench
    from paper_1408_0677_gb300 import inputs
    for wl in (inputs.small_random(62, 300, 2, 41, 29, 2, 1, 0.07),
               inputs.fourier_mix(52, 20000, 2, 77, 53, 2, 1, 0.02)):
        for view in ((0.0, 0.0, 1.0, 1.0), (0.2, 0.1, 0.7, 0.45), (0.31, 0.42, 0.3725, 0.4625)):
            w = dataclasses.replace(wl, view=view)
            r = oracle.mls(w.xy, w.F, w.degree, w.weight, w.h, w.W, w.H, view=view)
            assert bench.pairs_in_discs(w) == int(r.count.sum())
