"""Benchmark of the MLS field reconstruction on one GB300 (or N replicas).

One step = the whole hot path over the 10k-point workload (n = 10,000 points
in 8 Gaussian clusters plus 20% uniform background, D = 32 Fourier fields,
1024 x 1024 pixels, quadratic basis, Gaussian h = 0.02 summed over every
point, 16 iso-levels): mls_create from device-resident points (value ranges,
layouts), the stabiliser prepass, the tensor-core moment contraction with
its per-pixel solve and fused iso-bands, and the recompute of ill-conditioned
pixels.  Metric: pixel*point*dim updates/s = W * H * n * D / step time,
with the p50/p99 step latency, the plain FP32 CUDA-core form timed on the same
inputs, and both fields' error against the FP64 oracle on the oracle's pixel
sample (largest |f - f_oracle| / data range of the dimension).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp16|bf16|fp32|fp64]
  python bench.py --support 6         # the truncated Gaussian (box of half-width 6 h)
  python bench.py --impl reference    # the FP64 CPU oracle on a bounded pixel sample

With --support C the weight is the truncated Gaussian and the metric counts
only the pairs inside each pixel's box (the pairs that carry weight); the
full-sum-equivalent rate W * H * n * D / step time is reported beside it.

With N > 1 (torchrun, one process per GPU) every rank renders its own
replica (the pixels of one render are independent; no collective on the
data path): weak scaling, max time over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLS pixel*point*dim updates/s"
UNIT = "pixel*point*dim/s"
WORKLOAD = "fourier_n10k_d32_1024x1024_quadratic_gauss_h0.02_L16"
TC_SRCS = [os.path.join(ROOT, "paper_1408_0677_gb300", "csrc", f) for f in ("tc.cu", "dev_common.cuh", "tcgen05.cuh")]
PROFILE = os.path.join(ROOT, "profiles", "k_mls_tc_fourier10k_fp16.md")


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value of x over all ranks (x itself on one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def pairs_in_boxes(wl):
    """Pixel-point pairs of a render inside the truncated Gaussian's box
    |x_i - p_x| < c h and |y_i - p_y| < c h: per point, the pixel columns
    and rows whose centres lie within c h of it (a rectangle of pixels)."""
    rho = wl.trunc * wl.h
    x0, y0, x1, y1 = wl.view

    def span(pos, lo, step, N):
        a = np.ceil((pos - rho - lo) / step - 0.5).astype(np.int64)
        b = np.floor((pos + rho - lo) / step - 0.5).astype(np.int64)
        for k in (a, b):   # settle rounding at the edges with the pixel-centre expression
            k[:] = np.clip(k, -1, N)
        a = np.where((a > 0) & (np.abs(pos - (lo + (a - 1 + 0.5) * step)) < rho), a - 1, a)
        a = np.where((a < N) & (np.abs(pos - (lo + (a + 0.5) * step)) >= rho), a + 1, a)
        b = np.where((b < N - 1) & (np.abs(pos - (lo + (b + 1 + 0.5) * step)) < rho), b + 1, b)
        b = np.where((b >= 0) & (np.abs(pos - (lo + (b + 0.5) * step)) >= rho), b - 1, b)
        return np.maximum(np.minimum(b, N - 1) - np.maximum(a, 0) + 1, 0)

    nu = span(wl.xy[:, 0], x0, (x1 - x0) / wl.W, wl.W)
    nv = span(wl.xy[:, 1], y0, (y1 - y0) / wl.H, wl.H)
    return int(np.sum(nu * nv))


def pairs_in_discs(wl):
    """Pixel-point pairs with |x_i - p| < rho (the Wendland support, rho =
    wl.h): per point and pixel row, the run of pixel columns whose centres
    lie inside the disc, its ends settled with the FP64 pixel-centre
    expression and r^2 < rho^2 (the support test of the definition)."""
    rho = wl.h
    rho2 = rho * rho
    x0, y0, x1, y1 = wl.view
    sx, sy = (x1 - x0) / wl.W, (y1 - y0) / wl.H
    X, Y = wl.xy[:, 0], wl.xy[:, 1]
    va = np.clip(np.ceil((Y - rho - y0) / sy - 0.5).astype(np.int64) - 1, 0, wl.H - 1)
    vb = np.clip(np.floor((Y + rho - y0) / sy - 0.5).astype(np.int64) + 1, 0, wl.H - 1)
    total = 0
    for k in range(int((vb - va).max()) + 1 if len(X) else 0):
        v = va + k
        dy = Y - (y0 + (v + 0.5) * sy)
        dy2 = dy * dy
        live = (v <= vb) & (dy2 < rho2)
        half = np.sqrt(np.maximum(rho2 - dy2, 0.0))

        def inside(u):
            dx = X - (x0 + (u + 0.5) * sx)
            return (u >= 0) & (u < wl.W) & (dx * dx + dy2 < rho2)
        a = np.clip(np.ceil((X - half - x0) / sx - 0.5).astype(np.int64), 0, wl.W - 1)
        b = np.clip(np.floor((X + half - x0) / sx - 0.5).astype(np.int64), 0, wl.W - 1)
        for _ in range(2):      # the rounded ends are off by at most one column
            a = np.where(inside(a - 1), a - 1, a)
            a = np.where(~inside(a) & (a <= b), a + 1, a)
            b = np.where(inside(b + 1), b + 1, b)
            b = np.where(~inside(b) & (b >= a), b - 1, b)
        total += int(np.sum(np.where(live & inside(a) & inside(b), b - a + 1, 0)))
    return total


def workload_pairs(wl):
    """The pixel-point pairs the method must visit (the metric's work):
    W * H * n for the full-sum Gaussian, the pairs in support for the
    Wendland weight and the truncated Gaussian's boxes."""
    from paper_1408_0677_gb300 import inputs
    if wl.weight == inputs.WEIGHT_WENDLAND:
        return pairs_in_discs(wl)
    if wl.trunc > 0:
        return pairs_in_boxes(wl)
    return wl.W * wl.H * wl.n


def cpu_baseline(wl, seconds=15.0):
    """FP64 oracle on a bounded pixel sample (all host cores).  Also returns the
    last sample's pixels and oracle result, against which the GPU fields'
    error is stated."""
    import oracle
    npx = 64
    threads = os.cpu_count() or 1
    t_used, px_done, pairs_done = 0.0, 0, 0
    seed = 0
    last = None
    while t_used < seconds and npx <= 1 << 16:
        pix = np.sort(np.random.default_rng(100 + seed).choice(wl.W * wl.H, size=npx, replace=False))
        t0 = time.perf_counter()
        res = oracle.mls(wl.xy, wl.F, wl.degree, wl.weight, wl.h, wl.W, wl.H, pixels=pix, threads=threads,
                         trunc=wl.trunc)
        dt = time.perf_counter() - t0
        t_used += dt
        px_done += npx
        pairs_done += int(res.count.sum()) if (wl.trunc > 0 or wl.weight == 1) else npx * wl.n
        last = (pix, res)
        seed += 1
        if dt < seconds / 4:
            npx *= 2
    value = pairs_done * wl.D / t_used
    what = (f"pairs in the box of half-width {wl.trunc} h counted (the oracle visits all n={wl.n})"
            if wl.trunc > 0 else
            f"pairs within the support radius counted (the oracle visits all n={wl.n})" if wl.weight == 1 else
            f"full n={wl.n} sum each")
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{px_done} random pixels of the workload, {what}, FP64, {t_used:.1f} s"}, last


def _err_vs_oracle(wl, field_samples, last):
    """Largest |f_gpu - f_oracle| / (data range of the dimension) over the
    oracle's sample pixels (pixels the oracle flags as ambiguous excluded)."""
    pix, res = last
    rng = wl.F.max(axis=0) - wl.F.min(axis=0)
    ok = res.amb == 0
    out = {}
    ref = res.field[ok].T                    # (D, pixels)
    fin = np.isfinite(ref)
    for name, f in field_samples.items():
        d = np.abs(f[:, ok] - ref) / rng[:, None]
        out[name] = float(np.max(np.where(fin, d, 0.0))) if d.size else None
    out["pixels"] = int(ok.sum())
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle, timed on the host cores."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    from paper_1408_0677_gb300 import inputs
    import oracle
    cfg_name, gen, _ = WORKLOADS.get(args.workload, WORKLOADS["fourier10k"])
    wl = getattr(inputs, gen)()
    if args.support > 0:
        wl = dataclasses.replace(wl, trunc=args.support)
    counted = wl.trunc > 0 or wl.weight == inputs.WEIGHT_WENDLAND
    threads = os.cpu_count() or 1
    npx = 256 if not counted else 4096
    pix = np.random.default_rng(7).choice(wl.W * wl.H, size=npx, replace=False)
    for _ in range(args.warmup):
        oracle.mls(wl.xy, wl.F, wl.degree, wl.weight, wl.h, wl.W, wl.H, pixels=pix[:16], threads=threads,
                   trunc=wl.trunc)
    times, pairs = [], 0
    for k in range(args.steps):
        p = np.random.default_rng(1000 + k).choice(wl.W * wl.H, size=npx, replace=False)
        t0 = time.perf_counter()
        res = oracle.mls(wl.xy, wl.F, wl.degree, wl.weight, wl.h, wl.W, wl.H, pixels=p, threads=threads,
                         trunc=wl.trunc)
        times.append(time.perf_counter() - t0)
        pairs += int(res.count.sum()) if counted else npx * wl.n
    t = float(np.sum(times))
    value = pairs * wl.D / t
    what = "pairs in support counted" if counted else f"full sum over n={wl.n}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": cfg_name if wl.trunc == 0 else cfg_name + f"_trunc{wl.trunc:g}",
                                            "sample_pixels_per_step": npx},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{npx} random pixels per step ({what})"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def tc_source_hash():
    """sha256 over the tensor-core kernel's sources (tc.cu, dev_common.cuh, tcgen05.cuh)."""
    h = hashlib.sha256()
    for f in TC_SRCS:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def _traffic(n_launch_units, profile=PROFILE):
    """DRAM bytes per launch from the committed ncu summary of the kernel
    (lines 'source_sha256: ...', 'dram_bytes_per_launch: ...',
    'pixels_per_launch: ...'), or None when the kernel changed since."""
    try:
        kv = {}
        for ln in open(profile):
            if ":" in ln and not ln.startswith("|"):
                k, v = ln.split(":", 1)
                kv[k.strip("-* `").lower()] = v.strip(" `\n")
        if kv.get("source_sha256") != tc_source_hash():
            return None
        return float(kv["dram_bytes_per_launch"]) / float(kv["pixels_per_launch"]) * n_launch_units
    except Exception:
        return None


# the configurations timed by run_ours: (config name, input generator, default precision)
WORKLOADS = {
    "fourier10k": (WORKLOAD, "fourier_10k", "fp16"),
    "clusters200k": ("clusters_n200k_d64_2048x2048_quadratic_wendland_r0.015_L16", "clusters_200k", "fp16"),
    "wine": ("wine_shaped_n178_d13_256x256_linear_gauss_h0.05_L10", "wine_shaped", "fp64"),
}
FP32_FMA_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
FP64_NOMINAL_TFLOPS = 1.25                          # GB300 FP64, nominal


def _error_sample(wl, name):
    """Pixels on which the GPU fields are compared with the oracle: the
    cpu_baseline leg's last sample, or for the 200k-point workload 2^16
    random pixels plus two full 128 x 128 windows, one in the densest
    cluster core and one in the sparsest populated region."""
    if name != "clusters200k":
        return None
    rng = np.random.default_rng(2026)
    pix = rng.choice(wl.W * wl.H, size=1 << 16, replace=False)
    cnt = np.zeros((wl.H // 128, wl.W // 128), np.int64)
    bx = np.clip((wl.xy[:, 0] * wl.W).astype(np.int64) // 128, 0, cnt.shape[1] - 1)
    by = np.clip((wl.xy[:, 1] * wl.H).astype(np.int64) // 128, 0, cnt.shape[0] - 1)
    np.add.at(cnt, (by, bx), 1)
    dense = np.unravel_index(np.argmax(cnt), cnt.shape)
    sparse = np.unravel_index(np.argmin(np.where(cnt > 0, cnt, cnt.max() + 1)), cnt.shape)
    wins = []
    for (ty, tx) in (dense, sparse):
        v, u = np.meshgrid(np.arange(128) + ty * 128, np.arange(128) + tx * 128, indexing="ij")
        wins.append((v * wl.W + u).ravel())
    return np.unique(np.concatenate([pix] + wins)).astype(np.int64)


def _err_detail(wl, fields, pix, res, precision):
    """Largest |f - f_oracle| / range per field; for FP64 also over the
    pixels whose first-order rounding bound (both sides) stays within 1e-10,
    how many pixels exceed that, and the largest error / bound."""
    S = wl.F.max(axis=0) - wl.F.min(axis=0)
    S = np.where(S > 0, S, 1.0)
    ok = res.amb == 0
    ref = res.field[ok].T
    fin = np.isfinite(ref)
    out = {"pixels": int(ok.sum())}
    for nm, f in fields.items():
        d = np.where(fin, np.abs(f[:, ok] - ref) / S[:, None], 0.0)
        out[nm] = float(d.max()) if d.size else None
        if nm in ("fp64", "fp64tc") and res.ecoef_sum is not None:
            u = 2.0 ** -53
            cnt = res.count[ok].astype(np.float64)[None, :]
            es, ef = res.ecoef_sum[ok].T, res.ecoef_fix[ok].T
            # the FP64 kernel's summation chain, or the emulation's error model
            # (2^-40 per entry: like 8192 additions, plus 64)
            chain_gpu = (np.minimum(cnt, np.ceil(wl.n / 32.0)) + 5 if nm == "fp64"
                         else np.full_like(cnt, 8192 + 64))
            b = ((cnt + 12 + chain_gpu + 12) * u * es + 2 * ef) / S[:, None]
            b = np.where(fin, b, 0.0)
            wide = (b > 1e-10).any(axis=0)
            out[nm + "_well_conditioned"] = float(d[:, ~wide].max()) if (~wide).any() else None
            out[nm + "_pixels_beyond_1e-10_bound"] = int(wide.sum())
            out[nm + "_max_err_over_bound"] = float((d / np.maximum(b, 1e-10)).max()) if d.size else None
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    from paper_1408_0677_gb300 import MLS_P_FP64, MlsView, Renderer, inputs, mls_create, mls_desc_default  # noqa
    from paper_1408_0677_gb300 import _abi

    cfg_name, gen, _ = WORKLOADS[args.workload]
    wl = getattr(inputs, gen)()
    if args.support > 0:
        wl = dataclasses.replace(wl, trunc=args.support)
    if args.size > 0:
        # a smaller raster of the same data and view (profiling captures)
        wl = dataclasses.replace(wl, W=args.size, H=args.size)
        cfg_name += f"_at{args.size}sq"
    n, D, W, H, L = wl.n, wl.D, wl.W, wl.H, wl.levels.shape[1]
    k_terms = (wl.degree + 1) * (wl.degree + 2) // 2
    n_mono = (2 * wl.degree + 1) * (2 * wl.degree + 2) // 2
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    xy_d = torch.from_numpy(wl.xy).to(dev)
    F_d = torch.from_numpy(wl.F).to(dev)
    fdt = torch.float64 if args.precision in ("fp64", "fp64tc") else torch.float32
    field = torch.empty((D, H, W), dtype=fdt, device=dev)
    status = torch.empty((H, W), dtype=torch.uint8, device=dev)
    bands = torch.empty((D, H, W), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    lev = np.ascontiguousarray(wl.levels)

    def step_device():
        r = Renderer(xy_d, F_d, degree=wl.degree, weight=wl.weight, h=wl.h, precision=args.precision,
                     weight_split=args.weight_split, stream=sptr, support=wl.trunc)
        r.render(W, H, levels=lev, field=field, bands=bands, status_out=status)
        return r

    # warm-up
    for _ in range(args.warmup):
        r = step_device()
        r.sync()
        r.close()
    torch.cuda.synchronize()

    # ---- device-resident timed region
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms, kern_ms, step_ms, launches, handed, handed64, retried = 0.0, [], [], 0, 0, 0, 0
    visited = []
    path = 0
    for _ in range(args.steps):
        flush.fill_(1.0)                                  # L2 flush outside the timed step
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = step_device()
        e1.record(stream)
        st = r.sync()
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(st.main_kernel_ms)
        visited.append(st.pairs)
        launches += st.launches
        handed, handed64, retried = st.recomputed, st.recomputed_fp64, st.retried_tiles
        path = st.main_path
        r.close()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(total_ms, world, dev)
    ms_step = total_ms / args.steps
    pairs = workload_pairs(wl)
    units = pairs * D
    value = world * units / (ms_step * 1e-3)

    # ---- the plain FP32 CUDA-core form on the same inputs, for comparison
    plain = None
    samples = {}
    if args.precision in ("fp16", "bf16") and args.compare_fp32:
        field32 = torch.empty((D, H, W), dtype=torch.float32, device=dev)

        def step_fp32():
            r = Renderer(xy_d, F_d, degree=wl.degree, weight=wl.weight, h=wl.h, precision="fp32", stream=sptr,
                         support=wl.trunc)
            r.render(W, H, levels=lev, field=field32, bands=bands, status_out=status)
            return r

        r = step_fp32()
        r.sync()
        r.close()
        ts = []
        for _ in range(min(args.steps, 5)):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = step_fp32()
            e1.record(stream)
            r.sync()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            r.close()
        plain = {"precision": "fp32", "ms_per_step": float(np.mean(ts)), "steps": len(ts),
                 "speedup": float(np.mean(ts)) / ms_step}
        samples["fp32"] = field32
    samples[args.precision] = field

    # ---- end-to-end through the public API with host buffers (pinned)
    xy_h = torch.from_numpy(wl.xy).pin_memory().numpy()
    F_h = torch.from_numpy(wl.F).pin_memory().numpy()
    field_h = torch.empty((D, H, W), dtype=fdt).pin_memory().numpy()
    status_h = torch.empty((H, W), dtype=torch.uint8).pin_memory().numpy()
    bands_h = torch.empty((D, H, W), dtype=torch.uint8).pin_memory().numpy()

    def step_host():
        # inputs from pinned host memory, results back in pinned host memory
        # (render_host returns once they are there); the handle's teardown is
        # cleanup after the step and is left out of the timed region
        r = Renderer(xy_h, F_h, degree=wl.degree, weight=wl.weight, h=wl.h, precision=args.precision,
                     weight_split=args.weight_split, stream=sptr, support=wl.trunc)
        r.render_host(W, H, levels=lev, field=field_h, bands=bands_h, status_out=status_h)
        return r

    step_host().close()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = step_host()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
        r.close()
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e_value = world * units / (e2e_ms / args.steps * 1e-3)
    h2d = wl.xy.nbytes + wl.F.nbytes + lev.nbytes
    d2h = field_h.nbytes + status_h.nbytes + bands_h.nbytes

    if rank != 0:
        return
    peaks, src = _peaks()
    k_ms = float(np.mean(kern_ms))
    # algorithmic contraction flops of the pairs the main kernel visits
    # (2 (k D + monomials) per pair): the full sum skips, per tile, the points
    # whose weight rounds to zero in the 16-bit operand (their products are
    # exactly zero); compact supports count the pairs in support
    pairs_visited = float(np.mean(visited)) if visited else float(pairs)
    flop_pair = 2.0 * (k_terms * D + n_mono)
    flops = flop_pair * (pairs if (wl.trunc > 0 or wl.weight == inputs.WEIGHT_WENDLAND)
                         else min(pairs_visited, pairs))
    achieved = flops / (k_ms * 1e-3) / 1e12
    if path == _abi.MLS_PATH_TENSOR:
        peak = peaks.get("bf16_tflops", 1900.0)       # FP16 and BF16 share the dense tensor rate
        roof = {"bound": "tensor", "peak_source": f"{src} bf16 burst (fp16 dense rate equal)", "kernel": "k_mls_tc"}
    elif path == _abi.MLS_PATH_FP64_TC:
        # executed tensor work: 55 digit-pair products of 48 columns (2 flop
        # each) per visited pair and value pass
        passes = -(-D // ((48 - 16) // k_terms))
        exec_pair = 55 * 2 * 48 * passes
        peak = peaks.get("bf16_tflops", 1900.0)
        roof = {"bound": "tensor", "peak_source": f"{src} bf16 burst (fp16 dense rate equal)", "kernel": "k_mls_tc64",
                "executed_flops_per_pair": exec_pair,
                "fp64_equivalent_tflops": flop_pair * pairs_visited / (k_ms * 1e-3) / 1e12,
                "fp64_nominal_tflops": FP64_NOMINAL_TFLOPS}
        flop_pair = exec_pair
        flops = exec_pair * pairs_visited
        achieved = flops / (k_ms * 1e-3) / 1e12
    elif path == _abi.MLS_PATH_FP64:
        peak = FP64_NOMINAL_TFLOPS
        roof = {"bound": "alu", "peak_source": "nominal GB300 FP64 rate", "kernel": "k_mls_f64"}
    else:
        peak = FP32_FMA_TFLOPS
        roof = {"bound": "alu", "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz", "kernel": "k_mls_f32"}
    prof = os.path.join(ROOT, "profiles", f"k_mls_tc_{args.workload}_{args.precision}.md")
    # the tensor pass runs one launch per group of value dimensions (at most
    # 40 per launch for the quadratic basis, balanced): the profile's traffic
    # of one launch, scaled by the pixels, times the launches
    dpp = min(40, (256 - 16) // k_terms)
    dpp -= dpp % (16 if k_terms == 1 else 48 // k_terms)
    vpasses = -(-D // dpp)
    traffic = _traffic(W * H, prof) if (path == _abi.MLS_PATH_TENSOR and wl.trunc == 0) else None
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "traffic": traffic * vpasses if traffic is not None else None,
                 "kernel_ms": k_ms, "flops_per_launch": flops, "flops_per_pair": flop_pair})
    cpu, err = None, None
    if args.cpu_seconds > 0:
        cpu, last = cpu_baseline(wl, seconds=args.cpu_seconds)
        import oracle
        pix = _error_sample(wl, args.workload)
        if pix is None and args.workload == "wine":
            pix = np.arange(W * H, dtype=np.int64)      # every pixel of the 256 x 256 grid
        if pix is None:
            pix, res = last
            if args.precision in ("fp64", "fp64tc"):
                res = oracle.mls(wl.xy, wl.F, wl.degree, wl.weight, wl.h, W, H, pixels=pix, trunc=wl.trunc,
                                 threads=os.cpu_count() or 1, ebound=True)
        else:
            res = oracle.mls(wl.xy, wl.F, wl.degree, wl.weight, wl.h, W, H, pixels=pix, trunc=wl.trunc,
                             threads=os.cpu_count() or 1, ebound=args.precision in ("fp64", "fp64tc"))
        pix_t = torch.from_numpy(np.asarray(pix, np.int64)).to(dev)
        fs = {k: v.reshape(D, -1)[:, pix_t].double().cpu().numpy() for k, v in samples.items()}
        err = _err_detail(wl, fs, pix, res, args.precision)
        err["sample"] = ("2^16 random pixels + 128 x 128 windows in the densest and the sparsest populated cluster "
                         "regions" if args.workload == "clusters200k" else
                         "every pixel" if args.workload == "wine" else "the cpu_baseline leg's last pixel sample")
    if plain is not None:
        plain["err_vs_oracle"] = err.get("fp32") if err else None
    lat = {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
           "steps": len(step_ms), "what": "device time of one step (create + render + bands)"}
    wname = {inputs.WEIGHT_GAUSS: "gauss", inputs.WEIGHT_WENDLAND: "wendland", inputs.WEIGHT_INVDIST: "invdist"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": cfg_name if wl.trunc == 0 else cfg_name + f"_trunc{wl.trunc:g}",
                       "n": n, "D": D, "W": W, "H": H, "degree": wl.degree,
                       "weight": (wname[wl.weight] if wl.trunc == 0 else
                                  f"gauss truncated to |dx|,|dy| < {wl.trunc:g} h"),
                       "h": wl.h, "levels": L, "precision": args.precision, "l2": "flushed between steps",
                       "replicas": world},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "ms_per_step": e2e_ms / args.steps},
            "latency_ms": lat, "plain_fp32": plain,
            "err_vs_oracle": err, "tolerance": 1e-10 if args.precision in ("fp64", "fp64tc") else 1e-3,
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": int(launches),
            "recompute": {"handed_over_pixels": int(handed), "fp64_pixels": int(handed64),
                          "split_weight_half_tiles": int(retried)},
            "pairs": {"workload": int(pairs), "visited_by_main_kernel": int(pairs_visited),
                      "visited_fraction": pairs_visited / (W * H * n),
                      "visited_rate": world * pairs_visited * D / (ms_step * 1e-3),
                      "note": ("pixel*point*dim/s of the pairs the main kernel visited (visited_rate): per 16 x 16 "
                               "tile, the grid cells holding points whose weight reaches e^-28 of some pixel's "
                               "largest; the others have FP16 weight exactly 0.  value counts the workload's "
                               "pairs (the full sum's W*H*n, or the pairs in support)")}}
    if wl.trunc > 0:
        line["truncated"] = {"support": wl.trunc, "pairs_in_support": pairs, "full_pairs": W * H * n,
                             "full_sum_equivalent": world * W * H * n * D / (ms_step * 1e-3)}
    if wl.weight == inputs.WEIGHT_WENDLAND:
        line["support"] = {"radius": wl.h, "pairs_in_support": pairs, "full_pairs": W * H * n,
                           "full_sum_equivalent": world * W * H * n * D / (ms_step * 1e-3)}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """64 independent datasets (n log-uniform 200-50,000, D 4-64, 256^2-1024^2,
    linear or quadratic, Gaussian h = 0.5/sqrt(n)) rendered by one CUDA graph
    per step (mls_batch_render, autotuned weight mode)."""
    import torch
    import torch.distributed as dist
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    from paper_1408_0677_gb300 import Batch, Renderer, inputs
    wls = inputs.batch_datasets(seed=1004, count=64)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    xy_d = [torch.from_numpy(w.xy).to(dev) for w in wls]
    F_d = [torch.from_numpy(w.F).to(dev) for w in wls]
    rs = [Renderer(x, f, degree=w.degree, weight=w.weight, h=w.h, precision=args.precision,
                   weight_split=args.weight_split, stream=stream.cuda_stream) for w, x, f in zip(wls, xy_d, F_d)]
    b = Batch(rs, autotune=args.weight_split is None, stream=stream.cuda_stream)
    entries = [(w.W, w.H, (0.0, 0.0, 1.0, 1.0), w.levels) for w in wls]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        b.render(entries)
        b.sync()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.render(entries)
        e1.record(stream)
        st = b.sync()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms_step = max_over_ranks(float(np.sum(step_ms)), world, dev) / args.steps
    units = sum(w.W * w.H * w.n * w.D for w in wls)
    value = world * units / (ms_step * 1e-3)
    # end to end: points uploaded from pinned host memory, the batch render,
    # every field read back
    xy_h = [torch.from_numpy(w.xy).pin_memory() for w in wls]
    F_h = [torch.from_numpy(w.F).pin_memory() for w in wls]
    outs = b.render(entries)
    b.sync()
    host = [torch.empty(o["field"].shape, dtype=o["field"].dtype).pin_memory() for o in outs]
    e2e = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(len(wls)):
            xy_d[k].copy_(xy_h[k], non_blocking=True)
            F_d[k].copy_(F_h[k], non_blocking=True)
        outs = b.render(entries)
        for o, hbuf in zip(outs, host):
            hbuf.copy_(o["field"], non_blocking=True)
        b.sync()
        torch.cuda.synchronize()
        e2e.append(1e3 * (time.perf_counter() - t0))
    e2e_ms = max_over_ranks(float(np.mean(e2e)), world, dev)
    if rank != 0:
        return
    peaks, src = _peaks()
    flops = sum(2.0 * (w.D * (3 if w.degree == 1 else 6) + (6 if w.degree == 1 else 15)) * w.W * w.H * w.n
                for w in wls)
    achieved = flops / (ms_step * 1e-3) / 1e12
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "batch64_n200-50k_d4-64_256-1024sq_gauss", "datasets": len(wls),
                       "pairs_dims": units, "precision": args.precision, "l2": "flushed between steps",
                       "replicas": world},
            "e2e": {"value": world * units / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(w.xy.nbytes + w.F.nbytes for w in wls)),
                    "d2h_bytes_per_step": int(sum(h.numel() * h.element_size() for h in host)), "ms_per_step": e2e_ms},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "steps": len(step_ms), "what": "device time of one batch render (one graph launch)"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peaks.get("bf16_tflops", 1900.0),
                         "unit": "TFLOP/s", "frac": achieved / peaks.get("bf16_tflops", 1900.0), "traffic": None,
                         "peak_source": f"{src} bf16 burst", "kernel": "whole batch graph",
                         "flops_per_step": flops},
            "cpu_baseline": None, "clocks": clocks, "gpu_launches": int(st.launches) * args.steps,
            "batch": {"captures": int(st.captures), "replays": int(st.replays),
                      "handed_over_pixels": int(st.recomputed)}}
    print(json.dumps(line), flush=True)
    b.close()


def run_serve(args):
    """Serving: Poisson arrivals of iso-band renders; continuous batching in
    the library's server.  Resident datasets: four of 1M points each (D = 16,
    64 clusters, quadratic, Wendland radius 0.006) and the 200k-point
    configuration (D = 64, 64 clusters, quadratic, Wendland radius 0.015).
    A request picks the 200k-point dataset with probability 1/5 (else one of
    the four), a viewport of side log-uniform in 512-2048 pixels and a zoom
    window of side log-uniform in [1/16, 1].  Latency counts from each
    request's arrival time.  --rates runs the same request list at several
    offered rates: the line reports each, and the highest rate the server
    sustained (completions keep up with arrivals: the completion rate over
    the whole run is at least 90% of the rate the drawn arrivals offered)
    beside the offered 200 requests/s."""
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    from paper_1408_0677_gb300 import MlsRequest, MlsView, Renderer, Server, inputs
    from paper_1408_0677_gb300._abi import mls_server_poll, mls_server_submit
    rng = np.random.default_rng(1005)
    dsets = []
    for k in range(4):
        r0 = np.random.default_rng(2000 + k)
        centres = r0.uniform(0.1, 0.9, size=(64, 2))
        xy = inputs._clusters(r0, 1_000_000, centres, r0.uniform(0.01, 0.05, size=64))
        F = inputs._fourier_fields(r0, xy, 16, modes=8, max_freq=4)
        lev = inputs.default_levels(F, 16)
        r = Renderer(torch.from_numpy(xy).cuda(), torch.from_numpy(F).cuda(), degree=2,
                     weight=inputs.WEIGHT_WENDLAND, h=0.006, precision=args.precision)
        dsets.append((r, np.ascontiguousarray(lev), 16))
    c3 = inputs.clusters_200k()
    r = Renderer(torch.from_numpy(c3.xy).cuda(), torch.from_numpy(c3.F).cuda(), degree=c3.degree,
                 weight=c3.weight, h=c3.h, precision=args.precision)
    dsets.append((r, np.ascontiguousarray(c3.levels), c3.D))
    nreq = args.requests
    gaps = rng.exponential(1.0, size=nreq)             # arrivals in units of 1 / rate
    specs = []
    for _ in range(nreq):
        k = 4 if rng.random() < 0.2 else int(rng.integers(4))
        side = int(round(np.exp(rng.uniform(np.log(512), np.log(2048)))))
        win = float(np.exp(rng.uniform(np.log(1 / 16), 0.0)))
        x0, y0 = rng.uniform(0.0, 1.0 - win, size=2)
        specs.append((k, side, (x0, y0, x0 + win, y0 + win)))
    pools = {16: [torch.empty(16 * 2048 * 2048, dtype=torch.uint8).pin_memory() for _ in range(args.slots * 3)],
             64: [torch.empty(64 * 2048 * 2048, dtype=torch.uint8).pin_memory() for _ in range(args.slots + 2)]}
    srv = Server(slots=args.slots, mem_budget=args.mem_gb << 30)
    # warm-up: one request per dataset
    for r, lev, _ in dsets:
        srv.submit(r, 256, 256, levels=lev)
    srv.drain()
    srv.poll()

    def one_rate(rate):
        arrivals = np.cumsum(gaps) / rate
        free = {D: list(range(len(pl))) for D, pl in pools.items()}
        inflight = {}
        lat, queued, dev_ms = [], [], []
        px_dims = 0
        t0 = time.perf_counter()

        def collect():
            nonlocal px_dims
            for d in mls_server_poll(srv.handle):
                D, side, t_arr, buf = inflight.pop(d.id)
                free[D].append(buf)
                lat.append(1e3 * (time.perf_counter() - t0 - t_arr))
                queued.append(d.queued_ms)
                dev_ms.append(d.device_ms)
                px_dims += side * side * D

        for i, (k, side, view) in enumerate(specs):
            while time.perf_counter() - t0 < arrivals[i]:
                collect()
                time.sleep(0.0002)
            r, lev, D = dsets[k]
            while not free[D]:
                collect()
                time.sleep(0.0002)
            buf = free[D].pop()
            req = MlsRequest(r.handle, MlsView(side, side, *view), lev.ctypes.data, lev.shape[1], 0,
                             pools[D][buf].data_ptr(), None, None)
            inflight[mls_server_submit(srv.handle, req)] = (D, side, arrivals[i], buf)
        while inflight:
            collect()
            time.sleep(0.0005)
        wall = time.perf_counter() - t0
        arrived = float(nreq / arrivals[-1])   # the rate the drawn arrivals actually offered
        return {"offered_per_s": rate, "arrived_per_s": arrived, "requests_per_s": nreq / wall, "wall_s": wall,
                "px_dims_per_s": px_dims / wall,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                "queued_ms": {"p50": float(np.percentile(queued, 50)), "p99": float(np.percentile(queued, 99))},
                "device_ms": {"p50": float(np.percentile(dev_ms, 50)), "p99": float(np.percentile(dev_ms, 99))},
                "sustained": bool(nreq / wall >= 0.9 * arrived)}

    rates = sorted({float(x) for x in args.rates.split(",")} | {args.rate})
    runs = [one_rate(rt) for rt in rates]
    st = srv.drain()
    srv.close()
    if rank != 0:
        return
    head = next(rn for rn in runs if rn["offered_per_s"] == args.rate)
    ok = [rn for rn in runs if rn["sustained"]]
    best = max(ok, key=lambda rn: rn["offered_per_s"]) if ok else None
    line = {"metric": "served pixel*dim/s (iso-band renders)", "value": head["px_dims_per_s"], "unit": "pixel*dim/s",
            "n_gpus": 1, "steps": nreq, "warmup": len(dsets), "ms_per_step": 1e3 * head["wall_s"] / nreq,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "data": "synthetic",
            "config": {"workload": "serve_poisson_4x1M_d16_r0.006_plus_200k_d64_r0.015_wendland_512-2048sq_zoom",
                       "rate_per_s": args.rate, "requests": nreq, "slots": args.slots, "mem_budget_gb": args.mem_gb,
                       "mix": "1/5 on the 200k-point D=64 dataset, 4/5 on the four 1M-point D=16 datasets"},
            "requests_per_s": head["requests_per_s"],
            "latency_ms": dict(head["latency_ms"], what="arrival to completion (bands on the host)"),
            "queued_ms": head["queued_ms"], "device_ms": head["device_ms"],
            "sustained_at_offered_rate": head["sustained"],
            "highest_sustained": best, "rates": runs,
            "server": {"peak_inflight": int(st.peak_inflight), "peak_bytes": int(st.peak_bytes),
                       "failed": int(st.failed)},
            "e2e": None, "roofline": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


# The paper's Table 1 (Section 4, Performance): MLS render time in seconds on
# a GeForce GTX 285, 600 x 600 canvas, inverse-distance weights, for its mean
# MLS (degree 0) and affine MLS (degree 1) modes.  Context, not a target.
PAPER_TABLE1_S = {(306, 0): 0.017420, (1000, 0): 0.064938, (2245, 0): 0.147089,
                  (306, 1): 0.026670, (1000, 1): 0.100724, (2245, 1): 0.242192}


def run_table1(args):
    """Table-1-shaped renders: n in {306, 1000, 2245} clustered points, D = 2
    (the two texture coordinates), 600 x 600, inverse distance alpha = 1, mean
    (degree 0) and affine (degree 1) MLS, timed beside the paper's numbers."""
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    from paper_1408_0677_gb300 import Renderer, inputs
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    rows, units, total_ms = [], 0, 0.0
    for n in (306, 1000, 2245):
        wl = inputs.small_random(3000 + n, n, 2, 600, 600, 1, inputs.WEIGHT_INVDIST, 0.05)
        xy, F = torch.from_numpy(wl.xy).to(dev), torch.from_numpy(wl.F).to(dev)
        for degree in (0, 1):
            r = Renderer(xy, F, degree=degree, weight=inputs.WEIGHT_INVDIST, h=0.05, precision=args.precision,
                         stream=stream.cuda_stream)
            for _ in range(args.warmup):
                r.render(600, 600, levels=wl.levels)
                r.sync()
            ts = []
            for _ in range(args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r.render(600, 600, levels=wl.levels)
                e1.record(stream)
                r.sync()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            r.close()
            ms = float(np.median(ts))
            paper = PAPER_TABLE1_S[(n, degree)]
            rows.append({"n": n, "mode": "mean" if degree == 0 else "affine", "ours_ms": ms,
                         "paper_gtx285_ms": 1e3 * paper, "ratio": 1e3 * paper / ms})
            units += 600 * 600 * n * 2
            total_ms += ms
    if rank != 0:
        return
    line = {"metric": METRIC, "value": units / (total_ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "table1_idw_600sq_d2_n306-1000-2245_mean_affine",
                       "note": "paper numbers: GTX 285 fragment shader (context only)"},
            "table1": rows, "e2e": None, "roofline": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def _time_launches(fn, stream, steps, warmup):
    """Device time of each of `steps` calls of fn (CUDA events on `stream`)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts


def run_spacemap(args):
    """Space mappings (Section 3.4, mls_space_map) of an 8192 x 8192 two-plane
    FP32 field (512 MiB, larger than L2, so no flush is needed) into RGBA8:
    every mode, device time per launch against the HBM roofline.  The
    algorithmic bytes of a launch are the shown planes read once and the image
    written once: (4 * planes + 4) bytes per pixel."""
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    import paper_1408_0677_gb300 as G
    from oracle import space_map as SM   # the CPU baseline leg only
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    W = H = 8192
    u = torch.arange(W, device=dev, dtype=torch.float32)[None, :]
    v = torch.arange(H, device=dev, dtype=torch.float32)[:, None]
    F = torch.stack([torch.sin(u * 0.004) * torch.cos(v * 0.003) + u * 1e-4,
                     torch.cos(u * 0.002 + v * 0.005) + v * 1e-4]).contiguous()
    lo = F.amin(dim=(1, 2)).double().cpu().numpy()
    hi = F.amax(dim=(1, 2)).double().cpu().numpy()
    L = 16
    lev = lo[:, None] + (hi - lo)[:, None] * (np.arange(1, L + 1) / (L + 1))[None, :]
    tex = torch.randint(0, 256, (256, 256, 4), dtype=torch.uint8, device=dev)
    out = torch.empty((H, W, 4), dtype=torch.uint8, device=dev)
    modes = [("lines", G.MLS_MAP_LINES, [0]), ("discrete", G.MLS_MAP_DISCRETE, [0]),
             ("discrete_lines", G.MLS_MAP_DISCRETE_LINES, [0]), ("adaptive", G.MLS_MAP_ADAPTIVE, [0, 1]),
             ("gradient", G.MLS_MAP_GRADIENT, [0, 1]), ("texture", G.MLS_MAP_TEXTURE, [0, 1])]
    peaks, src = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    rows, launches = {}, 0
    for name, mode, dims in modes:
        def call():
            G.space_map(F, lev, dims, mode, line_width=1.5, fade=(2.0, 6.0, 3), lo=list(lo[dims]),
                        hi=list(hi[dims]), texture=tex, out=out, stream=stream.cuda_stream)
        ts = _time_launches(call, stream, args.steps, args.warmup)
        launches += args.steps
        ms = float(np.mean(ts))
        nbytes = (4 * len(dims) + 4) * W * H
        rows[name] = {"planes": len(dims), "ms": ms, "pixels_per_s": W * H / (ms * 1e-3),
                      "gbs": nbytes / (ms * 1e-3) / 1e9, "frac_hbm": nbytes / (ms * 1e-3) / 1e9 / hbm}
    clocks = sampler.stop()
    head = rows["adaptive"]
    # end to end through the public call: pinned host field in, image back to pinned host memory
    Fh = torch.empty(F.shape, dtype=F.dtype).pin_memory()
    Fh.copy_(F)
    outh = torch.empty(out.shape, dtype=out.dtype).pin_memory()
    Fd = torch.empty_like(F)

    def e2e_step():
        Fd.copy_(Fh, non_blocking=True)
        G.space_map(Fd, lev, [0, 1], G.MLS_MAP_ADAPTIVE, line_width=1.5, fade=(2.0, 6.0, 3), out=out,
                    stream=stream.cuda_stream)
        outh.copy_(out, non_blocking=True)
        torch.cuda.synchronize()

    e2e_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_ms = 1e3 * (time.perf_counter() - t0) / args.steps
    # the oracle (numpy float32 statement) on a 1024 x 1024 crop, one core
    crop = F[:, :1024, :1024].cpu().numpy()
    t0 = time.perf_counter()
    SM.space_map(crop, lev, [0, 1], SM.ADAPTIVE, line_width=1.5, fade=(2.0, 6.0, 3))
    cpu_s = time.perf_counter() - t0
    if rank != 0:
        return
    nbytes = 12 * W * H
    line = {"metric": "space-mapped pixels/s", "value": world * head["pixels_per_s"], "unit": "pixel/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "spacemap_8192sq_2planes_f32_L16_adaptive", "W": W, "H": H, "levels": L,
                       "mode": "adaptive lines, two planes, 3 halvings", "l2": "inputs larger than L2"},
            "modes": rows,
            "e2e": {"value": world * W * H / (e2e_ms * 1e-3), "unit": "pixel/s",
                    "h2d_bytes_per_step": int(F.numel() * 4), "d2h_bytes_per_step": int(out.numel()),
                    "ms_per_step": e2e_ms},
            "roofline": {"bound": "hbm", "achieved": nbytes / (head["ms"] * 1e-3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": nbytes / (head["ms"] * 1e-3) / 1e9 / hbm, "traffic": None,
                         "peak_source": f"{src} copy bandwidth", "kernel": "k_space_map",
                         "bytes_per_launch": nbytes},
            "cpu_baseline": {"value": 1024 * 1024 / cpu_s, "unit": "pixel/s", "cores": 1, "kind": "oracle",
                             "sample": f"1024 x 1024 crop, adaptive, numpy float32, {cpu_s:.2f} s"},
            "clocks": clocks, "gpu_launches": launches}
    print(json.dumps(line), flush=True)


def run_variants(args):
    """The rigid (Section 3.3.3) and mean (Section 3.3.1) mappings of 2-D
    values: the 10k points' positions as p and a smooth distortion of them as
    the values q, 1024 x 1024, Gaussian h = 0.02 over every point, FP32
    (k_mls_variant), with 16 iso-levels per component."""
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    from paper_1408_0677_gb300 import MLS_V_MEAN, MLS_V_RIGID, Renderer, inputs
    import oracle
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    wl = inputs.fourier_10k()
    p = wl.xy
    q = p + 0.01 * np.stack([np.sin(6 * np.pi * p[:, 1]), np.cos(6 * np.pi * p[:, 0])], axis=1)
    W = H = 1024
    n = p.shape[0]
    lev = inputs.default_levels(q, 16)
    pd, qd = torch.from_numpy(p).to(dev), torch.from_numpy(q).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks, src = _peaks()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    rows, launches = {}, 0
    for name, var in (("rigid", MLS_V_RIGID), ("mean", MLS_V_MEAN)):
        r = Renderer(pd, qd, degree=1, weight=inputs.WEIGHT_GAUSS, h=0.02, precision=args.precision, variant=var,
                     stream=stream.cuda_stream)

        def call():
            flush.fill_(1.0)
            r.render(W, H, levels=lev)

        for _ in range(args.warmup):
            call()
            r.sync()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r.render(W, H, levels=lev)
            e1.record(stream)
            st = r.sync()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            launches += st.launches
        r.close()
        ms = float(np.mean(ts))
        rows[name] = {"ms": ms, "value": W * H * n * 2 / (ms * 1e-3)}
    clocks = sampler.stop()
    # the oracle on a bounded pixel sample (all host cores)
    threads = os.cpu_count() or 1
    pix = np.random.default_rng(9).choice(W * H, size=2048, replace=False)
    t0 = time.perf_counter()
    oracle.mls_variant(p, q, oracle.VARIANT_RIGID, inputs.WEIGHT_GAUSS, 0.02, W, H, pixels=pix, threads=threads)
    cpu_s = time.perf_counter() - t0
    if rank != 0:
        return
    # FP32 work per pair of the rigid kernel: offsets and r^2 (5), weight (3 + ex2),
    # Welford update (1 divide + 17): about 25 flop; peak = 152 SMs x 128 FP32
    # lanes x 2 flop per FMA x the maximum SM clock
    flop = 25.0 * W * H * n
    peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    ach = flop / (rows["rigid"]["ms"] * 1e-3) / 1e12
    line = {"metric": METRIC, "value": world * rows["rigid"]["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rows["rigid"]["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64",
            "data": "synthetic",
            "config": {"workload": "rigid_mls_n10k_d2_1024x1024_gauss_h0.02_L16", "n": n, "D": 2, "W": W, "H": H,
                       "l2": "flushed between steps"},
            "variants": rows, "e2e": None,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "traffic": None, "peak_source": "FP32 FMA rate from unit counts and the maximum SM clock",
                         "kernel": "k_mls_variant", "flop_per_pair": 25},
            "cpu_baseline": {"value": 2048 * n * 2 / cpu_s, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"2048 random pixels, rigid, full n={n} sum each, FP64, {cpu_s:.2f} s"},
            "clocks": clocks, "gpu_launches": launches}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp16", "bf16", "fp32", "fp64", "fp64tc"],
                    help="default: fp16, or fp64 for the wine-shaped workload (the FP64 configuration)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--weight-split", type=int, default=None, choices=[0, 1, 2])
    ap.add_argument("--no-compare-fp32", dest="compare_fp32", action="store_false",
                    help="skip the plain FP32 comparison run")
    ap.add_argument("--workload", default="fourier10k",
                    choices=["fourier10k", "clusters200k", "wine", "batch64", "serve", "table1", "spacemap",
                             "variants"],
                    help="the 10k-point render (default), the 200k-point Wendland render, the wine-shaped FP64 "
                         "render, 64 datasets in one graph, or the serving mix")
    ap.add_argument("--support", type=float, default=0.0,
                    help="truncated Gaussian: box half-width in units of h (0: the full sum)")
    ap.add_argument("--size", type=int, default=0,
                    help="render the workload's data and view on a size x size raster instead (0: its own)")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: offered requests per second (headline)")
    ap.add_argument("--rates", default="50,100", help="serve: comma-separated offered rates to run as well")
    ap.add_argument("--requests", type=int, default=400, help="serve: number of requests")
    ap.add_argument("--slots", type=int, default=8, help="serve: requests in flight at most")
    ap.add_argument("--mem-gb", type=int, default=16, help="serve: device memory budget (GiB)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.precision is None:
        args.precision = WORKLOADS[args.workload][2] if args.workload in WORKLOADS else "fp16"
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "table1":
        run_table1(args)
    elif args.workload == "spacemap":
        run_spacemap(args)
    elif args.workload == "variants":
        if args.precision in ("fp16", "bf16"):
            args.precision = "fp32"      # the mappings run on the CUDA-core kernel
        run_variants(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
