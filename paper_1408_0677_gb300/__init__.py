"""GB300-native moving-least-squares field reconstruction (arXiv:1408.0677, Section 3.3).

The compute path is the CUDA library ``libmls.so`` (sm_103a) behind the C ABI
of ``include/mls.h``; ``_abi`` binds it with ctypes and ``Renderer`` below
marshals torch tensors / numpy arrays into those calls.  PyTorch only
provides device memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import (MLS_P_BF16, MLS_P_FP16, MLS_P_FP32, MLS_P_FP64, MLS_P_FP64_TC, MLS_W_GAUSS, MLS_W_INVDIST,  # noqa: F401
                   MLS_W_WENDLAND, MLS_BATCH_AUTOTUNE, MLS_V_POLY, MLS_V_RIGID, MLS_V_MEAN, MlsBatchStats, MlsDesc, MlsError, MlsStats, MlsView,
                   mls_abi_version, mls_bands, mls_batch_create, mls_batch_destroy, mls_batch_render,
                   mls_batch_sync, mls_create, mls_desc_default, mls_destroy, mls_last_error, mls_render,
                   mls_server_create, mls_server_destroy, mls_server_drain, mls_server_poll, mls_server_submit,
                   mls_sync, MlsRequest, MlsMapDesc, mls_space_map, MLS_MAP_LINES, MLS_MAP_DISCRETE,
                   MLS_MAP_DISCRETE_LINES, MLS_MAP_ADAPTIVE, MLS_MAP_GRADIENT, MLS_MAP_TEXTURE)

PRECISIONS = {"fp64": MLS_P_FP64, "fp32": MLS_P_FP32, "bf16": MLS_P_BF16, "fp16": MLS_P_FP16,
              "fp64tc": MLS_P_FP64_TC}


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


def space_map(field, levels, dims, mode, line_width=1.0, fade=(2.0, 6.0, 3), lo=None, hi=None, texture=None,
              out=None, stream=None):
    """Space mapping of Section 3.4 (``mls_space_map``): field (D, H, W)
    float32/float64 CUDA tensor, levels (D, L) host array, dims one or two
    plane indices, mode an MLS_MAP_* code; texture (Th, Tw, 4) uint8 CUDA
    tensor for MLS_MAP_TEXTURE.  Returns (H, W, 4) uint8 on the device."""
    import torch

    if not field.is_cuda or field.dtype not in (torch.float32, torch.float64) or field.dim() != 3:
        raise ValueError("field must be a (D, H, W) float32 or float64 CUDA tensor")
    field = field.contiguous()
    D, H, W = field.shape
    dims = list(dims)
    lev = np.ascontiguousarray(levels, dtype=np.float64).reshape(D, -1)
    if out is None:
        out = torch.empty((H, W, 4), dtype=torch.uint8, device=field.device)
    d = MlsMapDesc()
    d.mode, d.ndim = int(mode), len(dims)
    for k, x in enumerate(dims):
        d.dim[k] = int(x)
    d.line_width = float(line_width)
    d.fade_lo, d.fade_hi, d.sublevels = float(fade[0]), float(fade[1]), int(fade[2])
    lo = lo if lo is not None else [0.0] * len(dims)
    hi = hi if hi is not None else [1.0] * len(dims)
    for k in range(len(dims)):
        d.lo[k], d.hi[k] = float(lo[k]), float(hi[k])
    if texture is not None:
        texture = texture.contiguous()
        d.texture = texture.data_ptr()
        d.tex_h, d.tex_w = int(texture.shape[0]), int(texture.shape[1])
    mls_space_map(d, D, W, H, field.data_ptr(), field.dtype == torch.float64, lev.ctypes.data, lev.shape[1],
                  out.data_ptr(), _stream_ptr(stream))
    return out


def _check_host_out(name, a, shape, dtype):
    """A caller-supplied host output: a C-contiguous numpy array of exactly
    this shape and type, or None."""
    if a is None:
        return
    if not isinstance(a, np.ndarray):
        raise ValueError(f"{name} must be a numpy array")
    if a.shape != tuple(shape) or a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"] \
            or not a.flags["WRITEABLE"]:
        raise ValueError(f"{name} must be a writeable C-contiguous {np.dtype(dtype).name} array of shape "
                         f"{tuple(shape)}, got {a.dtype.name} {a.shape}"
                         f"{'' if a.flags['C_CONTIGUOUS'] else ' (not contiguous)'}")


def _check_dev_out(name, t, shape, dtype):
    """A caller-supplied device output: a contiguous CUDA tensor of exactly
    this shape and type, or None."""
    if t is None:
        return
    if not getattr(t, "is_cuda", False) or tuple(t.shape) != tuple(shape) or t.dtype != dtype \
            or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype} and shape {tuple(shape)}, "
                         f"got {getattr(t, 'dtype', type(t))} {tuple(getattr(t, 'shape', ()))}")


class Renderer:
    """A resident point set and its MLS description (one ``mls_handle``).

    xy: (n, 2) float64, F: (n, D) float64 -- CUDA torch tensors (read on the
    stream) or host numpy arrays (copied).  ``render`` returns CUDA tensors.
    """

    def __init__(self, xy, F, degree=1, weight=MLS_W_GAUSS, h=0.05, precision="fp32", alpha=1.0,
                 cond_fp64=None, rcond_degenerate=None, cond_recompute=None, weight_split=None, stream=None,
                 variant=0, support=0.0):
        import torch
        self.torch = torch
        d = mls_desc_default()
        on_device = isinstance(xy, torch.Tensor) and xy.is_cuda
        if on_device:
            xy = xy.to(torch.float64).contiguous()
            F = F.to(torch.float64).contiguous()
            if F.dim() == 1:
                F = F[:, None]
            n, D = F.shape
            xy_ptr, F_ptr = xy.data_ptr(), F.data_ptr()
            self._keep = (xy, F)
        else:
            xy = np.ascontiguousarray(xy, dtype=np.float64)
            F = np.ascontiguousarray(F, dtype=np.float64)
            if F.ndim == 1:
                F = F[:, None]
            n, D = F.shape
            xy_ptr, F_ptr = xy.ctypes.data, F.ctypes.data
            self._keep = (xy, F)
        d.n, d.D, d.degree, d.weight, d.h, d.alpha = n, D, degree, weight, h, alpha
        d.precision = PRECISIONS.get(precision, precision)
        if cond_fp64 is not None:
            d.cond_fp64 = cond_fp64
        if rcond_degenerate is not None:
            d.rcond_degenerate = rcond_degenerate
        if cond_recompute is not None:
            d.cond_recompute = cond_recompute
        if weight_split is not None:
            d.weight_split = int(weight_split)
        d.variant = int(variant)
        d.support = float(support)
        self.desc = d
        self.n, self.D = n, D
        self.stream = _stream_ptr(stream)
        self.handle = mls_create(d, xy_ptr, F_ptr, on_device, self.stream)

    @property
    def field_dtype(self):
        return self.torch.float64 if self.desc.precision in (MLS_P_FP64, MLS_P_FP64_TC) else self.torch.float32

    def render(self, W, H, view=(0.0, 0.0, 1.0, 1.0), levels=None, status=True, field=None, bands=None,
               status_out=None):
        torch = self.torch
        dev = torch.device("cuda", torch.cuda.current_device())
        _check_dev_out("field", field, (self.D, H, W), self.field_dtype)
        _check_dev_out("status_out", status_out, (H, W), torch.uint8)
        _check_dev_out("bands", bands, (self.D, H, W), torch.uint8)
        if field is None:
            field = torch.empty((self.D, H, W), dtype=self.field_dtype, device=dev)
        st = status_out
        if status and st is None:
            st = torch.empty((H, W), dtype=torch.uint8, device=dev)
        lev = None
        L = 0
        if levels is not None:
            lev = np.ascontiguousarray(levels, dtype=np.float64)
            L = lev.shape[1]
            if bands is None:
                bands = torch.empty((self.D, H, W), dtype=torch.uint8, device=dev)
        v = MlsView(W, H, *view)
        mls_render(self.handle, v, field.data_ptr(), st.data_ptr() if st is not None else 0,
                   lev.ctypes.data if lev is not None else 0, L,
                   bands.data_ptr() if (bands is not None and lev is not None) else 0, True, self.stream)
        return {"field": field, "status": st, "bands": bands if lev is not None else None}

    def render_host(self, W, H, view=(0.0, 0.0, 1.0, 1.0), levels=None, status=True, field=None, bands=None,
                    status_out=None):
        """Same as render, with host (numpy) outputs; returns after the copy-back.
        Supplied outputs must be C-contiguous numpy arrays of exactly the
        rendered shape and type (the library writes page-locked ones from the
        kernels and cannot check them itself)."""
        dt = np.float64 if self.desc.precision in (MLS_P_FP64, MLS_P_FP64_TC) else np.float32
        _check_host_out("field", field, (self.D, H, W), dt)
        _check_host_out("status_out", status_out, (H, W), np.uint8)
        _check_host_out("bands", bands, (self.D, H, W), np.uint8)
        if field is None:
            field = np.empty((self.D, H, W), dtype=dt)
        st = status_out if status_out is not None else (np.empty((H, W), np.uint8) if status else None)
        lev = None
        L = 0
        if levels is not None:
            lev = np.ascontiguousarray(levels, dtype=np.float64)
            L = lev.shape[1]
            if bands is None:
                bands = np.empty((self.D, H, W), np.uint8)
        v = MlsView(W, H, *view)
        mls_render(self.handle, v, field.ctypes.data, st.ctypes.data if st is not None else 0,
                   lev.ctypes.data if lev is not None else 0, L,
                   bands.ctypes.data if (bands is not None and lev is not None) else 0, False, self.stream)
        return {"field": field, "status": st, "bands": bands if lev is not None else None}

    def bands(self, field, levels, W, H, view=(0.0, 0.0, 1.0, 1.0), out=None):
        torch = self.torch
        lev = np.ascontiguousarray(levels, dtype=np.float64)
        if out is None:
            out = torch.empty((self.D, H, W), dtype=torch.uint8, device=field.device)
        mls_bands(self.handle, MlsView(W, H, *view), field.data_ptr(), lev.ctypes.data, lev.shape[1],
                  out.data_ptr(), True, self.stream)
        return out

    def sync(self, timeout_s=60.0) -> MlsStats:
        return mls_sync(self.handle, timeout_s)

    def close(self):
        if getattr(self, "handle", None):
            mls_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many resident datasets (``Renderer`` objects) rendered by one CUDA graph
    (``mls_batch_*``).  ``render`` takes one (W, H, view, levels) entry per
    dataset and returns one output dict per dataset; the outputs are reused by
    later calls with the same shapes, so the captured graph is replayed."""

    def __init__(self, renderers, autotune=False, stream=None):
        import torch
        self.torch = torch
        self.renderers = list(renderers)
        self.stream = _stream_ptr(stream)
        self.handle = mls_batch_create([r.handle for r in self.renderers],
                                       MLS_BATCH_AUTOTUNE if autotune else 0)
        self._out = None
        self._key = None

    def render(self, entries, status=True):
        """entries: list of (W, H, view, levels or None)."""
        torch = self.torch
        n = len(self.renderers)
        assert len(entries) == n
        key = tuple((W, H, tuple(view), None if lev is None else np.asarray(lev).shape)
                    for (W, H, view, lev) in entries)
        dev = torch.device("cuda", torch.cuda.current_device())
        if key != self._key:
            outs = []
            for r, (W, H, view, lev) in zip(self.renderers, entries):
                o = {"field": torch.empty((r.D, H, W), dtype=r.field_dtype, device=dev),
                     "status": torch.empty((H, W), dtype=torch.uint8, device=dev) if status else None,
                     "bands": torch.empty((r.D, H, W), dtype=torch.uint8, device=dev) if lev is not None else None}
                outs.append(o)
            self._out, self._key = outs, key
        outs = self._out
        views = (MlsView * n)(*[MlsView(W, H, *view) for (W, H, view, _) in entries])
        P = ctypes.c_void_p
        fields = (P * n)(*[o["field"].data_ptr() for o in outs])
        sts = (P * n)(*[o["status"].data_ptr() if o["status"] is not None else None for o in outs])
        levs = [None if lev is None else np.ascontiguousarray(lev, dtype=np.float64) for (_, _, _, lev) in entries]
        self._levs = levs
        lev_p = (P * n)(*[lv.ctypes.data if lv is not None else None for lv in levs])
        Ls = (ctypes.c_int32 * n)(*[lv.shape[1] if lv is not None else 0 for lv in levs])
        bnd = (P * n)(*[o["bands"].data_ptr() if o["bands"] is not None else None for o in outs])
        mls_batch_render(self.handle, views, fields, sts, lev_p, Ls, bnd, self.stream)
        return outs

    def sync(self, timeout_s=120.0) -> MlsBatchStats:
        return mls_batch_sync(self.handle, timeout_s)

    def close(self):
        if getattr(self, "handle", None):
            mls_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Request:
    """One submitted render request: its id, host outputs (page-locked) and,
    once polled, its completion record."""

    def __init__(self, rid, bands, status, field, keep):
        self.id, self.bands, self.status, self.field = rid, bands, status, field
        self._keep = keep
        self.done = None


class Server:
    """Continuous-batching render server over resident datasets
    (``mls_server_*``): requests are admitted into ``slots`` stream slots
    while the requests in flight hold less than ``mem_budget`` device bytes;
    ``submit`` returns at once, ``poll`` collects completions."""

    def __init__(self, slots=4, mem_budget=4 << 30):
        import torch
        self.torch = torch
        self.handle = mls_server_create(slots, mem_budget)
        self.pending = {}

    def submit(self, renderer, W, H, view=(0.0, 0.0, 1.0, 1.0), levels=None, field=False, status=True):
        torch = self.torch
        D = renderer.D
        lev = None if levels is None else np.ascontiguousarray(levels, dtype=np.float64)
        bands = torch.empty((D, H, W), dtype=torch.uint8).pin_memory() if lev is not None else None
        st = torch.empty((H, W), dtype=torch.uint8).pin_memory() if status else None
        fdt = torch.float64 if renderer.desc.precision in (MLS_P_FP64, MLS_P_FP64_TC) else torch.float32
        fld = torch.empty((D, H, W), dtype=fdt).pin_memory() if field else None
        req = MlsRequest(renderer.handle, MlsView(W, H, *view), lev.ctypes.data if lev is not None else None,
                         lev.shape[1] if lev is not None else 0, 0,
                         bands.data_ptr() if bands is not None else None, st.data_ptr() if st is not None else None,
                         fld.data_ptr() if fld is not None else None)
        rid = mls_server_submit(self.handle, req)
        r = Request(rid, bands, st, fld, (lev, renderer))
        self.pending[rid] = r
        return r

    def poll(self):
        out = []
        for d in mls_server_poll(self.handle):
            r = self.pending.pop(d.id, None)
            if r is not None:
                r.done = d
                out.append(r)
        return out

    def drain(self, timeout_s=300.0):
        return mls_server_drain(self.handle, timeout_s)

    def close(self):
        if getattr(self, "handle", None):
            mls_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
