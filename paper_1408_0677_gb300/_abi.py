"""ctypes binding of the C ABI declared in include/mls.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  The library
is the in-tree ``_build/libmls.so``; if it is missing the first call raises,
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

MLS_OK, MLS_E_INVAL, MLS_E_NOMEM, MLS_E_CUDA, MLS_E_TIMEOUT, MLS_E_UNSUPPORTED = range(6)
MLS_W_GAUSS, MLS_W_WENDLAND, MLS_W_INVDIST = range(3)
MLS_P_FP64, MLS_P_FP32, MLS_P_BF16, MLS_P_FP16, MLS_P_FP64_TC = range(5)
MLS_ST_DEGREE_MASK = 0x03
MLS_ST_NO_SUPPORT = 0x04
MLS_ST_FP64_SOLVE = 0x08
MLS_ST_RECOMPUTED = 0x10
MLS_ST_DEGRADED = 0x20
MLS_ST_COINCIDENT = 0x40

STATUS_NAMES = {MLS_OK: "MLS_OK", MLS_E_INVAL: "MLS_E_INVAL", MLS_E_NOMEM: "MLS_E_NOMEM",
                MLS_E_CUDA: "MLS_E_CUDA", MLS_E_TIMEOUT: "MLS_E_TIMEOUT",
                MLS_E_UNSUPPORTED: "MLS_E_UNSUPPORTED"}


class MlsDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("D", ctypes.c_int32), ("degree", ctypes.c_int32),
                ("weight", ctypes.c_int32), ("precision", ctypes.c_int32), ("h", ctypes.c_double),
                ("alpha", ctypes.c_double), ("cond_fp64", ctypes.c_double),
                ("rcond_degenerate", ctypes.c_double), ("cond_recompute", ctypes.c_double),
                ("weight_split", ctypes.c_int32), ("variant", ctypes.c_int32), ("support", ctypes.c_double)]


class MlsView(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double), ("x1", ctypes.c_double), ("y1", ctypes.c_double)]


class MlsStats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int64), ("recomputed", ctypes.c_int64), ("recomputed_fp64", ctypes.c_int64),
                ("device_error", ctypes.c_int64), ("launches", ctypes.c_int64), ("last_render_ms", ctypes.c_double),
                ("main_kernel_ms", ctypes.c_double), ("retried_tiles", ctypes.c_int64),
                ("main_path", ctypes.c_int32), ("reserved", ctypes.c_int32)]


MLS_PATH_NONE, MLS_PATH_TENSOR, MLS_PATH_FP32, MLS_PATH_FP64, MLS_PATH_VARIANT, MLS_PATH_FP64_TC = 0, 1, 2, 3, 4, 5


class MlsBatchStats(ctypes.Structure):
    _fields_ = [("datasets", ctypes.c_int64), ("pairs", ctypes.c_int64), ("recomputed", ctypes.c_int64),
                ("device_error", ctypes.c_int64), ("launches", ctypes.c_int64), ("captures", ctypes.c_int64),
                ("replays", ctypes.c_int64), ("last_render_ms", ctypes.c_double)]


MLS_BATCH_AUTOTUNE = 1
MLS_V_POLY, MLS_V_RIGID, MLS_V_MEAN = 0, 1, 2
(MLS_MAP_LINES, MLS_MAP_DISCRETE, MLS_MAP_DISCRETE_LINES, MLS_MAP_ADAPTIVE, MLS_MAP_GRADIENT,
 MLS_MAP_TEXTURE) = range(6)


class MlsServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("reserved", ctypes.c_int32), ("mem_budget", ctypes.c_int64)]


class MlsRequest(ctypes.Structure):
    _fields_ = [("dataset", ctypes.c_void_p), ("view", MlsView), ("levels", ctypes.c_void_p), ("L", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("bands", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("field", ctypes.c_void_p)]


class MlsRequestDone(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("latency_ms", ctypes.c_double), ("queued_ms", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("footprint", ctypes.c_int64)]


class MlsServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("peak_inflight", ctypes.c_int64), ("peak_bytes", ctypes.c_int64)]


class MlsMapDesc(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("ndim", ctypes.c_int32), ("dim", ctypes.c_int32 * 2),
                ("line_width", ctypes.c_float), ("fade_lo", ctypes.c_float), ("fade_hi", ctypes.c_float),
                ("sublevels", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
                ("texture", ctypes.c_void_p), ("tex_w", ctypes.c_int32), ("tex_h", ctypes.c_int32)]


class MlsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
P = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Open libmls.so (built in-tree by paper_1408_0677_gb300.build), or the
    in-tree variant named by the environment variable MLS_LIBRARY (the
    checked or sanitized build)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    default = path is None
    path = path or os.environ.get("MLS_LIBRARY") or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_1408_0677_gb300.build.build())")
    lib = ctypes.CDLL(path)
    lib.mls_abi_version.restype = ctypes.c_int32
    lib.mls_abi_version.argtypes = []
    lib.mls_last_error.restype = ctypes.c_char_p
    lib.mls_last_error.argtypes = []
    lib.mls_desc_default.restype = ctypes.c_int
    lib.mls_desc_default.argtypes = [ctypes.POINTER(MlsDesc)]
    lib.mls_create.restype = ctypes.c_int
    lib.mls_create.argtypes = [ctypes.POINTER(MlsDesc), P, P, ctypes.c_int32, P, ctypes.POINTER(P)]
    lib.mls_render.restype = ctypes.c_int
    lib.mls_render.argtypes = [P, ctypes.POINTER(MlsView), P, P, P, ctypes.c_int32, P, ctypes.c_int32, P]
    lib.mls_bands.restype = ctypes.c_int
    lib.mls_bands.argtypes = [P, ctypes.POINTER(MlsView), P, P, ctypes.c_int32, P, ctypes.c_int32, P]
    lib.mls_sync.restype = ctypes.c_int
    lib.mls_sync.argtypes = [P, ctypes.c_double, ctypes.POINTER(MlsStats)]
    lib.mls_destroy.restype = ctypes.c_int
    lib.mls_destroy.argtypes = [P]
    lib.mls_batch_create.restype = ctypes.c_int
    lib.mls_batch_create.argtypes = [ctypes.c_int32, P, ctypes.c_int32, ctypes.POINTER(P)]
    lib.mls_batch_render.restype = ctypes.c_int
    lib.mls_batch_render.argtypes = [P, P, P, P, P, P, P, P]
    lib.mls_batch_sync.restype = ctypes.c_int
    lib.mls_batch_sync.argtypes = [P, ctypes.c_double, ctypes.POINTER(MlsBatchStats)]
    lib.mls_batch_destroy.restype = ctypes.c_int
    lib.mls_batch_destroy.argtypes = [P]
    lib.mls_server_create.restype = ctypes.c_int
    lib.mls_server_create.argtypes = [ctypes.POINTER(MlsServerConfig), ctypes.POINTER(P)]
    lib.mls_server_submit.restype = ctypes.c_int
    lib.mls_server_submit.argtypes = [P, ctypes.POINTER(MlsRequest), ctypes.POINTER(ctypes.c_int64)]
    lib.mls_server_poll.restype = ctypes.c_int
    lib.mls_server_poll.argtypes = [P, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    lib.mls_server_drain.restype = ctypes.c_int
    lib.mls_server_drain.argtypes = [P, ctypes.c_double, ctypes.POINTER(MlsServerStats)]
    lib.mls_server_destroy.restype = ctypes.c_int
    lib.mls_server_destroy.argtypes = [P]
    lib.mls_bands_noalloc.restype = ctypes.c_int
    lib.mls_bands_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32, P,
                                      ctypes.c_int32, P, P]
    lib.mls_space_map.restype = ctypes.c_int
    lib.mls_space_map.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32, P,
                                  ctypes.c_int32, P, P]
    # test hooks (include/mls_debug.h)
    lib.mls_debug_wait_selftest.restype = ctypes.c_int
    lib.mls_debug_wait_selftest.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
    lib.mls_debug_operand_cut.restype = ctypes.c_int
    lib.mls_debug_operand_cut.argtypes = [P, ctypes.c_int32]
    lib.mls_debug_handover_split.restype = ctypes.c_int
    lib.mls_debug_handover_split.argtypes = [P, ctypes.c_int64, ctypes.c_int64]
    lib.mls_debug_host_output.restype = ctypes.c_int
    lib.mls_debug_host_output.argtypes = [P, ctypes.c_int32]
    lib.mls_debug_df_weight.restype = ctypes.c_int
    lib.mls_debug_df_weight.argtypes = [ctypes.c_int, P, P, ctypes.c_int64, P]
    if default:
        _lib = lib
    return lib


def _check(st: int, where: str):
    if st != MLS_OK:
        raise MlsError(st, where, mls_last_error())


def mls_abi_version() -> int:
    return load().mls_abi_version()


def mls_last_error() -> str:
    return load().mls_last_error().decode()


def mls_desc_default() -> MlsDesc:
    d = MlsDesc()
    _check(load().mls_desc_default(ctypes.byref(d)), "mls_desc_default")
    return d


def mls_create(desc: MlsDesc, xy_ptr: int, F_ptr: int, on_device: bool, stream: int = 0) -> int:
    h = P()
    _check(load().mls_create(ctypes.byref(desc), P(xy_ptr), P(F_ptr), int(bool(on_device)), P(stream),
                             ctypes.byref(h)), "mls_create")
    return h.value


def mls_render(handle: int, view: MlsView, field_ptr: int, status_ptr: int = 0, levels_ptr: int = 0,
               L: int = 0, bands_ptr: int = 0, on_device: bool = True, stream: int = 0):
    _check(load().mls_render(P(handle), ctypes.byref(view), P(field_ptr), P(status_ptr or None),
                             P(levels_ptr or None), int(L), P(bands_ptr or None), int(bool(on_device)),
                             P(stream)), "mls_render")


def mls_bands(handle: int, view: MlsView, field_ptr: int, levels_ptr: int, L: int, bands_ptr: int,
              on_device: bool = True, stream: int = 0):
    _check(load().mls_bands(P(handle), ctypes.byref(view), P(field_ptr), P(levels_ptr or None), int(L),
                            P(bands_ptr), int(bool(on_device)), P(stream)), "mls_bands")


def mls_bands_noalloc(D: int, W: int, H: int, field_ptr: int, field_fp64: bool, levels_ptr: int, L: int,
                      bands_ptr: int, stream: int = 0):
    """Iso-band labels into caller buffers, without any device allocation."""
    _check(load().mls_bands_noalloc(int(D), int(W), int(H), P(field_ptr), int(bool(field_fp64)), P(levels_ptr),
                                    int(L), P(bands_ptr), P(stream)), "mls_bands_noalloc")


def mls_space_map(desc: MlsMapDesc, D: int, W: int, H: int, field_ptr: int, field_fp64: bool, levels_ptr: int,
                  L: int, rgba_ptr: int, stream: int = 0):
    """Space mapping of Section 3.4 into a caller RGBA8 buffer (no allocation)."""
    _check(load().mls_space_map(ctypes.byref(desc), int(D), int(W), int(H), P(field_ptr), int(bool(field_fp64)),
                                P(levels_ptr), int(L), P(rgba_ptr), P(stream)), "mls_space_map")


def mls_batch_create(handles, flags: int = 0) -> int:
    arr = (P * len(handles))(*[P(h) for h in handles])
    out = P()
    _check(load().mls_batch_create(len(handles), ctypes.cast(arr, P), int(flags), ctypes.byref(out)),
           "mls_batch_create")
    return out.value


def mls_batch_render(batch: int, views, fields, status, levels, L, bands, stream: int = 0):
    """views: ctypes array of MlsView; the others ctypes pointer arrays (or None)."""
    _check(load().mls_batch_render(P(batch), ctypes.cast(views, P), ctypes.cast(fields, P),
                                   ctypes.cast(status, P) if status is not None else None,
                                   ctypes.cast(levels, P) if levels is not None else None,
                                   ctypes.cast(L, P) if L is not None else None,
                                   ctypes.cast(bands, P) if bands is not None else None, P(stream)),
           "mls_batch_render")


def mls_batch_sync(batch: int, timeout_s: float = 60.0) -> MlsBatchStats:
    st = MlsBatchStats()
    _check(load().mls_batch_sync(P(batch), float(timeout_s), ctypes.byref(st)), "mls_batch_sync")
    return st


def mls_batch_destroy(batch: int):
    _check(load().mls_batch_destroy(P(batch)), "mls_batch_destroy")


def mls_server_create(slots: int, mem_budget: int) -> int:
    cfg = MlsServerConfig(int(slots), 0, int(mem_budget))
    out = P()
    _check(load().mls_server_create(ctypes.byref(cfg), ctypes.byref(out)), "mls_server_create")
    return out.value


def mls_server_submit(server: int, req: MlsRequest) -> int:
    rid = ctypes.c_int64()
    _check(load().mls_server_submit(P(server), ctypes.byref(req), ctypes.byref(rid)), "mls_server_submit")
    return rid.value


def mls_server_poll(server: int, cap: int = 1024) -> list:
    arr = (MlsRequestDone * cap)()
    n = ctypes.c_int32()
    _check(load().mls_server_poll(P(server), ctypes.cast(arr, P), int(cap), ctypes.byref(n)), "mls_server_poll")
    return [arr[i] for i in range(n.value)]


def mls_server_drain(server: int, timeout_s: float = 120.0) -> MlsServerStats:
    st = MlsServerStats()
    _check(load().mls_server_drain(P(server), float(timeout_s), ctypes.byref(st)), "mls_server_drain")
    return st


def mls_server_destroy(server: int):
    _check(load().mls_server_destroy(P(server)), "mls_server_destroy")


def mls_sync(handle: int, timeout_s: float = 60.0) -> MlsStats:
    s = MlsStats()
    _check(load().mls_sync(P(handle), float(timeout_s), ctypes.byref(s)), "mls_sync")
    return s


def mls_destroy(handle: int):
    _check(load().mls_destroy(P(handle)), "mls_destroy")
