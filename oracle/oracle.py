"""ctypes front end of the FP64 C oracle (test infrastructure, see __init__)."""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mls_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libmls_oracle.so")
_lib = None

GAUSS, WENDLAND, INVDIST = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile mls_oracle.c into a shared object (gcc, OpenMP, no FP contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """Open a compiled oracle (the default build, or a test's planted-mistake variant)."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.oracle_mls.restype = ctypes.c_int
    lib.oracle_mls.argtypes = [ctypes.c_int64, ctypes.c_int32, P, P, ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_int64, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               P, P, P, P, P, P, P, P, ctypes.c_int32]
    lib.oracle_bands.restype = ctypes.c_int
    lib.oracle_bands.argtypes = [ctypes.c_int64, ctypes.c_int32, P, P, ctypes.c_int32, P]
    lib.oracle_mls_variant.restype = ctypes.c_int
    lib.oracle_mls_variant.argtypes = [ctypes.c_int64, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int64, P, P,
                                       P, ctypes.c_int32]
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = load_library(_LIB)
    return _lib


@dataclass
class OracleResult:
    field: np.ndarray     # (npix, D) float64
    deg_used: np.ndarray  # (npix,) int8, -1 = no support
    rcond: np.ndarray     # (npix,) float64
    count: np.ndarray     # (npix,) int64
    mstab: np.ndarray     # (npix,) float64
    amb: np.ndarray       # (npix,) uint8 ambiguity bits
    # first-order rounding-error bound coefficients of each value (npix, D),
    # only with ebound=True: an FP64 evaluation of the same fit whose longest
    # summation chain has N terms is within (N + 12) u ecoef_sum + ecoef_fix
    # of the exact value (u = 2^-53; see oracle_mls in mls_oracle.c)
    ecoef_sum: np.ndarray = None
    ecoef_fix: np.ndarray = None


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def mls(xy, F, degree, weight, h, W, H, view=(0.0, 0.0, 1.0, 1.0), pixels=None, alpha=1.0,
        rcond_min=1e-12, amb_factor=100.0, amb_boundary=1e-6, threads=0, lib=None, trunc=0.0,
        ebound=False) -> OracleResult:
    """Evaluate the FP64 MLS fit at the listed pixels (all pixels if None).
    trunc = c > 0 (Gaussian only): the truncated Gaussian, zero outside the
    box |dx|, |dy| < c h around each pixel.  ebound=True also returns the
    rounding-error bound coefficients (OracleResult.ecoef_sum / ecoef_fix)."""
    lib = lib or _load()
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    if F.ndim == 1:
        F = F[:, None]
    n, D = F.shape
    assert xy.shape == (n, 2)
    if pixels is None:
        npix = W * H
        pix_arr = None
    else:
        pix_arr = np.ascontiguousarray(pixels, dtype=np.int64)
        npix = pix_arr.size
    field = np.empty((npix, D), np.float64)
    deg = np.empty(npix, np.int8)
    rc = np.empty(npix, np.float64)
    cnt = np.empty(npix, np.int64)
    ms = np.empty(npix, np.float64)
    amb = np.empty(npix, np.uint8)
    es = np.empty((npix, D), np.float64) if ebound else None
    ef = np.empty((npix, D), np.float64) if ebound else None
    x0, y0, x1, y1 = view
    rcode = lib.oracle_mls(n, D, _p(xy), _p(F), degree, weight, h, alpha, float(trunc), W, H, x0, y0, x1, y1,
                           npix, _p(pix_arr) if pix_arr is not None else None, rcond_min,
                           amb_factor, amb_boundary, _p(field), _p(deg), _p(rc), _p(cnt), _p(ms),
                           _p(amb), _p(es) if ebound else None, _p(ef) if ebound else None, threads)
    if rcode != 0:
        raise ValueError("oracle_mls rejected its arguments")
    return OracleResult(field, deg, rc, cnt, ms, amb, es, ef)


def bands(field, levels, lib=None) -> np.ndarray:
    """Iso-band labels (npix, D) uint8 for a (npix, D) field and (D, L) levels."""
    lib = lib or _load()
    field = np.ascontiguousarray(field, dtype=np.float64)
    levels = np.ascontiguousarray(levels, dtype=np.float64)
    npix, D = field.shape
    L = levels.shape[1]
    out = np.empty((npix, D), np.uint8)
    if lib.oracle_bands(npix, D, _p(field), _p(levels), L, _p(out)) != 0:
        raise ValueError("oracle_bands rejected its arguments")
    return out


VARIANT_RIGID = 1
VARIANT_MEAN = 2


def mls_variant(xy, Q, variant, weight, h, W, H, view=(0.0, 0.0, 1.0, 1.0), pixels=None, alpha=1.0, threads=0,
                lib=None, aux=False, trunc=0.0):
    """The paper's rigid (variant 1, Eqs. eq-rigidmls / eq-rigidmlspartial) or
    mean-displacement (variant 2, Eq. eq-meanmls) mapping of 2-D values Q at
    the listed pixels (all if None): (npix, 2) float64, NaN without support.
    With aux=True also (npix, 4): q*_x, q*_y, |v - p*| and the rotation's
    conditioning kappa (see oracle_mls_variant)."""
    lib = lib or _load()
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    n = xy.shape[0]
    assert Q.shape == (n, 2)
    if pixels is None:
        npix, pix_arr = W * H, None
    else:
        pix_arr = np.ascontiguousarray(pixels, dtype=np.int64)
        npix = pix_arr.size
    field = np.empty((npix, 2), np.float64)
    ax = np.empty((npix, 4), np.float64) if aux else None
    x0, y0, x1, y1 = view
    rc = lib.oracle_mls_variant(n, _p(xy), _p(Q), int(variant), int(weight), float(h), float(alpha), float(trunc),
                                W, H, x0, y0,
                                x1, y1, npix, _p(pix_arr) if pix_arr is not None else None, _p(field),
                                _p(ax) if aux else None, threads)
    if rc != 0:
        raise ValueError("oracle_mls_variant rejected its arguments")
    return (field, ax) if aux else field
