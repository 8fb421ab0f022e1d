"""Seeded synthetic workloads for the MLS field reconstruction.

This module only draws inputs: point positions, data values, iso-levels and
view rectangles.  It holds none of the method's arithmetic, so both the CUDA
path and the FP64 oracle can consume exactly the same arrays.

The workloads stand in for the paper's datasets (Section 4: the wine data of
Section 4.3 has 178 samples and 13 dimensions; Table 1 uses unnamed datasets of
306, 1000 and 2245 points on a 600x600 canvas).  None of those datasets is
reproduced: every array below is drawn from a seeded ``numpy`` generator with
the shapes and distributions stated in each function.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Weight kinds, basis degrees and precision modes share their integer codes
# with the C header (include/mls.h).
WEIGHT_GAUSS = 0
WEIGHT_WENDLAND = 1
WEIGHT_INVDIST = 2


@dataclass
class Workload:
    """One MLS problem: points, values, kernel, view and iso-levels."""

    name: str
    xy: np.ndarray           # (n, 2) float64 point positions
    F: np.ndarray            # (n, D) float64 data values
    degree: int              # basis degree 0, 1 or 2
    weight: int              # WEIGHT_* code
    h: float                 # Gaussian h, Wendland support radius, or IDW basis scale
    W: int
    H: int
    view: tuple = (0.0, 0.0, 1.0, 1.0)   # x0, y0, x1, y1
    levels: np.ndarray = field(default=None)  # (D, L) float64 ascending
    alpha: float = 1.0       # IDW exponent (paper's Eq. eq-weights)
    trunc: float = 0.0       # truncated Gaussian: box half-width in units of h (0: full sum)

    @property
    def n(self) -> int:
        return int(self.xy.shape[0])

    @property
    def D(self) -> int:
        return int(self.F.shape[1])


def _clusters(rng, n, centres, sigmas, weights=None, resample=True):
    """Isotropic Gaussian clusters in [0,1]^2; points outside are redrawn."""
    k = len(centres)
    if weights is None:
        # equal membership: sizes differ by at most one
        sizes = np.full(k, n // k)
        sizes[: n % k] += 1
    else:
        sizes = rng.multinomial(n, weights)
    out = []
    for c, s, m in zip(centres, sigmas, sizes):
        pts = c + s * rng.standard_normal((m, 2))
        if resample:
            bad = np.any((pts < 0) | (pts > 1), axis=1)
            while bad.any():
                pts[bad] = c + s * rng.standard_normal((int(bad.sum()), 2))
                bad = np.any((pts < 0) | (pts > 1), axis=1)
        out.append(pts)
    return np.concatenate(out, axis=0)


def _fourier_fields(rng, xy, D, modes, max_freq):
    """D smooth random fields, each a sum of `modes` plane cosines."""
    n = xy.shape[0]
    F = np.zeros((n, D))
    for d in range(D):
        omega = rng.integers(-max_freq, max_freq + 1, size=(modes, 2))
        amp = rng.standard_normal(modes) / np.sqrt(modes)
        phase = rng.uniform(0, 2 * np.pi, size=modes)
        F[:, d] = (amp[None, :] * np.cos(2 * np.pi * (xy @ omega.T) + phase[None, :])).sum(1)
    return F


def default_levels(F: np.ndarray, L: int) -> np.ndarray:
    """L equally spaced iso-levels strictly inside each dimension's data range.

    t_{d,j} = lo_d + j (hi_d - lo_d) / (L + 1), j = 1..L, lo/hi the data
    min/max of dimension d over the points (Section 3.4 leaves the placement
    of the iso-levels open; this is the reading used throughout).
    """
    lo = F.min(axis=0)
    hi = F.max(axis=0)
    j = np.arange(1, L + 1, dtype=np.float64)
    return lo[:, None] + j[None, :] * ((hi - lo)[:, None] / (L + 1))


def wine_shaped(seed: int = 1001) -> Workload:
    """n=178, D=13, three isotropic clusters (sigma 0.08), 256x256, linear basis,
    Gaussian h=0.05, 10 iso-levels.  Shape of the wine data of Section 4.3."""
    rng = np.random.default_rng(seed)
    n, D = 178, 13
    centres = rng.uniform(0.2, 0.8, size=(3, 2))
    xy = _clusters(rng, n, centres, [0.08] * 3)
    F = np.zeros((n, D))
    for d in range(D):
        k = rng.integers(-3, 4, size=2)
        l = rng.integers(-3, 4, size=2)
        a, b = rng.uniform(0.5, 1.5, size=2)
        phi, psi = rng.uniform(0, 2 * np.pi, size=2)
        F[:, d] = a * np.sin(2 * np.pi * (xy @ k) + phi) + b * np.cos(2 * np.pi * (xy @ l) + psi)
    F += rng.normal(0.0, 0.05, size=F.shape)
    w = Workload("wine_shaped_n178_d13_256sq_linear_gauss", xy, F, 1, WEIGHT_GAUSS, 0.05, 256, 256)
    w.levels = default_levels(F, 10)
    return w


def fourier_10k(seed: int = 1002, W: int = 1024, H: int = 1024) -> Workload:
    """n=10,000 points (8 Gaussian clusters, sigma U(0.02,0.06), plus 20% uniform),
    D=32 random Fourier fields (8 modes), 1024x1024, quadratic basis,
    Gaussian h=0.02 full sum, 16 iso-levels."""
    rng = np.random.default_rng(seed)
    n, D = 10_000, 32
    n_uni = n // 5
    centres = rng.uniform(0.1, 0.9, size=(8, 2))
    sig = rng.uniform(0.02, 0.06, size=8)
    xy = np.concatenate([_clusters(rng, n - n_uni, centres, sig),
                         rng.uniform(0.0, 1.0, size=(n_uni, 2))], axis=0)
    xy = xy[rng.permutation(n)]
    F = _fourier_fields(rng, xy, D, modes=8, max_freq=4)
    w = Workload("fourier_n10k_d32_1024sq_quadratic_gauss", xy, F, 2, WEIGHT_GAUSS, 0.02, W, H)
    w.levels = default_levels(F, 16)
    return w


def clusters_200k(seed: int = 1003, W: int = 2048, H: int = 2048) -> Workload:
    """n=200,000 points in 64 clusters (sigma U(0.01,0.05)), D=64 Fourier fields,
    2048x2048, quadratic basis, Wendland C2 support radius 0.015, 16 iso-levels."""
    rng = np.random.default_rng(seed)
    n, D = 200_000, 64
    centres = rng.uniform(0.1, 0.9, size=(64, 2))
    sig = rng.uniform(0.01, 0.05, size=64)
    xy = _clusters(rng, n, centres, sig)
    xy = xy[rng.permutation(n)]
    F = _fourier_fields(rng, xy, D, modes=8, max_freq=4)
    w = Workload("clusters_n200k_d64_2048sq_quadratic_wendland", xy, F, 2, WEIGHT_WENDLAND, 0.015, W, H)
    w.levels = default_levels(F, 16)
    return w


def fourier_mix(seed: int, n: int, D: int, W: int, H: int, degree: int, weight: int, h: float,
                L: int = 16) -> Workload:
    """Scaled-down workload with the structure of the 10k-point configuration:
    8 Gaussian clusters (sigma U(0.02,0.06)) plus 20% uniform points, D random
    Fourier fields with 8 modes of integer frequency up to 4."""
    rng = np.random.default_rng(seed)
    n_uni = n // 5
    centres = rng.uniform(0.1, 0.9, size=(8, 2))
    sig = rng.uniform(0.02, 0.06, size=8)
    xy = np.concatenate([_clusters(rng, n - n_uni, centres, sig),
                         rng.uniform(0.0, 1.0, size=(n_uni, 2))], axis=0)
    xy = xy[rng.permutation(n)]
    F = _fourier_fields(rng, xy, D, modes=8, max_freq=4)
    w = Workload(f"fourier_mix_n{n}_d{D}_{W}x{H}_deg{degree}_w{weight}", xy, F, degree, weight, h, W, H)
    w.levels = default_levels(F, L)
    return w


def heldout(seed: int) -> tuple:
    """A randomly shaped case drawn from a wider family than the workloads
    above, for parity checks on inputs that no threshold was tuned on.

    Gaussian (two thirds) or Wendland weight; 3-16 clusters (sigma
    U(0.01, 0.06)) plus 0-30% uniform points; n log-uniform in 2k-40k
    (Gaussian) or 20k-150k (Wendland); D uniform in 3-40; linear or quadratic
    basis; h U(0.012, 0.035) (Gaussian) or radius U(0.01, 0.03); fields with
    3-12 modes of integer frequency up to between 2 and 1/(6 h) (wavelength
    at least 6 h); a zoom window of side log-uniform in [1/16, 1] at a random
    place in [0,1]^2, with pixels of 0.08-0.3 h (at most 1024 columns) and a
    height of 0.6-1 times the width; 8-20 iso-levels.

    Returns (workload, sampled pixel indices): 2048 random pixels plus one
    dense 24 x 24 window."""
    rng = np.random.default_rng(seed)
    gauss = rng.random() < 2.0 / 3.0
    if gauss:
        n = int(round(np.exp(rng.uniform(np.log(2000), np.log(40000)))))
        h = float(rng.uniform(0.012, 0.035))
    else:
        n = int(round(np.exp(rng.uniform(np.log(20000), np.log(150000)))))
        h = float(rng.uniform(0.01, 0.03))
    D = int(rng.integers(3, 41))
    degree = int(rng.integers(1, 3))
    k = int(rng.integers(3, 17))
    n_uni = int(n * rng.uniform(0.0, 0.3))
    centres = rng.uniform(0.1, 0.9, size=(k, 2))
    sig = rng.uniform(0.01, 0.06, size=k)
    xy = np.concatenate([_clusters(rng, n - n_uni, centres, sig),
                         rng.uniform(0.0, 1.0, size=(n_uni, 2))], axis=0)
    xy = xy[rng.permutation(n)]
    modes = int(rng.integers(3, 13))
    max_freq = int(rng.integers(2, max(3, int(1.0 / (6.0 * h))) + 1))
    F = _fourier_fields(rng, xy, D, modes=modes, max_freq=max_freq)
    side = float(np.exp(rng.uniform(np.log(1.0 / 16.0), 0.0)))
    x0, y0 = rng.uniform(0.0, 1.0 - side, size=2)
    W = int(min(1024, max(64, np.ceil(side / (h * rng.uniform(0.08, 0.3))))))
    H = int(max(32, round(W * rng.uniform(0.6, 1.0))))
    view = (float(x0), float(y0), float(x0 + side), float(y0 + side * H / W))
    wt = WEIGHT_GAUSS if gauss else WEIGHT_WENDLAND
    w = Workload(f"heldout{seed}_n{n}_d{D}_{W}x{H}_deg{degree}_w{wt}", xy, F, degree, wt, h, W, H, view=view)
    w.levels = default_levels(F, int(rng.integers(8, 21)))
    pix = sample_pixels(seed, W, H, 2048)
    u0, v0 = int(rng.integers(0, W - 24)), int(rng.integers(0, H - 24))
    win = np.array([(v0 + dv) * W + u0 + du for dv in range(24) for du in range(24)], np.int64)
    return w, np.unique(np.concatenate([pix, win]))


def batch_datasets(seed: int = 1004, count: int = 64, n_range=(200, 50_000), D_range=(4, 64),
                   side_range=(256, 1024)) -> list:
    """Independent datasets for batched rendering: n log-uniform in n_range,
    D uniform in D_range, a square grid with side uniform in side_range,
    linear or quadratic basis, Gaussian h = 0.5 / sqrt(n), each with the
    cluster + background structure and Fourier fields of fourier_mix."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        D = int(rng.integers(D_range[0], D_range[1] + 1))
        side = int(rng.integers(side_range[0], side_range[1] + 1))
        degree = int(rng.integers(1, 3))
        wl = fourier_mix(int(rng.integers(1 << 30)), n, D, side, side, degree, WEIGHT_GAUSS, 0.5 / np.sqrt(n))
        wl.name = f"batch{k}_n{n}_d{D}_{side}sq_deg{degree}"
        out.append(wl)
    return out


def small_random(seed: int, n: int, D: int, W: int, H: int, degree: int, weight: int,
                 h: float, L: int = 8, clustered: bool = True) -> Workload:
    """A small seeded case of the same structure, for tests."""
    rng = np.random.default_rng(seed)
    if clustered and n >= 8:
        k = max(1, min(4, n // 4))
        centres = rng.uniform(0.2, 0.8, size=(k, 2))
        xy = _clusters(rng, n, centres, rng.uniform(0.05, 0.15, size=k))
    else:
        xy = rng.uniform(0.0, 1.0, size=(n, 2))
    F = _fourier_fields(rng, xy, D, modes=4, max_freq=2)
    w = Workload(f"small_n{n}_d{D}_{W}x{H}_deg{degree}_w{weight}", xy, F, degree, weight, h, W, H)
    w.levels = default_levels(F, L)
    return w


def sample_pixels(seed: int, W: int, H: int, count: int) -> np.ndarray:
    """`count` distinct pixel indices (v*W+u), seeded, sorted."""
    rng = np.random.default_rng(seed)
    count = min(count, W * H)
    return np.sort(rng.choice(W * H, size=count, replace=False)).astype(np.int64)
