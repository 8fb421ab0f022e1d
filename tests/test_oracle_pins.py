"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

The paper prints no worked field values, so the oracle is pinned by
polynomial reproduction (Section 3.3, criterion 3), invariances, the paper's
own affine formula (Eq. eq-affinemls), textbook reductions (weighted mean of
Section 3.3.1; global least squares; nearest neighbour), hand-derived golden
fixtures under tests/golden/, and brute force by an SVD least-squares solver.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import pin_forms as pf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
G, WD, ID = oracle.oracle.GAUSS, oracle.oracle.WENDLAND, oracle.oracle.INVDIST


def _pts(seed, n, lo=0.05, hi=0.95):
    return np.random.default_rng(seed).uniform(lo, hi, size=(n, 2))


def _poly_field(xy, degree, seed):
    rng = np.random.default_rng(seed)
    x, y = xy[:, 0], xy[:, 1]
    cols = [np.ones_like(x)]
    if degree >= 1:
        cols += [x, y]
    if degree >= 2:
        cols += [x * x, x * y, y * y]
    B = np.stack(cols, 1)
    C = rng.normal(size=(B.shape[1], 3))
    return B @ C, C


def _poly_eval(px, py, degree, C):
    cols = [np.ones_like(px)]
    if degree >= 1:
        cols += [px, py]
    if degree >= 2:
        cols += [px * px, px * py, py * py]
    return np.stack(cols, 1) @ C


@pytest.mark.parametrize("weight,h", [(G, 0.2), (WD, 0.6), (ID, 0.3)])
@pytest.mark.parametrize("degree", [0, 1, 2])
def test_polynomial_reproduction(weight, h, degree):
    """A degree-k basis reproduces a degree-k field exactly (Section 3.3 criterion 3)."""
    xy = _pts(1, 40)
    F, C = _poly_field(xy, degree, 2)
    W = H = 9
    r = oracle.mls(xy, F, degree, weight, h, W, H)
    px, py = pf.pixel_centres(W, H)
    expect = _poly_eval(px, py, degree, C)
    assert np.all(r.deg_used == degree)
    np.testing.assert_allclose(r.field, expect, rtol=0, atol=1e-10 * np.abs(expect).max())


def test_quadratic_not_reproduced_by_linear():
    """Guard that the reproduction test can fail: a linear basis misses a quadratic field."""
    xy = _pts(3, 40)
    F, C = _poly_field(xy, 2, 4)
    r = oracle.mls(xy, F, 1, G, 0.2, 6, 6)
    px, py = pf.pixel_centres(6, 6)
    assert np.abs(r.field - _poly_eval(px, py, 2, C)).max() > 1e-4


@pytest.mark.parametrize("degree", [0, 1, 2])
def test_affine_invariance_in_values(degree):
    xy = _pts(5, 30)
    F = np.random.default_rng(6).normal(size=(30, 4))
    a, b = -2.5, 7.25
    r1 = oracle.mls(xy, F, degree, G, 0.15, 8, 8)
    r2 = oracle.mls(xy, a * F + b, degree, G, 0.15, 8, 8)
    scale = np.abs(a * r1.field).max() + abs(b)
    np.testing.assert_allclose(r2.field, a * r1.field + b, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("weight,h", [(G, 0.15), (WD, 0.4), (ID, 0.2)])
def test_translation_invariance(weight, h):
    xy = _pts(7, 25)
    F = np.random.default_rng(8).normal(size=(25, 3))
    t = np.array([3.25, -1.5])
    r1 = oracle.mls(xy, F, 2, weight, h, 7, 5)
    r2 = oracle.mls(xy + t, F, 2, weight, h, 7, 5, view=(t[0], t[1], 1 + t[0], 1 + t[1]))
    assert np.array_equal(r1.deg_used, r2.deg_used)
    # shifting loses ~2 bits of each coordinate; the fit amplifies that by ~1/rcond
    ok = r1.rcond > 1e-6
    assert ok.sum() > 20
    np.testing.assert_allclose(r2.field[ok], r1.field[ok], rtol=0, atol=1e-9 * np.abs(r1.field).max())


def test_rotation_by_90_degrees():
    """Rotating points about the domain centre rotates the image (isotropic weights)."""
    xy = _pts(9, 30)
    F = np.random.default_rng(10).normal(size=(30, 2))
    W = H = 8
    r1 = oracle.mls(xy, F, 2, G, 0.2, W, H).field.reshape(H, W, 2)
    rot = np.stack([1.0 - xy[:, 1], xy[:, 0]], 1)     # (x, y) -> (1 - y, x)
    r2 = oracle.mls(rot, F, 2, G, 0.2, W, H).field.reshape(H, W, 2)
    # pixel (u, v) maps to (W-1-v, u)
    for v in range(H):
        for u in range(W):
            np.testing.assert_allclose(r2[u, W - 1 - v], r1[v, u], rtol=0, atol=1e-10)


def test_scaling_invariance():
    xy = _pts(11, 30)
    F = np.random.default_rng(12).normal(size=(30, 2))
    r1 = oracle.mls(xy, F, 2, WD, 0.5, 6, 6)
    r2 = oracle.mls(4.0 * xy, F, 2, WD, 2.0, 6, 6, view=(0, 0, 4, 4))
    np.testing.assert_allclose(r2.field, r1.field, rtol=0, atol=1e-10)


def test_dimension_independence():
    """Each dimension is fitted alone with the shared M: a D=1 run equals its column."""
    xy = _pts(13, 50)
    F = np.random.default_rng(14).normal(size=(50, 5))
    full = oracle.mls(xy, F, 2, G, 0.12, 6, 5).field
    for d in range(5):
        one = oracle.mls(xy, F[:, d], 2, G, 0.12, 6, 5).field[:, 0]
        assert np.array_equal(one, full[:, d])


def test_interpolation_linear_three_points():
    """n = k = 3: the unique plane through the points, whatever the weights."""
    xy = np.array([[0.2, 0.3], [0.8, 0.25], [0.45, 0.85]])
    f = np.array([1.0, -2.0, 0.5])
    A = np.c_[np.ones(3), xy]
    coef = np.linalg.solve(A, f)
    r = oracle.mls(xy, f, 1, G, 0.3, 5, 5)
    px, py = pf.pixel_centres(5, 5)
    np.testing.assert_allclose(r.field[:, 0], coef[0] + coef[1] * px + coef[2] * py, atol=1e-11)


def test_interpolation_quadratic_six_points():
    xy = np.array([[0.1, 0.1], [0.9, 0.2], [0.5, 0.9], [0.3, 0.6], [0.7, 0.55], [0.5, 0.3]])
    f = np.array([0.3, -1.0, 2.0, 0.7, -0.4, 1.1])
    x, y = xy[:, 0], xy[:, 1]
    V = np.stack([np.ones(6), x, y, x * x, x * y, y * y], 1)
    coef = np.linalg.solve(V, f)
    r = oracle.mls(xy, f, 2, G, 0.4, 4, 4)
    px, py = pf.pixel_centres(4, 4)
    expect = np.stack([np.ones_like(px), px, py, px * px, px * py, py * py], 1) @ coef
    assert np.all(r.deg_used == 2)
    np.testing.assert_allclose(r.field[:, 0], expect, atol=1e-9)


@pytest.mark.parametrize("weight,h,alpha", [(G, 0.15, 1.0), (WD, 0.45, 1.0), (ID, 0.1, 0.8)])
def test_degree0_is_weighted_mean(weight, h, alpha):
    xy = _pts(15, 20)
    F = np.random.default_rng(16).normal(size=(20, 3))
    W, H = 5, 4
    r = oracle.mls(xy, F, 0, weight, h, W, H, alpha=alpha)
    px, py = pf.pixel_centres(W, H)
    for q in range(W * H):
        r2 = (xy[:, 0] - px[q]) ** 2 + (xy[:, 1] - py[q]) ** 2
        if weight == G:
            w = pf.weights_gauss(r2, h)
        elif weight == WD:
            w = pf.weights_wendland(r2, h)
        else:
            w = pf.weights_invdist(r2, alpha)
        if w.sum() == 0:
            assert np.all(np.isnan(r.field[q]))
            continue
        np.testing.assert_allclose(r.field[q], pf.shepard(F, w), rtol=1e-12, atol=1e-13)


def test_affine_equals_paper_centroid_form():
    """Linear-basis moment form == Eq. eq-affinemls with weighted centroids."""
    xy = _pts(17, 35)
    F = np.random.default_rng(18).normal(size=(35, 4))
    W, H = 7, 6
    h = 0.18
    r = oracle.mls(xy, F, 1, G, h, W, H)
    px, py = pf.pixel_centres(W, H)
    for q in range(W * H):
        p = np.array([px[q], py[q]])
        w = pf.weights_gauss(((xy - p) ** 2).sum(1), h)
        np.testing.assert_allclose(r.field[q], pf.affine_centroid(xy, F, p, w), rtol=1e-10, atol=1e-11)


def test_large_h_is_global_least_squares():
    xy = _pts(19, 30)
    F = np.random.default_rng(20).normal(size=(30, 2))
    r = oracle.mls(xy, F, 2, G, 1e5, 4, 4)
    px, py = pf.pixel_centres(4, 4)
    for q in range(16):
        p = np.array([px[q], py[q]])
        np.testing.assert_allclose(r.field[q], pf.wls_lstsq(xy, F, p, np.ones(30), 2, s=0.3), atol=1e-7)


def test_small_h_is_nearest_neighbour_with_degree_fallback():
    """h -> 0 leaves one point of weight ~1: M is singular for degree >= 1, the policy
    falls back to degree 0 and the value is the nearest point's (Voronoi)."""
    g = np.linspace(0.1, 0.9, 5)
    xy = np.array([[a, b] for a in g for b in g])
    F = np.random.default_rng(21).normal(size=(25, 2))
    W = H = 10
    r = oracle.mls(xy, F, 2, G, 1e-3, W, H)
    px, py = pf.pixel_centres(W, H)
    for q in range(W * H):
        d2 = (xy[:, 0] - px[q]) ** 2 + (xy[:, 1] - py[q]) ** 2
        order = np.argsort(d2)
        if d2[order[1]] - d2[order[0]] < 1e-3:
            continue   # near a Voronoi edge: two comparable weights
        assert r.deg_used[q] == 0
        np.testing.assert_allclose(r.field[q], F[order[0]], atol=1e-12)


def test_wendland_single_point_and_empty_support():
    xy = np.array([[0.2, 0.2], [0.8, 0.8], [0.82, 0.78]])
    F = np.array([[5.0], [1.0], [2.0]])
    W = H = 10
    r = oracle.mls(xy, F, 2, WD, 0.1, W, H)
    px, py = pf.pixel_centres(W, H)
    for q in range(W * H):
        d2 = (xy[:, 0] - px[q]) ** 2 + (xy[:, 1] - py[q]) ** 2
        inside = d2 < 0.01
        if inside.sum() == 0:
            assert r.deg_used[q] == -1 and np.isnan(r.field[q, 0])
        elif inside.sum() == 1:
            assert r.deg_used[q] == 0
            assert r.field[q, 0] == pytest.approx(F[inside][0, 0], abs=1e-13)
    b = oracle.bands(r.field, np.array([[1.5, 3.0]]))
    assert np.all(b[np.isnan(r.field[:, 0])] == 255)


def test_idw_point_identity():
    """Section 3.3 criterion 2: f(p_i) = q_i for the inverse-distance weight."""
    W = H = 8
    px, py = pf.pixel_centres(W, H)
    idx = [3, 17, 42, 60]
    xy = np.stack([px[idx], py[idx]], 1)
    F = np.random.default_rng(22).normal(size=(4, 3))
    r = oracle.mls(xy, F, 1, ID, 0.2, W, H, alpha=1.2)
    for j, q in enumerate(idx):
        np.testing.assert_allclose(r.field[q], F[j], atol=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_tiny_cases(seed):
    """Tiny cases against an SVD least-squares solve of sqrt(w) B c = sqrt(w) f."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(6, 13))
    W, H = int(rng.integers(4, 17)), int(rng.integers(4, 17))
    degree = int(rng.integers(0, 3))
    weight = [G, WD, ID][seed % 3]
    h = [0.25, 0.7, 0.3][seed % 3]
    xy = rng.uniform(0, 1, size=(n, 2))
    F = rng.normal(size=(n, 3))
    r = oracle.mls(xy, F, degree, weight, h, W, H, alpha=1.0)
    px, py = pf.pixel_centres(W, H)
    for q in range(W * H):
        p = np.array([px[q], py[q]])
        r2 = ((xy - p) ** 2).sum(1)
        if weight == G:
            w = pf.weights_gauss(r2, h)
        elif weight == WD:
            w = pf.weights_wendland(r2, h)
        else:
            w = pf.weights_invdist(r2, 1.0)
        if r.deg_used[q] < 0:
            assert w.sum() == 0
            continue
        if r.amb[q]:
            continue
        ref = pf.wls_lstsq(xy, F, p, w / w.max(), int(r.deg_used[q]), s=h)
        # normal equations lose ~eps/rcond relative to the SVD solve
        tol = 1e-10 + 1e-14 / r.rcond[q]
        np.testing.assert_allclose(r.field[q], ref, rtol=0, atol=tol * np.abs(F).max())


def test_bands_definition_and_ties():
    field = np.array([[0.0, 1.0], [0.5, 2.0], [1.0, np.nan], [-1.0, 3.5]])
    levels = np.array([[0.0, 0.5, 0.75], [1.0, 2.0, 3.0]])
    b = oracle.bands(field, levels)
    # f = t counts as above the level
    expect = np.array([[1, 1], [2, 2], [3, 255], [0, 3]], np.uint8)
    assert np.array_equal(b, expect)
    # against a sorted search
    f = np.random.default_rng(23).normal(size=(200, 2))
    b = oracle.bands(f, levels)
    for d in range(2):
        assert np.array_equal(b[:, d], np.searchsorted(levels[d], f[:, d], side="right"))


def test_bands_outlier_ring_and_plateau():
    """Section 4.1: an isolated high point gives closed rings (a peak); a constant
    cluster gives a plateau (one label)."""
    rng = np.random.default_rng(24)
    bg = rng.uniform(0, 1, size=(300, 2))
    bg = bg[((bg - 0.5) ** 2).sum(1) > 0.01]
    xy = np.vstack([bg, [[0.5, 0.5]]])
    F = np.zeros((xy.shape[0], 1))
    F[-1, 0] = 10.0
    W = H = 41
    r = oracle.mls(xy, F, 0, G, 0.05, W, H)
    levels = np.array([[0.5, 2.0, 5.0]])
    b = oracle.bands(r.field, levels).reshape(H, W)
    c = W // 2
    assert b[c, c] == b.max() >= 2
    # labels do not increase moving away from the peak along the four axes
    for dv, du in [(0, 1), (0, -1), (1, 0), (-1, 0)]:
        ray = [b[c + k * dv, c + k * du] for k in range(c + 1)]
        assert all(ray[k] >= ray[k + 1] for k in range(len(ray) - 1))
        assert ray[-1] == 0
    # plateau: constant values inside a cluster -> one label over its interior
    cl = 0.5 + 0.05 * rng.standard_normal((200, 2))
    F2 = np.full((200, 1), 3.0)
    r2 = oracle.mls(cl, F2, 1, G, 0.05, 16, 16, view=(0.45, 0.45, 0.55, 0.55))
    b2 = oracle.bands(r2.field, levels)
    assert np.all(b2 == 2)


def _read_golden(name):
    pts, pix, meta = [], [], {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "points":
                pts.append([float(t) for t in tok[1:]])
            elif tok[0] == "pixel":
                pix.append((int(tok[1]), int(tok[2]), tok[3]))
            else:
                meta[tok[0]] = tok[1:]
    return np.array(pts), pix, meta


def test_golden_idw_two_points():
    pts, pix, meta = _read_golden("idw_two_points.txt")
    W, H = int(meta["grid"][0]), int(meta["grid"][1])
    r = oracle.mls(pts[:, :2], pts[:, 2:], 0, ID, 1.0, W, H, alpha=float(meta["alpha"][0]))
    for u, v, val in pix:
        assert r.field[v * W + u, 0] == pytest.approx(float(Fraction(val)), abs=1e-14)


def test_golden_gauss_two_points():
    pts, pix, meta = _read_golden("gauss_two_points.txt")
    W, H = int(meta["grid"][0]), int(meta["grid"][1])
    r = oracle.mls(pts[:, :2], pts[:, 2:], 0, G, float(meta["h"][0]), W, H)
    e4 = math.exp(-4.0)
    for u, v, expr in pix:
        assert r.field[v * W + u, 0] == pytest.approx(eval(expr, {"e4": e4}), abs=1e-14)


@pytest.mark.parametrize("weight", [G, WD, ID])
def test_golden_plane_four_points(weight):
    pts, pix, meta = _read_golden("plane_four_points.txt")
    W, H = int(meta["grid"][0]), int(meta["grid"][1])
    h = float(meta["h"][0]) * (4.0 if weight == WD else 1.0)
    r = oracle.mls(pts[:, :2], pts[:, 2:], 1, weight, h, W, H)
    for u, v, val in pix:
        assert r.field[v * W + u, 0] == pytest.approx(float(Fraction(val)), abs=1e-12)
