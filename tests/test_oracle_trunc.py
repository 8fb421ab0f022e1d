"""Pins of the oracle's truncated Gaussian: the Gaussian weight exp(-r^2/h^2)
kept only inside the box |dx|, |dy| < c h around each pixel (the reading of
skipping pairs whose weight is negligible, every pair left out having weight
below exp(-c^2) of the peak).  Checked against the full sum when the box
holds every point, the full-sum fit over the box's points selected with
numpy, a hand-computed weighted mean with exact edge cases, polynomial
reproduction and the mappings of Sections 3.3.1 / 3.3.3."""
import numpy as np
import pytest

import oracle

G = 0


def _centres(W, H, view=(0.0, 0.0, 1.0, 1.0)):
    x0, y0, x1, y1 = view
    u = np.arange(W * H) % W
    v = np.arange(W * H) // W
    return np.stack([x0 + (u + 0.5) * (x1 - x0) / W, y0 + (v + 0.5) * (y1 - y0) / H], axis=1)


def test_box_holding_every_point_is_the_full_sum():
    rng = np.random.default_rng(21)
    xy = rng.uniform(0, 1, (80, 2))
    F = rng.normal(size=(80, 3))
    for degree in (0, 1, 2):
        a = oracle.mls(xy, F, degree, G, 0.2, 9, 7)
        b = oracle.mls(xy, F, degree, G, 0.2, 9, 7, trunc=10.0)   # half-width 2 covers [0, 1]^2
        assert np.array_equal(a.field, b.field)
        assert np.array_equal(a.deg_used, b.deg_used)
        assert np.all(b.count == 80)


def test_equals_full_sum_over_the_points_in_the_box():
    rng = np.random.default_rng(22)
    xy = rng.uniform(0, 1, (300, 2))
    F = np.stack([np.sin(3 * xy[:, 0]) + xy[:, 1], np.cos(2 * xy[:, 1]) * xy[:, 0]], axis=1)
    F += rng.normal(scale=0.01, size=F.shape)
    h, c, W, H = 0.05, 3.0, 12, 10
    t = oracle.mls(xy, F, 1, G, h, W, H, trunc=c)
    for k, (px, py) in enumerate(_centres(W, H)):
        inb = (np.abs(xy[:, 0] - px) < c * h) & (np.abs(xy[:, 1] - py) < c * h)
        assert t.count[k] == inb.sum()
        if not inb.any():
            assert t.deg_used[k] == -1 and np.all(np.isnan(t.field[k]))
            continue
        sub = oracle.mls(xy[inb], F[inb], 1, G, h, W, H, pixels=[k])
        if t.amb[k] == 0 and sub.amb[0] == 0:
            assert t.deg_used[k] == sub.deg_used[0]
            np.testing.assert_allclose(t.field[k], sub.field[0], rtol=1e-10, atol=1e-10)


def test_box_not_disc_and_strict_edge():
    """One pixel centred at (0.5, 0.5), h = 1/8, c = 2: half-width 1/4 exactly.
    A point on the box edge is out (strict), a point inside the box but
    outside the disc of radius 1/4 is in; degree 0 gives the weighted mean."""
    xy = np.array([[0.5, 0.6], [0.75, 0.5], [0.3, 0.7], [0.5, 0.5 - 0.26], [0.75 - 2.0 ** -40, 0.45]])
    F = np.array([1.0, 100.0, 3.0, 50.0, 7.0])
    r = oracle.mls(xy, F, 0, G, 0.125, 1, 1, trunc=2.0)
    assert r.count[0] == 3
    inside = [0, 2, 4]
    w = np.exp(-((xy[inside] - 0.5) ** 2).sum(1) / 0.125 ** 2)
    np.testing.assert_allclose(r.field[0, 0], (w * F[inside]).sum() / w.sum(), rtol=1e-14)


def test_empty_box_is_nan():
    xy = np.array([[0.9, 0.9], [0.95, 0.9]])
    r = oracle.mls(xy, np.array([1.0, 2.0]), 1, G, 0.05, 2, 2, trunc=2.0)
    assert r.count[0] == 0 and r.deg_used[0] == -1 and np.isnan(r.field[0, 0])   # pixel (0.25, 0.25)


@pytest.mark.parametrize("degree", [1, 2])
def test_polynomial_reproduction(degree):
    rng = np.random.default_rng(23)
    xy = rng.uniform(0, 1, (200, 2))
    x, y = xy.T
    f = 2.0 + 3.0 * x - y + (0.5 * x * x - 0.25 * x * y + y * y if degree == 2 else 0.0)
    r = oracle.mls(xy, f, degree, G, 0.06, 10, 8, trunc=3.0)
    P = _centres(10, 8)
    px, py = P.T
    g = 2.0 + 3.0 * px - py + (0.5 * px * px - 0.25 * px * py + py * py if degree == 2 else 0.0)
    ok = r.deg_used == degree
    assert ok.sum() > 40
    np.testing.assert_allclose(r.field[ok, 0], g[ok], atol=1e-9)


def test_ambiguity_flag_at_the_box_edge():
    """A point within a relative 1e-6 of the box edge that could move the
    count across k sets amb bit 1."""
    xy = np.array([[0.5, 0.55], [0.5 + 0.25 * (1 - 1e-8), 0.5], [0.45, 0.45]])
    r = oracle.mls(xy, np.array([1.0, 2.0, 3.0]), 1, G, 0.125, 1, 1, trunc=2.0)
    assert r.count[0] == 3 and (r.amb[0] & 2)


def test_only_for_the_gaussian():
    xy = np.array([[0.5, 0.5]])
    with pytest.raises(ValueError):
        oracle.mls(xy, np.array([1.0]), 0, 1, 0.1, 2, 2, trunc=2.0)
    with pytest.raises(ValueError):
        oracle.mls(xy, np.array([1.0]), 0, G, 0.1, 2, 2, trunc=-1.0)


@pytest.mark.parametrize("variant", [oracle.VARIANT_RIGID, oracle.VARIANT_MEAN])
def test_mappings_with_the_truncated_gaussian(variant):
    rng = np.random.default_rng(24)
    xy = rng.uniform(0, 1, (120, 2))
    Q = xy @ np.array([[0.8, -0.6], [0.6, 0.8]]).T + 0.1 + rng.normal(scale=0.02, size=(120, 2))
    a = oracle.mls_variant(xy, Q, variant, G, 0.1, 7, 6)
    b = oracle.mls_variant(xy, Q, variant, G, 0.1, 7, 6, trunc=20.0)
    assert np.array_equal(a, b)
    t = oracle.mls_variant(xy, Q, variant, G, 0.05, 7, 6, trunc=3.0)
    for k, v in enumerate(_centres(7, 6)):
        inb = np.all(np.abs(xy - v) < 0.15, axis=1)
        sub = oracle.mls_variant(xy[inb], Q[inb], variant, G, 0.05, 7, 6, pixels=[k])
        np.testing.assert_allclose(t[k], sub[0], rtol=1e-11, atol=1e-12)
