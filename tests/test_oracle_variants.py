"""Pins of the oracle's rigid (Section 3.3.3, Eqs. eq-rigidmls and
eq-rigidmlspartial) and mean-displacement (Section 3.3.1, Eq. eq-meanmls)
mappings of 2-D values: exact reproduction of rigid motions and
translations, the identity when nothing is distorted (the paper's third
criterion in Section 3.3), point identity for inverse-distance weights, and
the weighted rigid fit found by brute-force search over rotation angles."""
import numpy as np
import pytest

import oracle

GW = [(0, 0.3), (1, 0.6), (2, 0.2)]   # (weight, h): Gaussian, Wendland (wide support), inverse distance


def _centres(W, H, view=(0.0, 0.0, 1.0, 1.0)):
    x0, y0, x1, y1 = view
    u = np.arange(W * H) % W
    v = np.arange(W * H) // W
    return np.stack([x0 + (u + 0.5) * (x1 - x0) / W, y0 + (v + 0.5) * (y1 - y0) / H], axis=1)


def _rot(th):
    return np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])


@pytest.mark.parametrize("weight,h", GW)
def test_rigid_reproduces_rigid_motions(weight, h):
    rng = np.random.default_rng(1 + weight)
    xy = rng.uniform(0, 1, (60, 2))
    for th, t in ((0.7, (0.2, -0.1)), (-2.5, (1.0, 3.0))):
        R, t = _rot(th), np.array(t)
        f = oracle.mls_variant(xy, xy @ R.T + t, oracle.VARIANT_RIGID, weight, h, 9, 7)
        P = _centres(9, 7)
        ok = np.isfinite(f[:, 0])
        assert ok.sum() > 40
        np.testing.assert_allclose(f[ok], (P @ R.T + t)[ok], atol=1e-12)


@pytest.mark.parametrize("weight,h", GW)
@pytest.mark.parametrize("variant", [oracle.VARIANT_RIGID, oracle.VARIANT_MEAN])
def test_identity_when_nothing_is_distorted(weight, h, variant):
    rng = np.random.default_rng(3)
    xy = rng.uniform(0, 1, (50, 2))
    f = oracle.mls_variant(xy, xy, variant, weight, h, 8, 6)
    ok = np.isfinite(f[:, 0])
    np.testing.assert_allclose(f[ok], _centres(8, 6)[ok], atol=1e-12)


@pytest.mark.parametrize("weight,h", GW)
def test_mean_reproduces_translations(weight, h):
    rng = np.random.default_rng(4)
    xy = rng.uniform(0, 1, (50, 2))
    t = np.array([0.25, -0.75])
    f = oracle.mls_variant(xy, xy + t, oracle.VARIANT_MEAN, weight, h, 8, 6)
    ok = np.isfinite(f[:, 0])
    np.testing.assert_allclose(f[ok], (_centres(8, 6) + t)[ok], atol=1e-12)


def test_mean_is_pixel_plus_weighted_mean_displacement():
    """Eq. eq-meanmls written out with numpy Gaussian weights."""
    rng = np.random.default_rng(5)
    xy = rng.uniform(0, 1, (30, 2))
    Q = rng.normal(size=(30, 2))
    h = 0.25
    f = oracle.mls_variant(xy, Q, oracle.VARIANT_MEAN, 0, h, 6, 5)
    P = _centres(6, 5)
    for k, v in enumerate(P):
        w = np.exp(-((xy - v) ** 2).sum(1) / h ** 2)
        np.testing.assert_allclose(f[k], v + (w[:, None] * (Q - xy)).sum(0) / w.sum(), rtol=1e-11, atol=1e-12)


def test_rigid_equals_best_weighted_rotation_by_search():
    """The rigid mapping is (v - p*) rotated by the angle minimising
    sum w |R p^ - q^|^2, plus q*: found here by a dense search over angles
    refined by golden-section steps (a different algorithm)."""
    rng = np.random.default_rng(6)
    xy = rng.uniform(0, 1, (25, 2))
    Q = xy @ _rot(0.9).T + rng.normal(scale=0.15, size=(25, 2))    # not rigid
    h = 0.35
    f = oracle.mls_variant(xy, Q, oracle.VARIANT_RIGID, 0, h, 5, 4)
    for k, v in enumerate(_centres(5, 4)):
        w = np.exp(-((xy - v) ** 2).sum(1) / h ** 2)
        ps = (w[:, None] * xy).sum(0) / w.sum()
        qs = (w[:, None] * Q).sum(0) / w.sum()
        ph, qh = xy - ps, Q - qs

        def err(th):
            return (w * ((ph @ _rot(th).T - qh) ** 2).sum(1)).sum()

        ths = np.linspace(0, 2 * np.pi, 7200, endpoint=False)
        th0 = ths[np.argmin([err(t) for t in ths])]
        a, b = th0 - 2e-3, th0 + 2e-3
        g = (np.sqrt(5) - 1) / 2
        for _ in range(80):
            c, d = b - g * (b - a), a + g * (b - a)
            if err(c) < err(d):
                b = d
            else:
                a = c
        th = 0.5 * (a + b)
        np.testing.assert_allclose(f[k], _rot(th) @ (v - ps) + qs, atol=1e-7)


@pytest.mark.parametrize("variant", [oracle.VARIANT_RIGID, oracle.VARIANT_MEAN])
def test_inverse_distance_point_identity(variant):
    """A pixel centre on a data point takes that point's value (criterion 2
    of Section 3.3)."""
    xy = np.array([[0.25, 0.5], [0.75, 0.5], [0.4, 0.9]])
    Q = np.array([[3.0, -1.0], [5.0, 2.0], [0.5, 0.5]])
    f = oracle.mls_variant(xy, Q, variant, 2, 0.2, 2, 1, view=(0.0, 0.0, 1.0, 1.0))
    np.testing.assert_allclose(f, Q[:2], atol=0)


@pytest.mark.parametrize("variant", [oracle.VARIANT_RIGID, oracle.VARIANT_MEAN])
def test_single_point_support_is_a_translation(variant):
    """One point in a Wendland support: the rotation of the rigid form is
    undetermined and no rotation is taken, so both forms move the pixel by
    that point's displacement q - p."""
    xy = np.array([[0.3, 0.3], [0.9, 0.8], [0.95, 0.8]])
    Q = np.array([[1.0, -2.0], [0.0, 0.0], [0.5, 0.1]])
    f, ax = oracle.mls_variant(xy, Q, variant, 1, 0.2, 4, 4, aux=True)
    P = _centres(4, 4)
    d = np.hypot(*(P - xy[0]).T)
    one = d < 0.2
    assert one.sum() >= 2
    np.testing.assert_allclose(f[one], (P + Q[0] - xy[0])[one], atol=1e-14)
    if variant == oracle.VARIANT_RIGID:
        assert np.all(np.isinf(ax[one, 3]))


def test_coincident_support_is_a_translation():
    """Every point of positive weight at one position (duplicates with
    different values): the rigid form translates by the mean displacement."""
    xy = np.array([[0.5, 0.5], [0.5, 0.5], [0.5, 0.5]])
    Q = np.array([[1.0, 0.0], [2.0, 1.0], [0.0, 2.0]])
    f = oracle.mls_variant(xy, Q, oracle.VARIANT_RIGID, 0, 0.3, 3, 3)
    np.testing.assert_allclose(f, _centres(3, 3) + Q.mean(0) - xy[0], atol=1e-14)


def test_rotation_conditioning():
    """kappa = sum w |dp||dq| / |mu| is 1 for a rigid motion (every pair
    agrees on the angle) and >= 1 always (triangle inequality); the reported
    q* and |v - p*| match numpy weighted means."""
    rng = np.random.default_rng(11)
    xy = rng.uniform(0, 1, (40, 2))
    h = 0.3
    _, ax = oracle.mls_variant(xy, xy @ _rot(1.1).T + 2.0, oracle.VARIANT_RIGID, 0, h, 6, 5, aux=True)
    np.testing.assert_allclose(ax[:, 3], 1.0, rtol=1e-12)
    Q = rng.normal(size=(40, 2))
    _, ax = oracle.mls_variant(xy, Q, oracle.VARIANT_RIGID, 0, h, 6, 5, aux=True)
    assert np.all(ax[:, 3] >= 1.0 - 1e-12) and np.any(ax[:, 3] > 1.5)
    for k, v in enumerate(_centres(6, 5)):
        w = np.exp(-((xy - v) ** 2).sum(1) / h ** 2)
        np.testing.assert_allclose(ax[k, :2], (w[:, None] * Q).sum(0) / w.sum(), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(ax[k, 2], np.hypot(*(v - (w[:, None] * xy).sum(0) / w.sum())), rtol=1e-12)
