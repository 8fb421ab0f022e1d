"""Pins of the space-mapping oracle (Section 3.4): hand-derived images of
fields whose gradient is known exactly, and planted mistakes that must fail
at least one pin.  Each pin takes the module under test as an argument so
that the same checks run against the planted variants."""
import importlib.util
import os

import numpy as np
import pytest

from oracle import space_map as SM

SRC = os.path.join(os.path.dirname(SM.__file__), "space_map.py")


def _ramp_field(W=32, H=4, slope=1.0):
    """f(u, v) = slope * u: gradient exactly slope per pixel everywhere."""
    u = np.arange(W, dtype=np.float32)
    return np.broadcast_to(u * np.float32(slope), (H, W)).astype(np.float32)[None]


def pin_line_coverage(sm=SM):
    """Levels 10.5 and 20.5 on f = u: the line centres fall between pixels,
    each neighbour is half a pixel away.  Width 1: both neighbours at half
    coverage (grey 128); width 3: the two black, the next ones half."""
    f = _ramp_field()
    lev = np.array([[10.5, 20.5]])
    img = sm.space_map(f, lev, [0], sm.LINES, line_width=1.0)
    row = img[0, :, 0]
    exp = np.full(32, 255, np.uint8)
    exp[[10, 11, 20, 21]] = 128
    assert np.array_equal(row, exp), row
    assert np.all(img[..., 3] == 255) and np.array_equal(img[..., 0], img[..., 1])
    img3 = sm.space_map(f, lev, [0], sm.LINES, line_width=3.0)
    exp3 = np.full(32, 255, np.uint8)
    exp3[[10, 11, 20, 21]] = 0
    exp3[[9, 12, 19, 22]] = 128
    assert np.array_equal(img3[2, :, 0], exp3), img3[2, :, 0]


def pin_level_on_pixel_centre(sm=SM):
    """A level exactly on a pixel's value: that pixel black, neighbours (one
    pixel away, beyond the half-pixel ramp of a width-1 line) white; with
    slope 2 the neighbours are two value units but one pixel away."""
    for slope in (1.0, 2.0):
        f = _ramp_field(slope=slope)
        img = sm.space_map(f, np.array([[15.0 * slope]]), [0], sm.LINES, line_width=1.0)
        row = img[1, :, 0]
        assert row[15] == 0 and row[14] == 255 and row[16] == 255


def pin_band_colours(sm=SM):
    """One level at 0.5: band 0 samples the ramp at 1/4 (halfway between the
    first two anchors), band 1 at 3/4 (halfway between the last two)."""
    f = np.zeros((1, 2, 2), np.float32)
    f[0, 1, :] = 1.0
    img = sm.space_map(f, np.array([[0.5]]), [0], sm.DISCRETE)
    a0, a1, a2 = (np.array(a) for a in ([0.16, 0.29, 0.78], [0.93, 0.93, 0.93], [0.78, 0.16, 0.16]))
    for v, e in ((0, (a0 + a1) / 2), (1, (a1 + a2) / 2)):
        np.testing.assert_allclose(img[v, 0, :3], e * 255, atol=0.5 + 1e-3)


def pin_gradient_corners(sm=SM):
    """Two dimensions at the corners of their ranges give the four corner
    colours (blue, pink along the first dimension, cyan along the second)."""
    f = np.zeros((2, 2, 2), np.float32)
    f[0, :, 1] = 4.0          # first dimension: lo 0 at u = 0, hi 4 at u = 1
    f[1, 0, :] = 1.0          # second dimension: lo 1 at v = 0, hi -1 at v = 1
    f[1, 1, :] = -1.0
    img = sm.space_map(f, np.zeros((2, 0)), [0, 1], sm.GRADIENT, lo=[0.0, 1.0], hi=[4.0, -1.0])
    corners = {(0, 0): [0.10, 0.20, 0.90], (0, 1): [0.95, 0.35, 0.75], (1, 0): [0.10, 0.85, 0.90],
               (1, 1): [0.95, 0.95, 0.75]}
    for (v, u), c in corners.items():
        np.testing.assert_allclose(img[v, u, :3], np.array(c) * 255, atol=0.5 + 1e-3)


def pin_texture_identity(sm=SM):
    """Field values at texel centres look the texture up unchanged."""
    rng = np.random.default_rng(5)
    tex = rng.integers(0, 256, (4, 8, 4), dtype=np.uint8)
    u = (np.arange(8, dtype=np.float32) + np.float32(0.5)) / np.float32(8)
    v = (np.arange(4, dtype=np.float32) + np.float32(0.5)) / np.float32(4)
    f = np.stack([np.broadcast_to(u, (4, 8)), np.broadcast_to(v[:, None], (4, 8))]).astype(np.float32)
    img = sm.space_map(f, np.zeros((2, 0)), [0, 1], sm.TEXTURE, lo=[0, 0], hi=[1, 1], texture=tex)
    assert np.array_equal(img, tex)


def pin_adaptive_fading(sm=SM):
    """f = u, levels 0 and 16 (spacing 16 px), fade from 2 to 6 px, 3 halvings:
    depth 1 (8 px apart) fully drawn at 8, depth 2 (4 px) half at 4 and 12,
    depth 3 (2 px) not at all."""
    f = _ramp_field(W=17)
    img = sm.space_map(f, np.array([[0.0, 16.0]]), [0], sm.ADAPTIVE, line_width=1.0, fade=(2.0, 6.0, 3))
    row = img[0, :, 0]
    assert row[0] == 0 and row[16] == 0 and row[8] == 0
    assert row[4] == 128 and row[12] == 128
    assert row[2] == 255 and row[6] == 255 and row[10] == 255


def pin_nan_transparent_and_one_sided(sm=SM):
    """NaN pixels are transparent; their neighbours take one-sided
    differences, so a line next to the hole looks as without it."""
    f = _ramp_field()
    f[0, 1, 12] = np.nan
    img = sm.space_map(f, np.array([[10.5]]), [0], sm.LINES)
    assert np.array_equal(img[1, 12], [0, 0, 0, 0])
    assert img[1, 11, 0] == 128 and img[1, 10, 0] == 128 and img[1, 13, 0] == 255


PINS = [pin_line_coverage, pin_level_on_pixel_centre, pin_band_colours, pin_gradient_corners,
        pin_texture_identity, pin_adaptive_fading, pin_nan_transparent_and_one_sided]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


MUTANTS = [
    ("central difference without the half", "both = (gr - gl) * f32(0.5)", "both = (gr - gl)"),
    ("line ramp not centred on the edge", "(f32(w) * f32(0.5) + f32(0.5)) - delta", "f32(w) * f32(0.5) - delta"),
    ("band colour sampled at b / L", "(b.astype(f32) + f32(0.5)) * _recip(f32(L + 1))",
     "b.astype(f32) * _recip(f32(L))"),
    ("sub-levels at even multiples", "m = f32(2.0) * np.floor(r * f32(0.5)) + f32(1.0)",
     "m = f32(2.0) * np.floor(r * f32(0.5))"),
    ("texture sampled at the texel corner", "x = s * f32(Tw) - f32(0.5)", "x = s * f32(Tw)"),
    ("corner colours swapped", "a = _lerp(CORNERS[0], CORNERS[1], s[..., None])",
     "a = _lerp(CORNERS[0], CORNERS[2], s[..., None])"),
    ("fade inverted", "alpha = _clamp01((sp - f32(fade_lo)) * inv_den)",
     "alpha = _clamp01((f32(fade_hi) - sp) * inv_den)"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    spec = importlib.util.spec_from_loader("space_map_mutant", loader=None)
    mod = importlib.util.module_from_spec(spec)
    exec(compile(src.replace(old, new), "space_map_mutant", "exec"), mod.__dict__)
    caught = False
    for pin in PINS:
        try:
            pin(mod)
        except (AssertionError, ValueError, IndexError):
            caught = True
            break
    assert caught, f"no pin caught the planted mistake: {name}"
