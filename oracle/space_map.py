"""Space mappings of Section 3.4 (test infrastructure, see the package header).

The paper turns the MLS field into an image in one of several ways: contour
lines, a discrete colour per band, both together, lines added adaptively
where the field's gradient leaves room for them, colour gradients between
the contours, or a texture looked up with the field as coordinates.  It
describes them in words only; this module writes down the reading used here
in plain numpy, one image-wide step at a time.  Every step is a float32
operation (+, -, *, /, sqrt, floor, comparisons) in a fixed order, so that a
kernel doing the same operations in the same order gives the same bytes.
Quotients are taken as products with a reciprocal formed once (1/grad and
1/spacing per pixel and plane, 1/(L + 1), 1/(hi - lo), 1/(fade_hi - fade_lo)
per image), which is the float sequence of this reading.

Per pixel and shown dimension d (one or two of the field's planes):
  g      the field value rounded to float32
  grad   |(g_x, g_y)| in value units per pixel: central differences, one-sided
         at the image edge or next to a NaN neighbour, 0 with no neighbour
  b      the band #{t_j <= f} (compared in the field's own precision)
  delta  distance in pixels to the nearer bounding level of the band,
         min |g - t| * (1 / grad) (0 on a level, infinite where grad = 0)
  cov    line coverage clamp(w/2 + 1/2 - delta, 0, 1) (a one-pixel ramp at the
         edge of a line of width w)
Adaptive lines: the band's level spacing is halved k = 1..K times; a level of
depth k (odd multiples of spacing / 2^k above the band's lower level) is drawn
with the same coverage rule, faded by clamp((spacing / 2^k / grad - fade_lo) /
(fade_hi - fade_lo), 0, 1): lines appear where the field changes slowly over
the screen (space expanded) and fade out where it changes fast.
Colours: a three-anchor ramp over [0, 1] for one dimension, a bilinear blend
of four corner colours (blue, pink along the first dimension, cyan along the
second) for two; the band's colour samples it at (b + 1/2) / (L + 1); the
gradient mapping at (g - lo) / (hi - lo) clamped to [0, 1]; the texture
mapping samples an RGBA8 texture bilinearly (clamp to edge) at those
coordinates.  Lines are black over white or over the colours.  A pixel where
a shown dimension is NaN is transparent (0, 0, 0, 0).
"""
from __future__ import annotations

import numpy as np

f32 = np.float32

LINES, DISCRETE, DISCRETE_LINES, ADAPTIVE, GRADIENT, TEXTURE = range(6)

RAMP = np.array([[0.16, 0.29, 0.78], [0.93, 0.93, 0.93], [0.78, 0.16, 0.16]], dtype=f32)
CORNERS = np.array([[0.10, 0.20, 0.90],     # (0, 0) blue
                    [0.95, 0.35, 0.75],     # (1, 0) pink
                    [0.10, 0.85, 0.90],     # (0, 1) cyan
                    [0.95, 0.95, 0.75]], dtype=f32)


def _lerp(a, b, t):
    return a + (b - a) * t


def _clamp01(x):
    return np.minimum(np.maximum(x, f32(0.0)), f32(1.0))


def gradient(g):
    """|grad g| in value units per pixel (float32), central or one-sided."""
    H, W = g.shape
    fin = ~np.isnan(g)

    def axis(gl, gr, has_l, has_r, gc):
        both = (gr - gl) * f32(0.5)
        right = gr - gc
        left = gc - gl
        return np.where(has_l & has_r, both, np.where(has_r, right, np.where(has_l, left, f32(0.0))))

    gp = np.pad(g, 1, constant_values=np.nan)
    fp = np.pad(fin, 1, constant_values=False)
    gx = axis(gp[1:-1, :-2], gp[1:-1, 2:], fp[1:-1, :-2], fp[1:-1, 2:], g)
    gy = axis(gp[:-2, 1:-1], gp[2:, 1:-1], fp[:-2, 1:-1], fp[2:, 1:-1], g)
    return np.sqrt(gx * gx + gy * gy).astype(f32)


def _recip(x):
    with np.errstate(divide="ignore"):
        return (f32(1.0) / x).astype(f32)


def _px_distance(dv, grad, inv_grad):
    with np.errstate(invalid="ignore"):
        q = dv * inv_grad
    return np.where(dv == 0, f32(0.0), np.where(grad > 0, q, f32(np.inf))).astype(f32)


def _coverage(delta, w):
    return _clamp01((f32(w) * f32(0.5) + f32(0.5)) - delta)


def _band(f, lev):
    b = np.zeros(f.shape, np.int64)
    for t in lev:
        b += (f >= t)
    return b


def dim_terms(field_d, lev_d, w, adaptive=None):
    """g, band, coverage (base lines, plus adaptive sub-levels when given
    (fade_lo, fade_hi, K)) of one field plane."""
    L = len(lev_d)
    g = field_d.astype(f32)
    grad = gradient(g)
    inv_grad = _recip(grad)
    b = _band(field_d, lev_d)
    t32 = lev_d.astype(f32)
    dv = np.full(g.shape, np.inf, f32)
    if L:
        bl = np.clip(b - 1, 0, L - 1)
        bh = np.clip(b, 0, L - 1)
        dlo = np.where(b >= 1, np.abs(g - t32[bl]), f32(np.inf))
        dhi = np.where(b < L, np.abs(g - t32[bh]), f32(np.inf))
        dv = np.minimum(dlo, dhi)
    cov = _coverage(_px_distance(dv, grad, inv_grad), w)
    if adaptive is not None and L >= 2:
        fade_lo, fade_hi, K = adaptive
        inner = (b >= 1) & (b <= L - 1)
        bl = np.clip(b - 1, 0, L - 1)
        bh = np.clip(b, 0, L - 1)
        spacing = np.where(inner, t32[bh] - t32[bl],
                           np.where(b == 0, t32[1] - t32[0], t32[L - 1] - t32[L - 2]))
        base = np.where(inner, t32[bl], np.where(b == 0, t32[0] - spacing, t32[L - 1]))
        inv_spacing = _recip(spacing)
        ok = (spacing > 0) & np.isfinite(inv_spacing)
        inv_den = _recip(f32(fade_hi) - f32(fade_lo))
        for k in range(1, K + 1):
            dk = spacing * f32(1.0 / (1 << k))
            inv_dk = inv_spacing * f32(1 << k)
            with np.errstate(invalid="ignore", over="ignore"):
                sp = np.where(grad > 0, dk * inv_grad, f32(np.inf))
                alpha = _clamp01((sp - f32(fade_lo)) * inv_den)
                r = (g - base) * inv_dk
            m = f32(2.0) * np.floor(r * f32(0.5)) + f32(1.0)
            dist = np.abs(r - m) * dk
            ck = _coverage(_px_distance(dist, grad, inv_grad), w) * alpha
            cov = np.where(ok & (alpha > 0), np.maximum(cov, ck), cov)
    return g, b, cov


def _ramp(s):
    lo = _lerp(RAMP[0], RAMP[1], (s * f32(2.0))[..., None])
    hi = _lerp(RAMP[1], RAMP[2], ((s - f32(0.5)) * f32(2.0))[..., None])
    return np.where((s <= f32(0.5))[..., None], lo, hi)


def _corner(s, t):
    a = _lerp(CORNERS[0], CORNERS[1], s[..., None])
    c = _lerp(CORNERS[2], CORNERS[3], s[..., None])
    return _lerp(a, c, t[..., None])


def _to_byte(c):
    q = np.floor(c * f32(255.0) + f32(0.5))
    return np.clip(np.where(np.isnan(q), f32(0.0), q), 0, 255).astype(np.uint8)


def _texture(tex, s, t):
    Th, Tw = tex.shape[:2]
    T = tex.astype(f32)
    x = s * f32(Tw) - f32(0.5)
    y = t * f32(Th) - f32(0.5)
    x0 = np.floor(x)
    y0 = np.floor(y)
    fx = (x - x0)[..., None]
    fy = (y - y0)[..., None]
    ix0 = np.clip(x0.astype(np.int64), 0, Tw - 1)
    ix1 = np.clip(x0.astype(np.int64) + 1, 0, Tw - 1)
    iy0 = np.clip(y0.astype(np.int64), 0, Th - 1)
    iy1 = np.clip(y0.astype(np.int64) + 1, 0, Th - 1)
    top = _lerp(T[iy0, ix0], T[iy0, ix1], fx)
    bot = _lerp(T[iy1, ix0], T[iy1, ix1], fx)
    c = _lerp(top, bot, fy)
    return np.clip(np.floor(c + f32(0.5)), 0, 255).astype(np.uint8)


def space_map(field, levels, dims, mode, line_width=1.0, fade=(2.0, 6.0, 3), lo=None, hi=None, texture=None):
    """RGBA8 image (H, W, 4) of the field (D, H, W) float32/float64 with
    levels (D, L) float64, showing the planes `dims` (one or two)."""
    field = np.asarray(field)
    dims = list(dims)
    H, W = field.shape[1:]
    lo = [0.0] * len(dims) if lo is None else list(lo)
    hi = [1.0] * len(dims) if hi is None else list(hi)
    terms = [dim_terms(field[d], np.asarray(levels[d], np.float64), line_width,
                       fade if mode == ADAPTIVE else None) for d in dims]
    L = np.asarray(levels).shape[1]
    valid = np.all([~np.isnan(field[d]) for d in dims], axis=0)
    draw_lines = mode in (LINES, DISCRETE_LINES, ADAPTIVE, GRADIENT)
    cov = np.zeros((H, W), f32)
    if draw_lines:
        for _, _, c in terms:
            cov = np.maximum(cov, c)
    black = np.zeros(3, f32)
    if mode in (DISCRETE, DISCRETE_LINES):
        s = [(b.astype(f32) + f32(0.5)) * _recip(f32(L + 1)) for _, b, _ in terms]
        col = _ramp(s[0]) if len(dims) == 1 else _corner(s[0], s[1])
    elif mode in (GRADIENT, TEXTURE):
        s = [_clamp01((g - f32(l)) * _recip(f32(h) - f32(l))) for (g, _, _), l, h in zip(terms, lo, hi)]
        if mode == TEXTURE:
            t = s[1] if len(dims) == 2 else np.full((H, W), f32(0.5), f32)
            # transparent pixels (NaN coordinates) look up texel 0, then are cleared
            rgba = _texture(np.asarray(texture), np.where(valid, s[0], f32(0.0)), np.where(valid, t, f32(0.0)))
            rgba[~valid] = 0
            return rgba
        col = _ramp(s[0]) if len(dims) == 1 else _corner(s[0], s[1])
    else:
        col = np.ones((H, W, 3), f32)
    if draw_lines:
        col = _lerp(col, black, cov[..., None])
    out = np.empty((H, W, 4), np.uint8)
    out[..., :3] = _to_byte(col)
    out[..., 3] = 255
    out[~valid] = 0
    return out
