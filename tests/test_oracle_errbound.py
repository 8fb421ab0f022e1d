"""The oracle's rounding-error bound holds, and is not vacuous.

oracle.mls(..., ebound=True) returns, per value, the coefficients of a
first-order bound on how far an FP64 evaluation of the fit (Section 3.3: the
weighted least-squares fit evaluated at the pixel) can be from the exact
value of the same inputs:  |f - f_exact| <= (N + 12) u A + B, with N the
longest summation chain and u = 2^-53.  The GPU parity tests widen the FP64
tolerance by this bound (for both sides) where it exceeds 1e-10 of the data
range, so the bound itself is pinned here against an independent evaluation
in 40-digit decimal arithmetic: weights, moments and the solve all carried
far beyond FP64, on tiny cases that include badly conditioned pixels far
from the data (extrapolation) and points near the Wendland support edge.
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
from oracle import oracle as orc

G, WD, ID = orc.GAUSS, orc.WENDLAND, orc.INVDIST
U = 2.0 ** -53


def _exact_fit(xy, F, degree, weight, h, alpha, px, py):
    """The fit at (px, py) in 40-digit decimals: every FP64 input is taken as
    the exact number it holds; h^2 is the FP64 product h*h that any FP64
    evaluation uses (a fit with that kernel width is the reference)."""
    getcontext().prec = 40
    X = [Decimal(float(v)) for v in xy[:, 0]]
    Y = [Decimal(float(v)) for v in xy[:, 1]]
    P, Q = Decimal(float(px)), Decimal(float(py))
    h2 = Decimal(float(h * h))
    hd = Decimal(float(h))
    r2 = [(x - P) ** 2 + (y - Q) ** 2 for x, y in zip(X, Y)]
    m = min(r2)
    w = []
    for r in r2:
        if weight == G:
            w.append((-(r - m) / h2).exp())
        elif weight == WD:
            if r < hd * hd:
                q = r.sqrt() / hd
                w.append((1 - q) ** 4 * (4 * q + 1))
            else:
                w.append(Decimal(0))
        else:
            w.append((m / r) ** Decimal(float(alpha)))
    inv_s = Decimal(float(1.0 / h))   # the basis scale only changes conditioning
    k = (degree + 1) * (degree + 2) // 2
    n, D = F.shape
    M = [[Decimal(0)] * k for _ in range(k)]
    R = [[Decimal(0)] * D for _ in range(k)]
    for i in range(n):
        if w[i] == 0:
            continue
        dx, dy = (X[i] - P) * inv_s, (Y[i] - Q) * inv_s
        b = [Decimal(1), dx, dy, dx * dx, dx * dy, dy * dy][:k]
        for a in range(k):
            for c in range(k):
                M[a][c] += w[i] * b[a] * b[c]
            for d in range(D):
                R[a][d] += w[i] * b[a] * Decimal(float(F[i, d]))
    # Gaussian elimination with partial pivoting on [M | R]
    A = [M[a][:] + R[a][:] for a in range(k)]
    for j in range(k):
        piv = max(range(j, k), key=lambda r: abs(A[r][j]))
        A[j], A[piv] = A[piv], A[j]
        for r in range(j + 1, k):
            f = A[r][j] / A[j][j]
            A[r] = [A[r][c] - f * A[j][c] for c in range(k + D)]
    C = [[Decimal(0)] * D for _ in range(k)]
    for j in range(k - 1, -1, -1):
        for d in range(D):
            s = A[j][k + d] - sum(A[j][c] * C[c][d] for c in range(j + 1, k))
            C[j][d] = s / A[j][j]
    return np.array([float(C[0][d]) for d in range(D)])


CASES = [
    # seed, n, D, degree, weight, h, alpha, view (pixels far outside the data are badly conditioned)
    (1, 12, 3, 2, G, 0.15, 1.0, (-0.6, -0.4, 1.7, 1.5)),
    (2, 9, 2, 1, G, 0.08, 1.0, (-1.0, -1.0, 2.0, 2.0)),
    (3, 25, 2, 2, WD, 0.35, 1.0, (0.0, 0.0, 1.0, 1.0)),
    (4, 14, 2, 1, ID, 0.3, 1.0, (-0.5, 0.0, 1.5, 1.0)),
    (5, 10, 4, 2, G, 0.4, 1.0, (-3.0, -3.0, 4.0, 4.0)),
]


@pytest.mark.parametrize("case", CASES, ids=[f"e{c[0]}" for c in CASES])
def test_first_order_bound_holds_against_decimal_evaluation(case):
    seed, n, D, degree, weight, h, alpha, view = case
    rng = np.random.default_rng(seed)
    xy = 0.3 + 0.4 * rng.random((n, 2))
    F = rng.standard_normal((n, D)) + 3.0 * xy[:, :1]
    W = H = 7
    ref = oracle.mls(xy, F, degree, weight, h, W, H, view=view, alpha=alpha, ebound=True)
    x0, y0, x1, y1 = view
    sx, sy = (x1 - x0) / W, (y1 - y0) / H
    checked = 0
    worst = 0.0
    for q in range(W * H):
        if ref.deg_used[q] != degree or np.isnan(ref.field[q]).any():
            continue     # the degree policy chose a lower degree: a different fit
        u, v = q % W, q // W
        px, py = x0 + (u + 0.5) * sx, y0 + (v + 0.5) * sy
        ex = _exact_fit(xy, F, degree, weight, h, alpha, px, py)
        bound = (ref.count[q] + 12) * U * ref.ecoef_sum[q] + ref.ecoef_fix[q]
        err = np.abs(ref.field[q] - ex)
        assert (err <= bound).all(), (q, err, bound, ref.rcond[q])
        worst = max(worst, float((err / bound).max()))
        checked += 1
    assert checked >= 10
    print(f"case {seed}: {checked} pixels, largest error / bound {worst:.3g}")


def test_bound_is_tight_enough_to_matter():
    """Inside the data the bound sits near the FP64 resolution of the values
    (far below the 1e-10 parity tolerance); far outside it, where the fit
    extrapolates from a few dominant points, it grows with the condition of
    the moment matrix."""
    rng = np.random.default_rng(9)
    xy = rng.random((200, 2))
    F = np.sin(3 * xy[:, :1]) + xy[:, 1:] ** 2
    W = 24
    ref = oracle.mls(xy, F, 2, G, 0.1, W, W, view=(-0.5, -0.5, 1.5, 1.5), ebound=True)
    S = F.max() - F.min()
    b = ((ref.count + 12) * U * ref.ecoef_sum[:, 0] + ref.ecoef_fix[:, 0]) / S
    u, v = np.arange(W * W) % W, np.arange(W * W) // W
    inner = (u >= 6) & (u < 18) & (v >= 6) & (v < 18)     # pixel centres inside [0,1]^2
    assert np.percentile(b[inner], 90) < 1e-12
    assert b[inner].max() < 1e-10
    assert b[~inner].max() > 1e3 * np.percentile(b[inner], 90)
    # the bound follows the conditioning (rank correlation over the pixels)
    ok = np.isfinite(b) & (ref.rcond > 0)
    ra = np.argsort(np.argsort(b[ok]))
    rb = np.argsort(np.argsort(-np.log(ref.rcond[ok])))
    assert np.corrcoef(ra, rb)[0, 1] > 0.5
