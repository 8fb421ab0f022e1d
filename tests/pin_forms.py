"""Independent closed forms used to pin the FP64 oracle.

None of these shares code with ``oracle/`` or with the CUDA path.  Each is a
different route to the same mathematical quantity:

* ``wls_lstsq`` solves the weighted least-squares problem by an SVD-based
  least-squares solver on sqrt(w) B c = sqrt(w) f (no normal equations);
* ``affine_centroid`` is the paper's affine MLS, Eq. eq-affinemls, written
  with the weighted centroids of Eqs. eq-pstar and eq-qstar and a 2x2 inverse;
* ``shepard`` is the weighted mean of Section 3.3.1 (Eq. eq-meanmls read on
  data values, without the displacement term).
"""
import numpy as np


def pixel_centres(W, H, view=(0.0, 0.0, 1.0, 1.0)):
    x0, y0, x1, y1 = view
    u = np.arange(W)
    v = np.arange(H)
    px = x0 + (u + 0.5) * ((x1 - x0) / W)
    py = y0 + (v + 0.5) * ((y1 - y0) / H)
    PX, PY = np.meshgrid(px, py)          # [H][W]
    return PX.ravel(), PY.ravel()


def weights_gauss(r2, h):
    return np.exp(-r2 / h ** 2)


def weights_wendland(r2, rho):
    q = np.sqrt(r2) / rho
    return np.where(q < 1.0, (1.0 - q) ** 4 * (4.0 * q + 1.0), 0.0)


def weights_invdist(r2, alpha):
    return 1.0 / r2 ** alpha


def monomials(dx, dy, degree):
    cols = [np.ones_like(dx)]
    if degree >= 1:
        cols += [dx, dy]
    if degree >= 2:
        cols += [dx ** 2, dx * dy, dy ** 2]
    return np.stack(cols, axis=-1)


def wls_lstsq(xy, F, p, w, degree, s=1.0):
    """Weighted LS polynomial fit evaluated at p, by SVD least squares."""
    dx = (xy[:, 0] - p[0]) / s
    dy = (xy[:, 1] - p[1]) / s
    B = monomials(dx, dy, degree)
    sw = np.sqrt(w)[:, None]
    c, *_ = np.linalg.lstsq(sw * B, sw * F, rcond=None)
    return c[0]


def affine_centroid(xy, F, p, w):
    """Eq. eq-affinemls: (p - p*) (sum w phat^T phat)^-1 sum w phat^T qhat + q*."""
    sw = w.sum()
    pstar = (w[:, None] * xy).sum(0) / sw
    qstar = (w[:, None] * F).sum(0) / sw
    ph = xy - pstar
    qh = F - qstar
    A = np.zeros((2, 2))
    Bm = np.zeros((2, F.shape[1]))
    for i in range(xy.shape[0]):
        A += w[i] * np.outer(ph[i], ph[i])
        Bm += w[i] * np.outer(ph[i], qh[i])
    a, b, c, d = A[0, 0], A[0, 1], A[1, 0], A[1, 1]
    det = a * d - b * c
    Ainv = np.array([[d, -b], [-c, a]]) / det
    return (p - pstar) @ Ainv @ Bm + qstar


def shepard(F, w):
    return (w[:, None] * F).sum(0) / w.sum()
