"""Planted mistakes in the oracle must fail at least one pin.

Each case copies oracle/mls_oracle.c to a temporary directory, applies one
plausible mistake (a dropped term, a wrong exponent, an off-by-half pixel
centre, a transposed operand, a wrong tie rule ...), compiles it with gcc and
runs the pin battery of test_oracle_pins.py against the variant.  The
mistake is planted on the CPU only; the committed oracle is untouched.
"""
import os
import subprocess
import tempfile

import pytest

import oracle
from oracle import oracle as orc
from tests import test_oracle_pins as pins

G, WD, ID = orc.GAUSS, orc.WENDLAND, orc.INVDIST

MUTANTS = [
    ("cross term dropped from the basis", "case 4: return dx * dy;", "case 4: return dx * dx;"),
    ("Gaussian on r instead of r^2", "w = exp(-(r2[i] - m) / h2);", "w = exp(-(sqrt(r2[i]) - sqrt(m)) / h);"),
    ("Wendland (1-q)^3", "w = t * t * t * t * (4.0 * qd + 1.0);", "w = t * t * t * (4.0 * qd + 1.0);"),
    ("inverse distance 1/r^(4 alpha)", "w = pow(m / r2[i], alpha);", "w = pow(m / r2[i], 2.0 * alpha);"),
    ("pixel centre without the half offset", "((double)u + 0.5) * s;", "((double)u) * s;"),
    ("fit read from the wrong coefficient", "sdiag[0] * Minv[c * k + 0]", "sdiag[k - 1] * Minv[c * k + k - 1]"),
    ("band tie counted below", "if (levels[d * L + j] <= f) c++;", "if (levels[d * L + j] < f) c++;"),
    ("value matrix read transposed", "Rbuf[a * D + d] += w * b[a] * F[i * D + d];",
     "Rbuf[a * D + d] += w * b[a] * F[d * n + i];"),
    ("weight dropped from M", "M[a * k + c] += w * b[a] * b[c];", "M[a * k + c] += b[a] * b[c];"),
    ("degeneracy test inverted", "if (!(rc >= rcond_min)) ok = 0;", "if (!(rc <= rcond_min)) ok = 0;"),
    ("Wendland support test off", "if (r2[i] < rho2) {", "if (r2[i] < 4.0 * rho2) {"),
    ("truncated box on one axis", "in_box = ax < rho_box && ay < rho_box;", "in_box = ax < rho_box;"),
    ("truncated box edge counted in", "in_box = ax < rho_box && ay < rho_box;", "in_box = ax <= rho_box && ay <= rho_box;"),
    ("truncated box half-width c h^2", "const double rho_box = trunc * h;", "const double rho_box = trunc * h * h;"),
]


def _battery():
    yield lambda: [pins.test_polynomial_reproduction(w, h, d)
                   for (w, h) in [(G, 0.2), (WD, 0.6), (ID, 0.3)] for d in (0, 1, 2)]
    yield lambda: [pins.test_degree0_is_weighted_mean(w, h, a)
                   for (w, h, a) in [(G, 0.15, 1.0), (WD, 0.45, 1.0), (ID, 0.1, 0.8)]]
    yield pins.test_affine_equals_paper_centroid_form
    yield pins.test_dimension_independence
    yield pins.test_small_h_is_nearest_neighbour_with_degree_fallback
    yield pins.test_wendland_single_point_and_empty_support
    yield pins.test_idw_point_identity
    yield pins.test_bands_definition_and_ties
    yield pins.test_golden_idw_two_points
    yield pins.test_golden_gauss_two_points
    yield lambda: [pins.test_golden_plane_four_points(w) for w in (G, WD, ID)]
    yield lambda: [pins.test_brute_force_tiny_cases(s) for s in range(6)]
    from tests import test_oracle_trunc as tp
    yield tp.test_box_not_disc_and_strict_edge
    yield tp.test_equals_full_sum_over_the_points_in_the_box
    yield tp.test_box_holding_every_point_is_the_full_sum


VARIANT_MUTANTS = [
    ("perpendicular of dp with the wrong sign", "{{dp[0], dp[1]}, {dp[1], -dp[0]}}",
     "{{dp[0], dp[1]}, {-dp[1], dp[0]}}"),
    ("mean form without the pixel centre", "out[0] = vx + (sq[0] - sp[0]) / sw;", "out[0] = (sq[0] - sp[0]) / sw;"),
    ("undetermined rotation collapses to q*", "out[0] = dv[0] + qs[0];", "out[0] = qs[0];"),
    ("rigid result not rescaled to |dv|", "out[0] = ndv * fp[0] / nfp + qs[0];", "out[0] = fp[0] / nfp + qs[0];"),
    ("q centroid from the positions", "sq[0] += w * Q[2 * i];", "sq[0] += w * xy[2 * i];"),
]


def _variant_battery():
    from tests import test_oracle_variants as vp
    yield lambda: [vp.test_rigid_reproduces_rigid_motions(w, h) for (w, h) in vp.GW]
    yield lambda: [vp.test_identity_when_nothing_is_distorted(w, h, v) for (w, h) in vp.GW
                   for v in (oracle.VARIANT_RIGID, oracle.VARIANT_MEAN)]
    yield lambda: [vp.test_mean_reproduces_translations(w, h) for (w, h) in vp.GW]
    yield vp.test_mean_is_pixel_plus_weighted_mean_displacement
    yield vp.test_rigid_equals_best_weighted_rotation_by_search
    yield lambda: [vp.test_single_point_support_is_a_translation(v)
                   for v in (oracle.VARIANT_RIGID, oracle.VARIANT_MEAN)]
    yield vp.test_coincident_support_is_a_translation


def _caught_by(battery, old, new, monkeypatch):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "mls_oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    with tempfile.TemporaryDirectory() as tmp:
        path_c = os.path.join(tmp, "mut.c")
        path_so = os.path.join(tmp, "libmut.so")
        open(path_c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", path_so, path_c, "-lm"])
        monkeypatch.setattr(orc, "_lib", orc.load_library(path_so))
        for check in battery():
            try:
                check()
            except (AssertionError, ValueError, FloatingPointError):
                return True
    return False


@pytest.mark.parametrize("name,old,new", VARIANT_MUTANTS, ids=[m[0] for m in VARIANT_MUTANTS])
def test_planted_variant_mistake_is_caught(name, old, new, monkeypatch):
    assert _caught_by(_variant_battery, old, new, monkeypatch), f"no pin caught the planted mistake: {name}"


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, monkeypatch):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "mls_oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    with tempfile.TemporaryDirectory() as tmp:
        path_c = os.path.join(tmp, "mut.c")
        path_so = os.path.join(tmp, "libmut.so")
        open(path_c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", path_so, path_c, "-lm"])
        monkeypatch.setattr(orc, "_lib", orc.load_library(path_so))
        caught = []
        for check in _battery():
            try:
                check()
            except (AssertionError, ValueError, FloatingPointError) as e:  # noqa: PERF203
                caught.append(type(e).__name__)
                break
        assert caught, f"no pin caught the planted mistake: {name}"
