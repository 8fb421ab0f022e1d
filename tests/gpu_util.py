"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
compare with the FP64 oracle under the tolerances of the method:
|f_gpu - f_oracle| <= tol * S_d with S_d the data range of dimension d
(1e-10 for the FP64 path, 1e-3 for FP32 and the tensor-core precisions);
band labels bit-exact except where the oracle value lies within that
tolerance of an iso-level; pixels the oracle flags as ambiguous (a
degeneracy decision within a factor 100 of its threshold, or a point on the
support boundary that can change the support count) are left out.

Where the fit itself is badly conditioned, no FP64 evaluation is held to
1e-10: both sides are allowed the oracle's first-order rounding-error bound
for an FP64 evaluation of that value (oracle.mls(..., ebound=True)),

    |f - f_exact| <= (N + 12) u A + B,     u = 2^-53,

with N the longest summation chain of the side: the number of points with a
positive weight for the oracle (it sums them in order), at most that number
or ceil(n / 32), plus the five butterfly levels, for the GPU's FP64 kernel
(one warp per pixel, lane-strided partial sums).  Every comparison counts
the pixels that use an allowance above the tolerance and asserts that they
stay below a stated fraction of the pixels compared; the counts are printed
at the end of the session.  Reduced precisions add the oracle's own bound
to their 1e-3."""
import numpy as np

TOL = {"fp64": 1e-10, "fp64tc": 1e-10, "fp32": 1e-3, "fp16": 1e-3, "bf16": 1e-3}
# The FP64 emulation on tensor cores (fp64tc) has no long summation chain
# (its digit products are summed exactly in FP32); its error model is a
# relative error of 2^-40 on every weight and operand entry (double-float
# weights and products, 60-bit fixed-point digits), which enters the bound
# like a chain of 2^-40 / u = 8192 additions, plus 64 for the FP64
# combination of the diagonals, the frame shift and the solve.
CHAIN_FP64TC = 8192 + 64
U = 2.0 ** -53
# one line per comparison: (test, precision, pixels compared, pixels with an
# allowance above the tolerance, largest error / range, largest error / allowance)
ALLOWANCE_LOG = []


def oracle_ref(wl, pixels=None):
    """The oracle at the listed pixels with its rounding-error bound."""
    import oracle
    return oracle.mls(wl.xy, wl.F, wl.degree, wl.weight, wl.h, wl.W, wl.H, view=wl.view, pixels=pixels,
                      alpha=wl.alpha, trunc=wl.trunc, ebound=True)


def allowance(wl, ref, precision):
    """Per (pixel, dimension) tolerance in units of the data range S_d:
    max(tol, bound) for FP64 (both sides' rounding-error bounds), tol plus
    the oracle's own bound for the reduced precisions."""
    tol = TOL[precision]
    S = wl.F.max(0) - wl.F.min(0)
    S = np.where(S > 0, S, 1.0)
    if ref.ecoef_sum is None:
        raise ValueError("compare() needs the oracle's error bound: call oracle_ref()")
    cnt = ref.count.astype(np.float64)[:, None]
    b_or = ((cnt + 12) * U * ref.ecoef_sum + ref.ecoef_fix) / S[None, :]
    b_or = np.where(np.isfinite(b_or), b_or, 0.0)
    if precision in ("fp64", "fp64tc"):
        chain_gpu = (np.minimum(cnt, np.ceil(wl.n / 32.0)) + 5 if precision == "fp64"
                     else np.full_like(cnt, CHAIN_FP64TC))
        b_gpu = ((chain_gpu + 12) * U * ref.ecoef_sum + ref.ecoef_fix) / S[None, :]
        b_gpu = np.where(np.isfinite(b_gpu), b_gpu, 0.0)
        return np.maximum(tol, b_or + b_gpu)
    return tol + b_or


def gpu_render(wl, precision, device_inputs=True, levels=True, operand_cut=True, handover_split=None, **kw):
    import ctypes

    import torch

    from paper_1408_0677_gb300 import Renderer, _abi
    if device_inputs:
        xy, F = torch.from_numpy(wl.xy).cuda(), torch.from_numpy(wl.F).cuda()
    else:
        xy, F = wl.xy, wl.F
    r = Renderer(xy, F, degree=wl.degree, weight=wl.weight, h=wl.h, precision=precision, alpha=wl.alpha,
                 support=wl.trunc, **kw)
    if not operand_cut:
        assert _abi.load().mls_debug_operand_cut(ctypes.c_void_p(r.handle), 0) == _abi.MLS_OK
    if handover_split is not None:
        cap, least = handover_split
        assert _abi.load().mls_debug_handover_split(ctypes.c_void_p(r.handle), int(cap), int(least)) == _abi.MLS_OK
    out = r.render(wl.W, wl.H, view=wl.view, levels=wl.levels if levels else None)
    stats = r.sync()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    res["stats"] = stats
    r.close()
    return res


# Largest fraction of the compared pixels that may need an allowance above
# the tolerance, unless a test states its own: FP64 pixels whose two-sided
# rounding bound exceeds 1e-10 of the range; for the reduced precisions,
# pixels where the oracle's own bound exceeds a tenth of 1e-3 (far from the
# data, where the fit extrapolates from a few dominant weights)
MAX_ALLOW_FRAC = {"fp64": 0.05, "fp64tc": 0.05, "fp32": 0.10, "fp16": 0.10, "bf16": 0.10}


def compare(wl, res, ref, precision, pixels=None, check_bands=True, check_status=True, max_allow_frac=None):
    """Assert parity; returns (max error / range, number of pixels compared).
    max_allow_frac: the largest fraction of the compared pixels that may
    need an allowance above the tolerance (ill-conditioned fits); None takes
    MAX_ALLOW_FRAC[precision]."""
    import os
    if max_allow_frac is None:
        max_allow_frac = MAX_ALLOW_FRAC[precision]
    D = wl.D
    f = res["field"].astype(np.float64).reshape(D, -1).T
    st = res["status"].reshape(-1) if res["status"] is not None else None
    b = res["bands"].reshape(D, -1).T if res.get("bands") is not None else None
    if pixels is not None:
        f = f[pixels]
        st = st[pixels] if st is not None else None
        b = b[pixels] if b is not None else None
    tol = TOL[precision]
    S = wl.F.max(0) - wl.F.min(0)
    S = np.where(S > 0, S, 1.0)
    ok = ref.amb == 0
    nan_or = np.isnan(ref.field)
    nan_gpu = np.isnan(f)
    assert np.array_equal(nan_or[ok], nan_gpu[ok]), "NaN (no support) pixels differ"
    err = np.abs(f - ref.field) / S[None, :]
    err = np.where(nan_or, 0.0, err)
    allow = allowance(wl, ref, precision)
    widened = ((allow > tol * (1.0 if precision in ("fp64", "fp64tc") else 1.1)) & ~nan_or).any(axis=1) & ok
    n_allow = int(widened.sum())
    npx = int(ok.sum())
    bad = (err > allow) & ok[:, None]
    ratio = float(np.where(ok[:, None], err / allow, 0).max()) if npx else 0.0
    ALLOWANCE_LOG.append((os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], precision, npx, n_allow,
                          float(np.where(ok[:, None], err, 0).max()) if npx else 0.0, ratio))
    if bad.any():
        i, d = np.argwhere(bad)[0]
        raise AssertionError(f"{precision}: {bad.sum()} values out of tolerance; first pixel {i} dim {d}: "
                             f"gpu {f[i, d]!r} oracle {ref.field[i, d]!r} err {err[i, d]:.3g} "
                             f"allowed {allow[i, d]:.3g} (rcond {ref.rcond[i]:.3g}, deg {ref.deg_used[i]})")
    assert n_allow <= max_allow_frac * max(npx, 1), \
        f"{precision}: {n_allow} of {npx} pixels need an allowance above {tol} (stated limit {max_allow_frac})"
    if check_status and st is not None:
        sti = st.astype(np.int32)
        deg = np.where(sti & 0x04, -1, sti & 0x03).astype(np.int8)
        mism = (deg != ref.deg_used) & ok
        assert not mism.any(), f"degree used differs at {np.argwhere(mism)[:5].ravel()}"

    if check_bands and b is not None:
        import oracle
        bo = oracle.bands(ref.field, wl.levels)
        near = np.abs(ref.field[:, :, None] - wl.levels[None, :, :]) <= (allow * S[None, :])[:, :, None]
        near = near.any(axis=2)
        diff = (bo != b) & ~near & ok[:, None]
        assert not diff.any(), f"{diff.sum()} band labels differ away from iso-levels"
    return float(np.where(ok[:, None], err, 0).max()), npx
