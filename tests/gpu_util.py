"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
compare with the FP64 oracle under the tolerances of the method:
|f_gpu - f_oracle| <= tol * S_d with S_d the data range of dimension d
(1e-10 for the FP64 path, 1e-3 for FP32 and the tensor-core precisions);
band labels bit-exact except where the oracle value lies within that
tolerance of an iso-level; pixels the oracle flags as ambiguous (a
degeneracy decision within a factor 100 of its threshold, or a point on the
support boundary that can change the support count) are left out."""
import numpy as np

TOL = {"fp64": 1e-10, "fp32": 1e-3, "fp16": 1e-3, "bf16": 1e-3}


def gpu_render(wl, precision, device_inputs=True, levels=True, operand_cut=True, **kw):
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
    out = r.render(wl.W, wl.H, view=wl.view, levels=wl.levels if levels else None)
    stats = r.sync()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    res["stats"] = stats
    r.close()
    return res


def compare(wl, res, ref, precision, pixels=None, check_bands=True, check_status=True):
    """Assert parity; returns (max error / range, number of pixels compared)."""
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
    # the FP64 path may differ by kappa * eps where the moment matrix is ill conditioned
    allow = np.full(err.shape[0], tol)
    if precision == "fp64":
        # a different but equally valid summation order moves an FP64 result by
        # about kappa * eps (kappa = 1/rcond of the equilibrated moment matrix)
        kappa = np.where(ref.rcond > 0, 1.0 / np.maximum(ref.rcond, 1e-300), 1.0)
        allow = np.maximum(tol, 30.0 * kappa * 2.2e-16)
    bad = (err > allow[:, None]) & ok[:, None]
    if bad.any():
        i, d = np.argwhere(bad)[0]
        raise AssertionError(f"{precision}: {bad.sum()} values out of tolerance; first pixel {i} dim {d}: "
                             f"gpu {f[i, d]!r} oracle {ref.field[i, d]!r} err {err[i, d]:.3g} "
                             f"(rcond {ref.rcond[i]:.3g}, deg {ref.deg_used[i]})")
    if check_status and st is not None:
        sti = st.astype(np.int32)
        deg = np.where(sti & 0x04, -1, sti & 0x03).astype(np.int8)
        mism = (deg != ref.deg_used) & ok
        assert not mism.any(), f"degree used differs at {np.argwhere(mism)[:5].ravel()}"

    if check_bands and b is not None:
        import oracle
        bo = oracle.bands(ref.field, wl.levels)
        near = np.zeros_like(bo, dtype=bool)
        for j in range(wl.levels.shape[1]):
            near |= np.abs(ref.field - wl.levels[:, j][None, :]) <= tol * S[None, :]
        diff = (bo != b) & ~near & ok[:, None]
        assert not diff.any(), f"{diff.sum()} band labels differ away from iso-levels"
    return float(np.where(ok[:, None], err, 0).max()), int(ok.sum())
