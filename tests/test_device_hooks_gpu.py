"""Device self-checks through the C ABI test hooks: the bounded wait of the
tensor-core kernel gives up with an error code instead of hanging, and the
double-float weight functions of the hand-over path reach ~1e-13."""
import ctypes

import numpy as np
import pytest

from paper_1408_0677_gb300 import _abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return _abi.load()


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _df_args(a64):
    hi = a64.astype(np.float32)
    lo = (a64 - hi.astype(np.float64)).astype(np.float32)
    return hi, lo, hi.astype(np.float64) + lo.astype(np.float64)


def _run(lib, kind, hi, lo):
    out = np.empty(hi.shape[0], np.float64)
    assert lib.mls_debug_df_weight(kind, _ptr(hi), _ptr(lo), hi.shape[0], _ptr(out)) == _abi.MLS_OK
    return out


def test_wait_gives_up_with_error_code_and_context_survives(lib):
    code = ctypes.c_int(-1)
    # 1 ms limit on an mbarrier phase that nothing completes
    assert lib.mls_debug_wait_selftest(1_000_000, ctypes.byref(code)) == _abi.MLS_OK
    assert code.value == 1
    # the context is still usable afterwards
    hi, lo, a = _df_args(np.array([-1.0, 0.0]))
    np.testing.assert_allclose(_run(lib, 0, hi, lo), np.exp(a), rtol=1e-13)


def test_df_exp_relative_error(lib):
    rng = np.random.default_rng(5)
    a64 = np.concatenate([-rng.uniform(0, 70, 200_000), -rng.uniform(0, 1e-3, 1000), rng.uniform(0, 1, 1000),
                          [0.0, -40.0, -70.0, 1.0], -np.log(2) / 128 * np.arange(1, 200)])
    hi, lo, a = _df_args(a64)
    out = _run(lib, 0, hi, lo)
    rel = np.abs(out / np.exp(a) - 1.0)
    assert rel.max() < 5e-14, rel.max()


def test_df_wendland_and_sqrt(lib):
    rng = np.random.default_rng(6)
    r2 = np.concatenate([rng.uniform(0, 0.98, 100_000), [0.0, 1e-12, 0.25, 0.5]])
    hi, lo, a = _df_args(r2)
    q = np.sqrt(a)
    np.testing.assert_allclose(_run(lib, 2, hi, lo), q, rtol=2e-14, atol=1e-20)
    w = (1 - q) ** 4 * (4 * q + 1)
    np.testing.assert_allclose(_run(lib, 1, hi, lo), w, rtol=1e-11, atol=1e-15)
