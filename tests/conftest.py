import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter):
    """Per parity comparison: pixels compared, how many needed an allowance
    above the tolerance (ill-conditioned fits, FP64 rounding-error bound),
    the largest error in units of the data range, and the largest error as a
    fraction of what was allowed."""
    try:
        from tests.gpu_util import ALLOWANCE_LOG
    except Exception:
        return
    if not ALLOWANCE_LOG:
        return
    tr = terminalreporter
    tr.section("parity allowances")
    tr.write_line(f"{'test':72s} {'prec':5s} {'pixels':>8s} {'allow>tol':>9s} {'max err':>9s} {'err/allow':>9s}")
    for name, prec, npx, na, err, ratio in ALLOWANCE_LOG:
        tr.write_line(f"{name[-72:]:72s} {prec:5s} {npx:8d} {na:9d} {err:9.2e} {ratio:9.3f}")
