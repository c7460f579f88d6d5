"""Failure detection on the GPU without a fault: a bounded device-side wait on
a barrier that nothing completes runs out, the kernel reports
LBM_ERR_TIMEOUT through its status word, and the context stays usable."""
import time

import numpy as np
import pytest

from paper_1109_6672_gb300 import inputs
from paper_1109_6672_gb300 import lbm

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports_timeout():
    t0 = time.perf_counter()
    st = lbm.lbm_selftest_wait(20_000_000)  # 20 ms
    dt = time.perf_counter() - t0
    assert st == lbm.LBM_ERR_TIMEOUT
    assert dt >= 0.02
    # the context still works afterwards
    p, f = inputs.couette(ny=9, precision=lbm.LBM_P_FP32)
    g = lbm.Lbm(p).init(*f).step(5)
    rho, ux, uy, T = g.moments()
    assert np.isfinite(rho).all() and abs(rho.mean() - 1.0) < 1e-5
    g.close()
