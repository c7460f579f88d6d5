"""The allocation-free conserved-sums entry point (lbm_conserved_noalloc)
against the allocating one (lbm_conserved), on two calls in a row.

It exists for callers that cannot allocate device memory when they need the
sums (stream capture, pool-owned device memory, latency-bound loops).  Here
the test owns all device memory through torch; the entry point under test
receives the state buffer and the output location and allocates nothing.
This file is collected last so that a failure here stops a run only after
every other test has run.
"""
import numpy as np
import pytest

from paper_1109_6672_gb300 import inputs
from paper_1109_6672_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [lbm.LBM_P_FP64, lbm.LBM_P_FP32, lbm.LBM_P_FP32_FP16,
                                       lbm.LBM_P_FP32_BF16])
def test_noalloc_matches_lbm_conserved(precision):
    torch = pytest.importorskip("torch")
    p = inputs.base_params(300, 77, tau_f=0.35, tau_h=0.5, precision=precision,
                           bc=[inputs.WALL_ISOTHERMAL, inputs.WALL_ISOTHERMAL,
                               inputs.WALL_ADIABATIC, inputs.WALL_ADIABATIC],
                           T_wall=[1.1, 0.9, 1.0, 1.0], energy_model=inputs.E_INTERNAL, b=5.0,
                           g=1e-4)
    fields = inputs.uniform_fields(p["nx"], p["ny"], seed=9, u_amp=0.02, T_amp=0.05,
                                   rho_amp=0.02)
    nbytes = lbm.lbm_state_bytes(p)
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    g = lbm.Lbm(p, device_buffer=buf.data_ptr(), nbytes=nbytes).init(*fields)
    for steps in (7, 10):  # two calls in a row, the state in each of the two buffers
        g.step(steps)
        ref = g.conserved()
        k = g.steps_done
        d_state = buf.data_ptr() + (k % 2) * (nbytes // 2)
        lbm.lbm_conserved_noalloc(p, d_state, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    g.close()


def test_noalloc_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    p = inputs.base_params(16, 16)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError):
        lbm.lbm_conserved_noalloc(p, 0, out.data_ptr())
    with pytest.raises(lbm.LbmError):
        lbm.lbm_conserved_noalloc(dict(p, tau_f=-1.0), out.data_ptr(), out.data_ptr())
