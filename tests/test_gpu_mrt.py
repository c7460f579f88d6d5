"""The MRT collision (Eqs. 43-45) on the CUDA path against the oracle's MRT
scheme, on the same cases, launch shapes and tolerances as the BGK parity
tests; its reduction to BGK at uniform rates; MRT grids in a batch; and the
variant that is built for BGK only."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs
from paper_1109_6672_gb300 import lbm
from test_gpu_parity import CASES, make_case, rel

pytestmark = pytest.mark.gpu

RATES = dict(collision=lbm.LBM_COLL_MRT, s_e=1.3, s_eps=1.1, s_q=1.6)


def run_mrt(name, precision, steps, launch=None, rates=RATES):
    p, fields = make_case(name, precision)
    p = dict(p, **rates)
    o = orc.Oracle(p).init(*fields).step(steps)
    g = lbm.Lbm(p)
    if launch:
        g.set_launch(*launch)
    g.init(*fields).step(steps)
    return p, fields, o, g


@pytest.mark.parametrize("launch", [None, (1, 3), (64, 7)])
@pytest.mark.parametrize("name", sorted(CASES))
def test_mrt_fp64_parity(name, launch):
    p, _, o, g = run_mrt(name, lbm.LBM_P_FP64, 60, launch)
    assert rel(g.pops(), o.pops()) <= 1e-12
    np.testing.assert_allclose(g.conserved(), o.conserved(), rtol=1e-12, atol=1e-12)
    g.close()


@pytest.mark.parametrize("name", ["periodic_total", "couette_walls", "cavity", "all_iso_moving"])
def test_mrt_fp32_and_16bit(name):
    _, _, o, g = run_mrt(name, lbm.LBM_P_FP32, 50)
    assert rel(g.pops(), o.pops()) <= 2e-5
    g.close()
    p, _, o, g = run_mrt(name, lbm.LBM_P_FP32_FP16, 50)
    ref = orc.Oracle(dict(p, nx=1, ny=1, bc=[inputs.PERIODIC] * 4)).init(1.0, 0.0, 0.0,
                                                                      p["T0"]).pops()
    po = o.pops()
    assert np.abs(g.pops() - po).max() <= 8 * 2.0 ** -11 * np.abs(po - ref).max()
    g.close()


@pytest.mark.parametrize("name", ["couette_walls", "cavity"])
def test_uniform_rates_equal_bgk_on_gpu(name):
    p, fields = make_case(name, lbm.LBM_P_FP64)
    bgk = lbm.Lbm(p).init(*fields).step(40)
    mrt = lbm.Lbm(dict(p, collision=lbm.LBM_COLL_MRT)).init(*fields).step(40)
    assert rel(mrt.pops(), bgk.pops()) <= 1e-12
    bgk.close()
    mrt.close()


def test_mrt_and_bgk_grids_in_one_batch():
    grids = []
    for name, rates in (("cavity", RATES), ("couette_walls", {}), ("periodic_total", RATES),
                        ("x_walls_y_periodic", RATES)):
        p, fields = make_case(name, lbm.LBM_P_FP64)
        grids.append((dict(p, **rates), fields))
    b = lbm.Batch(lbm.LBM_P_FP64, 8, 1 << 28)
    slots = [b.add(p, f, 30) for p, f in grids]
    b.run(30)
    for (p, f), s in zip(grids, slots):
        o = orc.Oracle(p).init(*f).step(30)
        assert rel(b.pops(s), o.pops()) <= 1e-12
    b.close()


def test_two_node_variant_rejects_mrt():
    p, fields = make_case("periodic_total", lbm.LBM_P_FP32)
    g = lbm.Lbm(dict(p, **RATES))
    with pytest.raises(lbm.LbmError) as e:
        g.set_launch(2, 0)
    assert e.value.status == lbm.LBM_ERR_PARAM
    g.close()
