"""Serving loop on the GPU: every request served in the mix gives the same
result as the same request served alone (bitwise: a grid's arithmetic does not
depend on the other grids of the batch or on the segment lengths)."""
import numpy as np
import pytest

from paper_1109_6672_gb300 import lbm, serve

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone_and_in_the_mix():
    prec = lbm.LBM_P_FP32_BF16
    trace = serve.make_trace(12, seed=11, rate=400.0, cavity_sides=(32, 160), couette_ny=(17, 65),
                             steps_range=(60, 300))
    b = lbm.Batch(prec, 6, 1 << 27)  # room for a few at a time: queueing happens
    srv = serve.Server(b, prec, seg_max=48, seg_min=8, keep_moments=True)
    res = srv.run(trace)
    b.close()
    assert sorted(r.rid for r in res) == list(range(12))
    stats = serve.summarize(res, srv.wall, srv.node_updates)
    assert stats["p99_s"] >= stats["p50_s"] > 0
    by_id = {r.rid: r for r in res}
    for req in trace:
        alone = lbm.Batch(prec, 1, 1 << 27)
        p, f = req.materialize(prec)
        s = alone.add(p, f, req.steps)
        while alone.remaining(s):
            alone.run(min(97, alone.remaining(s)))
        mom = alone.moments(s)
        alone.close()
        for a, m in zip(mom, by_id[req.rid].moments):
            np.testing.assert_array_equal(a, m)
