"""The seeded workload generators (shared by the oracle tests and the GPU path; they
hold no arithmetic of the method)."""
import math

import numpy as np

from paper_1908_05218_gb300 import inputs


def test_batch_instances_follow_their_recipe():
    ws = inputs.workload_batch(48)
    again = inputs.workload_batch(48)
    assert len(ws) == 48
    for w, v in zip(ws, again):  # seeded: the same instances every time
        np.testing.assert_array_equal(w.points, v.points)
    ns = np.array([w.points.shape[0] for w in ws])
    assert ns.min() >= 4096 and ns.max() <= 131072
    # log-uniform: the logs of N spread over most of [log 4096, log 131072]
    lg = np.log(ns)
    assert lg.max() - lg.min() > 0.7 * (math.log(131072) - math.log(4096))
    for w in ws:
        ext = w.points.max(axis=0) - w.points.min(axis=0)
        assert ext[0] <= 1.0 and ext[1] <= 8.0 and ext[2] <= 8.0
        assert w.kernel.kind == 0  # 1/(4 pi r)


def test_cube_array_sizes():
    w = inputs.workload_cube_array(2, 3, 512)
    assert w.points.shape == (2 * 3 * 512, 3)
    assert np.isfinite(w.points).all()
