"""GPU edge cases of the product against the oracle: degenerate trees and partitions
(one point, a single leaf, only near-field blocks, two points), coincident points (the
kernel's self term at r = 0, ties in the bisection), points on a line, and a truncation
threshold so large that most ranks fall to zero.  The inputs are built by the oracle and
imported; the float64 product must equal the oracle's element by element (reading of
the tolerances in test_gpu_parity), with equal ranks.  The GPU construction (h2_build)
must accept the same degenerate point sets.
"""
import numpy as np
import pytest

from oracle import h2 as oh2
from oracle import mmp as ommp
from paper_1908_05218_gb300 import inputs

from oracle_bridge import pack, ranks

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1908_05218_gb300 import h2
    return h2


def _pts(name):
    rng = np.random.default_rng(11)
    if name == "one_point":
        return rng.random((1, 3)), 32, 1.0
    if name == "two_points":
        return np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0]]), 1, 1.0
    if name == "single_leaf_20":
        return rng.random((20, 3)), 32, 1.0
    if name == "near_only_60":
        return rng.random((60, 3)), 32, 1.0
    if name == "duplicates_200":
        p = rng.random((100, 3))
        return np.concatenate([p, p[::-1]]), 16, 1.0
    if name == "line_512":
        x = np.linspace(0.0, 1.0, 512)
        return np.stack([x, np.zeros_like(x), np.zeros_like(x)], axis=1), 16, 1.0
    raise KeyError(name)


EDGES = ["one_point", "two_points", "single_leaf_20", "near_only_60", "duplicates_200", "line_512"]


@pytest.mark.parametrize("name", EDGES)
@pytest.mark.parametrize("mode,eps", [("paper", 1e-4), ("sv", 1e-3)])
def test_degenerate_inputs_match_the_oracle(lib, name, mode, eps):
    pts, leaf, eta = _pts(name)
    h = max(1e-3, len(pts) ** (-1 / 3))
    A = oh2.build(pts, inputs.laplace_spec(h), leaf, eta, 1e-6)
    B = oh2.rotate_bases(oh2.build(pts, inputs.inv_r2_spec(h), leaf, eta, 1e-6), seed=3)
    C = ommp.mmp(A, B, eps, mode)
    ga = lib.h2_import(pts, leaf, eta, pack(A))
    gb = lib.h2_import(pts, leaf, eta, pack(B))
    gc = ga.mmp(gb, eps, trunc=mode, rank_cap=64)
    e = gc.export()
    ckr, ckc = ranks(C)
    np.testing.assert_array_equal(e.kr[: len(ckr)], ckr)
    np.testing.assert_array_equal(e.kc[: len(ckc)], ckc)
    d_gpu = gc.to_dense().cpu().numpy()
    d_orc = oh2.to_dense(C)
    scale = max(float(np.max(np.abs(d_orc))), 1e-300)
    assert float(np.max(np.abs(d_gpu - d_orc))) <= TOL * scale
    # the mixed product of the same inputs: finite and within 2 eps of the float64 one
    gm = ga.mmp(gb, eps, trunc=mode, rank_cap=64, precision=lib.MIXED_FP32)
    d_mix = gm.to_dense().cpu().numpy()
    assert np.all(np.isfinite(d_mix))
    assert np.linalg.norm(d_mix - d_gpu) <= 2 * max(eps, 2e-5) * max(np.linalg.norm(d_gpu), 1e-300)


def test_large_threshold_drops_ranks_to_zero(lib):
    # eps = 0.5: most clusters keep one direction or none; C is then mostly its dense
    # blocks, and still equals the oracle's
    w = inputs.workload_cube_array(2, 2, 256)
    A = oh2.build(w.points, w.kernel, 32, 1.0, 1e-4)
    C = ommp.mmp(A, A, 0.5, "paper")
    ga = lib.h2_import(w.points, 32, 1.0, pack(A))
    gc = ga.mmp(ga, 0.5, trunc="paper")
    e = gc.export()
    ckr, ckc = ranks(C)
    np.testing.assert_array_equal(e.kr[: len(ckr)], ckr)
    assert int(np.max(e.kr)) <= 2
    d_gpu = gc.to_dense().cpu().numpy()
    d_orc = oh2.to_dense(C)
    assert float(np.max(np.abs(d_gpu - d_orc))) <= TOL * float(np.max(np.abs(d_orc)))


@pytest.mark.parametrize("name", EDGES)
def test_gpu_construction_accepts_degenerate_inputs(lib, name):
    pts, leaf, eta = _pts(name)
    h = max(1e-3, len(pts) ** (-1 / 3))
    g = lib.h2_build(pts, inputs.laplace_spec(h), leaf, eta, 1e-4)
    from oracle import kernels
    from oracle.tree import build_partition, build_tree
    from oracle_bridge import unpack
    o = unpack(g.export(), build_partition(build_tree(pts, leaf), eta))
    K = kernels.dense(inputs.laplace_spec(h), pts)
    err = np.linalg.norm(oh2.to_dense(o) - K) / np.linalg.norm(K)
    assert err <= 2e-4, err
