"""Pins for oracle.tree: cluster tree and block partition (Sec. II, Eq. admCond)."""
import numpy as np
import pytest

from oracle import tree as T
from paper_1908_05218_gb300 import inputs


def _pts(kind, n):
    if kind == "uniform":
        return inputs.uniform_cube(n, seed=3)
    if kind == "cubes":
        return inputs.cube_array_surface(2, 2, n // 4, seed=1)
    return inputs.fibonacci_sphere(n, 1.0)


@pytest.mark.parametrize("kind,n,leaf", [("uniform", 1000, 32), ("cubes", 1024, 32),
                                         ("sphere", 777, 20), ("uniform", 64, 1)])
def test_tree_is_a_balanced_partition(kind, n, leaf):
    pts = _pts(kind, n)
    tr = T.build_tree(pts, leaf)
    assert sorted(tr.perm.tolist()) == list(range(n))
    for l in range(tr.L + 1):
        sizes = tr.size[l]
        assert sum(sizes) == n and max(sizes) - min(sizes) <= 1
        for t in range(1 << l):
            assert tr.start[l][t] == (0 if t == 0 else tr.start[l][t - 1] + tr.size[l][t - 1])
    assert max(tr.size[tr.L]) <= leaf
    assert tr.L == 0 or -(-n // (1 << (tr.L - 1))) > leaf
    # each split separates the two children along one coordinate axis
    for l in range(tr.L):
        for t in range(1 << l):
            p1 = pts[tr.perm[tr.range(l + 1, 2 * t)]]
            p2 = pts[tr.perm[tr.range(l + 1, 2 * t + 1)]]
            assert any(p1[:, d].max() <= p2[:, d].min() for d in range(3))


@pytest.mark.parametrize("kind,n,leaf,eta", [("uniform", 512, 16, 1.0), ("cubes", 1024, 32, 1.0),
                                             ("sphere", 600, 20, 2.0)])
def test_partition_tiles_matrix_and_respects_admissibility(kind, n, leaf, eta):
    pts = _pts(kind, n)
    tr = T.build_tree(pts, leaf)
    part = T.build_partition(tr, eta)
    cover = np.zeros((n, n), dtype=np.int32)
    for l in range(tr.L + 1):
        for (t, s, kind_) in part.blocks[l]:
            rt, rs = tr.range(l, t), tr.range(l, s)
            if kind_ in (T.R, T.F):
                cover[rt, rs] += 1
            if kind_ == T.F:
                assert l == tr.L
            if kind_ == T.NL:
                kids = {(a, b) for (a, b, _) in part.blocks[l + 1]}
                assert all((2 * t + a, 2 * s + b) in kids for a in (0, 1) for b in (0, 1))
            # brute force on the point sets: admissible blocks are far apart, F/NL are not
            # admissible by the box test (box test is implied by the point-set test)
            P, Q = pts[tr.perm[rt]], pts[tr.perm[rs]]
            d = np.sqrt(((P[:, None, :] - Q[None, :, :]) ** 2).sum(-1))
            diam_t = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)).max()
            diam_s = np.sqrt(((Q[:, None, :] - Q[None, :, :]) ** 2).sum(-1)).max()
            if kind_ == T.R:
                assert max(diam_t, diam_s) <= eta * d.min() + 1e-12
            else:
                box_t = np.linalg.norm(P.max(0) - P.min(0))
                box_s = np.linalg.norm(Q.max(0) - Q.min(0))
                gap = np.maximum(0, np.maximum(Q.min(0) - P.max(0), P.min(0) - Q.max(0)))
                assert not (np.linalg.norm(gap) > 0 and max(box_t, box_s) <= eta * np.linalg.norm(gap) * (1 - 1e-12))
    assert (cover == 1).all()


def test_points_on_a_line_give_the_textbook_partition():
    # 16 equispaced points on a line, leaf 2, eta 1: clusters of width w on a level
    # are admissible iff their gap is at least w (brute force from the definition)
    pts = np.zeros((16, 3))
    pts[:, 0] = np.arange(16)
    tr = T.build_tree(pts, 2)
    assert tr.L == 3
    part = T.build_partition(tr, 1.0)
    for l in range(tr.L + 1):
        w = 16 >> l
        for (t, s, kind) in part.blocks[l]:
            gap = abs(t - s) * w - (w - 1)
            expect = T.R if gap >= (w - 1) and gap > 0 else (T.F if l == tr.L else T.NL)
            assert kind == expect, (l, t, s, kind, expect)


def test_csp_counts_blocks_per_cluster():
    pts = _pts("cubes", 1024)
    part = T.build_partition(T.build_tree(pts, 32), 1.0)
    # brute force: for every cluster, the blocks it forms as a row and as a column
    # cluster on its level; C_sp is the largest of these counts (Sec. V-B)
    cnt = 0
    for l in range(part.L + 1):
        for t in range(1 << l):
            cnt = max(cnt, sum(1 for (a, _, _) in part.blocks[l] if a == t),
                      sum(1 for (_, b, _) in part.blocks[l] if b == t))
    assert T.csp(part) == cnt and cnt > 0
