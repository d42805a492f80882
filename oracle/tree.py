"""Cluster tree and block partition (oracle; test infrastructure only).

Sec. II: the matrix is split into multilevel admissible blocks R and inadmissible
leaf blocks F; a block (t, s) is admissible under Eq. admCond,
    max(diam(Omega_t), diam(Omega_s)) <= eta * dist(Omega_t, Omega_s).
Sec. III: the tree is indexed with the root at level 0 and the leaves at level L;
the same tree serves rows and columns and A, B and C share one partition.

Readings taken where the paper is silent:
  * the tree is a complete binary tree built by cardinality-balanced bisection along
    the longest side of the cluster's bounding box, ties of the coordinate broken by
    the point's user index; a cluster of n points gives (n+1)//2 points to its first
    child; L is the smallest level with at most leaf_size points per cluster;
  * diam is the diagonal of the axis-aligned bounding box and dist the distance
    between two boxes; both are compared squared, summed over x, y, z in that order,
    so that the test is reproducible bit for bit; a block is admissible only if the
    boxes are apart (dist > 0).

Pins: tests/test_oracle_tree.py (leaf blocks tile the matrix exactly once, every R
block admissible and every F block inadmissible at the leaf level, children of an
inadmissible non-leaf block, brute force classification on small inputs).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

R, F, NL = "R", "F", "NL"


@dataclass
class ClusterTree:
    n: int
    leaf_size: int
    L: int
    perm: np.ndarray                 # tree position -> user index
    start: list                      # start[l][t]
    size: list                       # size[l][t]
    lo: list                         # lo[l][t] = bbox minimum (3,)
    hi: list                         # hi[l][t] = bbox maximum (3,)

    def range(self, l: int, t: int) -> slice:
        s = self.start[l][t]
        return slice(s, s + self.size[l][t])

    def nclusters(self, l: int) -> int:
        return 1 << l


def num_levels(n: int, leaf_size: int) -> int:
    L = 0
    while -(-n // (1 << L)) > leaf_size:
        L += 1
    return L


def build_tree(points: np.ndarray, leaf_size: int) -> ClusterTree:
    points = np.asarray(points, dtype=np.float64)
    n = points.shape[0]
    L = num_levels(n, leaf_size)
    perm = np.arange(n, dtype=np.int64)
    start = [[0]]
    size = [[n]]
    for l in range(L):
        ns, nz = [], []
        for t in range(1 << l):
            s0, m = start[l][t], size[l][t]
            idx = perm[s0:s0 + m]
            p = points[idx]
            lo, hi = p.min(axis=0), p.max(axis=0)
            ext = hi - lo
            axis = 0
            for d in (1, 2):
                if ext[d] > ext[axis]:
                    axis = d
            order = np.lexsort((idx, p[:, axis]))     # by coordinate, then user index
            perm[s0:s0 + m] = idx[order]
            m1 = (m + 1) // 2
            ns += [s0, s0 + m1]
            nz += [m1, m - m1]
        start.append(ns)
        size.append(nz)
    lo_l, hi_l = [], []
    for l in range(L + 1):
        los, his = [], []
        for t in range(1 << l):
            p = points[perm[start[l][t]:start[l][t] + size[l][t]]]
            los.append(p.min(axis=0))
            his.append(p.max(axis=0))
        lo_l.append(los)
        hi_l.append(his)
    return ClusterTree(n, leaf_size, L, perm, start, size, lo_l, hi_l)


def diam2(lo, hi) -> float:
    d0, d1, d2 = hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]
    return d0 * d0 + d1 * d1 + d2 * d2


def dist2(lo_t, hi_t, lo_s, hi_s) -> float:
    acc = 0.0
    for d in range(3):
        g = max(0.0, lo_s[d] - hi_t[d], lo_t[d] - hi_s[d])
        acc = acc + g * g
    return acc


def admissible(tree: ClusterTree, l: int, t: int, s: int, eta: float) -> bool:
    """Eq. admCond with box diameters and box distance, compared squared."""
    dd = dist2(tree.lo[l][t], tree.hi[l][t], tree.lo[l][s], tree.hi[l][s])
    if not dd > 0.0:
        return False
    dt = diam2(tree.lo[l][t], tree.hi[l][t])
    ds = diam2(tree.lo[l][s], tree.hi[l][s])
    return max(dt, ds) <= (eta * eta) * dd


@dataclass
class Partition:
    """Blocks per level: blocks[l] is a list of (t, s, kind), sorted by (t, s)."""
    tree: ClusterTree
    eta: float
    blocks: list = field(default_factory=list)
    kind: list = field(default_factory=list)        # kind[l][(t, s)] -> R/F/NL

    @property
    def L(self) -> int:
        return self.tree.L


def build_partition(tree: ClusterTree, eta: float) -> Partition:
    part = Partition(tree, eta)
    cand = [(0, 0)]
    for l in range(tree.L + 1):
        out = []
        nxt = []
        for (t, s) in sorted(cand):
            if admissible(tree, l, t, s, eta):
                out.append((t, s, R))
            elif l == tree.L:
                out.append((t, s, F))
            else:
                out.append((t, s, NL))
                for a in (0, 1):
                    for b in (0, 1):
                        nxt.append((2 * t + a, 2 * s + b))
        part.blocks.append(out)
        part.kind.append({(t, s): k for (t, s, k) in out})
        cand = nxt
    return part


def csp(part: Partition) -> int:
    """Sparsity constant: the largest number of blocks one cluster forms on a level."""
    best = 0
    for l in range(part.L + 1):
        cnt = {}
        for (t, s, _) in part.blocks[l]:
            cnt[("r", t)] = cnt.get(("r", t), 0) + 1
            cnt[("c", s)] = cnt.get(("c", s), 0) + 1
        if cnt:
            best = max(best, max(cnt.values()))
    return best
