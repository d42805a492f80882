"""Pins for the Gram terms of oracle.mmp (Sec. III-C, Eqs. Gr1L-Gr3L and case1-ch to
case3-ch; Sec. IV-C, Eqs. case1-ch-nl to case3-ch-nl).

The full-mode pin keeps every eigenvector and so cannot see the Gram matrices.  The
tests here check the new bases of truncated products against facts that do not go
through the oracle's Gram code:

* leaf level, exact: for every leaf cluster and side the three contributions of
  Sec. III-C are rebuilt from DENSE slices of A and B (to_dense_tree, the block kinds
  painted onto an N x N map by brute force), normalised and summed into G.  The new
  basis must be the top eigenspace of that G: its rank is #{lambda > thr lambda_1}, the
  residual ||(I - V V^H) G (I - V V^H)||_2 equals lambda_{k+1}(G) to rounding, and every
  normalised component obeys ||(I - V V^H) G_m (I - V V^H)||_2 <= thr lambda_1(G);
* every level, in the expanded space: the expanded new basis U_t of cluster t on level
  l must span the exact product's far-field block (A B)[t, far_l(t)] (all columns of
  admissible blocks of C on levels <= l that hold t or an ancestor) to a relative
  residual below c sqrt(thr), and the column bases likewise; c = 2 (the normalised
  components keep lambda_{k+1}(G) <= thr lambda_1 <= 3 thr, so a contribution with a
  unit-weight Gram leaves at most sqrt(3 thr) outside the span; the correct oracle
  measures at most 0.98 sqrt(thr) on these inputs);
* planted mistakes in the oracle, each a one-line change of oracle/mmp.py's source
  applied in memory (a dropped or transposed Gram term, leaf and non-leaf, row and
  column), must break one of these pins.
"""
import math
import types

import numpy as np
import pytest

from oracle import basis as Bs
from oracle import h2, mmp
from oracle.tree import F, R
from paper_1908_05218_gb300 import inputs

# one-line mistakes planted in oracle/mmp.py: name -> (text, replacement)
MUTANTS = {
    "drop leaf G1 row": ("G1r[i].append(X @ _h(X))", "pass"),
    "drop leaf G1 column": ("G1c[k].append(X.T @ X.conj())", "pass"),
    "transpose X in leaf G1 column": ("G1c[k].append(X.T @ X.conj())", "G1c[k].append(X @ _h(X))"),
    "drop leaf G2 row": ("g2 = Y @ _h(Y) if g2 is None else g2 + Y @ _h(Y)   # Eq. Gr2L", "pass"),
    "drop leaf G2 column": ("g2 = Y.T @ Y.conj() if g2 is None else g2 + Y.T @ Y.conj()   # Eq. case2-ch", "pass"),
    "drop leaf G3 row": ("g3 = A.Vr[i] @ _h(A.Vr[i])", "g3 = None"),
    "drop leaf G3 column": ("g3 = Bm.Vc[k] @ _h(Bm.Vc[k])", "g3 = None"),
    "drop non-leaf G1 row": ("g1 = m @ _h(m) if g1 is None else g1 + m @ _h(m)", "pass"),
    "drop non-leaf G1 column": ("g1 = m.T @ m.conj() if g1 is None else g1 + m.T @ m.conj()", "pass"),
    "drop non-leaf G2 row": ("g2 = Y @ _h(Y) if g2 is None else g2 + Y @ _h(Y)       # Eq. case2-ch-nl", "pass"),
    "drop non-leaf G3 row": ("g3 = W @ _h(W)                                                 # Eq. case3-ch-nl",
                             "g3 = None"),
}
LEAF_MUTANTS = [k for k in MUTANTS if "non-leaf" not in k]
NONLEAF_MUTANTS = [k for k in MUTANTS if "non-leaf" in k]


def mutant(name):
    old, new = MUTANTS[name]
    src = open(mmp.__file__).read()
    assert src.count(old) == 1, f"planted mistake {name!r} no longer matches the oracle source"
    mod = types.ModuleType("oracle._planted")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), f"<oracle/mmp.py with {name}>", "exec"), mod.__dict__)
    return mod


class Dense:
    """A, B, A B as dense tree-ordered matrices and the admissible blocks painted."""

    def __init__(self, A, B):
        self.A, self.B = A, B
        self.part, self.tree, self.L = A.part, A.tree, A.L
        self.DA, self.DB = h2.to_dense_tree(A), h2.to_dense_tree(B)
        self.AB = self.DA @ self.DB
        n = self.tree.n
        # level of the admissible block that holds entry (r, c); -1: none (near field)
        self.adm_level = -np.ones((n, n), dtype=np.int64)
        for l in range(self.L + 1):
            for (t, s, kind) in self.part.blocks[l]:
                if kind == R:
                    self.adm_level[self.tree.range(l, t), self.tree.range(l, s)] = l
        self.fpairs = [(t, s) for (t, s, k) in self.part.blocks[self.L] if k == F]
        self._comps = {}

    def leaf_components(self, t, col, norm="fro"):
        """Unit-Frobenius Gram components of leaf t from dense slices (Sec. III-C):
        case-1 products F F landing in an admissible block of C, the near-field blocks
        of A (resp. B) times B's row (A's column) basis, and the cluster's own basis."""
        key = (t, col, norm)
        if key in self._comps:
            return self._comps[key]
        L, tr, A, B = self.L, self.tree, self.A, self.B
        rt = tr.range(L, t)
        z1, z2 = [], []
        for (a, b) in self.fpairs:
            if not col and a == t:
                rj = tr.range(L, b)
                z2.append(self.DA[rt, rj] @ B.Vr[b])
                for (jj, k) in self.fpairs:
                    if jj == b and self.adm_level[rt.start, tr.range(L, k).start] >= 0:
                        z1.append(self.DA[rt, rj] @ self.DB[rj, tr.range(L, k)])
            if col and b == t:
                rj = tr.range(L, a)
                z2.append(self.DB[rj, rt].T @ A.Vc[a])
                for (i, jj) in self.fpairs:
                    if jj == a and self.adm_level[tr.range(L, i).start, rt.start] >= 0:
                        z1.append((self.DA[tr.range(L, i), rj] @ self.DB[rj, rt]).T)
        z3 = B.Vc[t] if col else A.Vr[t]
        out = []
        for z in (z1, z2, [z3]):
            if z:
                zm = np.hstack(z)
                g = zm @ zm.T
                nrm = np.linalg.norm(g) if norm == "fro" else np.linalg.eigvalsh(g)[-1]
                if nrm > 0:
                    out.append(g / nrm)
        self._comps[key] = out
        return out


def leaf_pin_violations(d: Dense, C, eps, mode, norm="fro"):
    """Leaf clusters whose new basis is not the truncated top eigenspace of the
    dense-built G; clusters with an eigenvalue within 1e-9 of the threshold are
    skipped (the rank there is decided by rounding)."""
    thr = Bs.threshold(eps, mode)
    bad = []
    for t in range(1 << d.L):
        for col in (False, True):
            cs = d.leaf_components(t, col, norm)
            G = sum(cs)
            lam = np.sort(np.linalg.eigvalsh(G))[::-1]
            if np.min(np.abs(lam / lam[0] - thr)) < 1e-9:
                continue
            V = (C.Vc if col else C.Vr)[t]
            k = V.shape[1]
            if k != int(np.sum(lam > thr * lam[0])):
                bad.append((t, col, "rank"))
                continue
            P = np.eye(V.shape[0]) - V @ V.T
            lk1 = lam[k] if k < len(lam) else 0.0
            if np.linalg.norm(P @ G @ P, 2) - lk1 > 1e-12 * lam[0]:
                bad.append((t, col, "not the top eigenspace"))
                continue
            for g in cs:
                if np.linalg.norm(P @ g @ P, 2) > thr * lam[0] * (1 + 1e-9):
                    bad.append((t, col, "component bound"))
    return bad


def span_residuals(d: Dense, C, eps, mode):
    """max over clusters of each level of the relative far-field residual outside the
    expanded new basis, in units of sqrt(thr): (rows, columns) per level."""
    thr = Bs.threshold(eps, mode)
    tr, AB = d.tree, d.AB
    out = {}
    for l in range(d.L + 1):
        wr = wc = 0.0
        for t in range(1 << l):
            rt = tr.range(l, t)
            lv = d.adm_level[rt, :]
            cols = np.where(((lv >= 0) & (lv <= l)).any(axis=0))[0]
            if cols.size:
                U = h2.expand_basis(C, l, t)
                blk = AB[rt][:, cols]
                wr = max(wr, np.linalg.norm(blk - U @ (U.T @ blk)) / np.linalg.norm(blk))
            lv = d.adm_level[:, rt]
            rows = np.where(((lv >= 0) & (lv <= l)).any(axis=1))[0]
            if rows.size:
                W = h2.expand_basis(C, l, t, True)
                blk = AB[rows][:, rt]
                wc = max(wc, np.linalg.norm(blk - (blk @ W) @ W.T) / np.linalg.norm(blk))
        out[l] = (wr / math.sqrt(thr), wc / math.sqrt(thr))
    return out


@pytest.fixture(scope="module")
def dense_pair(cube2x2_pair):
    _, _, A, B = cube2x2_pair
    return Dense(A, B)


@pytest.fixture(scope="module")
def dense_lowrank_pair():
    # input bases at eps_H2 = 1e-2: few directions in V^A, V^B, so the Gram terms
    # carry different subspaces
    wa = inputs.workload_cube_array(2, 2, 512)
    wb = inputs.workload_cube_array(2, 2, 512, kernel="invr2")
    return Dense(h2.build(wa.points, wa.kernel, 32, 1.0, 1e-2), h2.build(wb.points, wb.kernel, 32, 1.0, 1e-2))


@pytest.mark.parametrize("eps,mode,norm", [(1e-4, "paper", "fro"), (1e-3, "sv", "fro"), (1e-4, "paper", "spectral")])
def test_leaf_bases_are_the_top_eigenspace_of_the_dense_gram_sum(dense_pair, eps, mode, norm):
    C = mmp.mmp(dense_pair.A, dense_pair.B, eps, mode, norm=norm)
    assert leaf_pin_violations(dense_pair, C, eps, mode, norm) == []
    if norm == "spectral":      # the two readings give different bases
        assert leaf_pin_violations(dense_pair, C, eps, mode, "fro") != []


@pytest.mark.parametrize("name", LEAF_MUTANTS)
def test_planted_leaf_gram_mistakes_break_the_leaf_pin(dense_pair, name):
    eps, mode = 1e-4, "paper"
    C = mutant(name).mmp(dense_pair.A, dense_pair.B, eps, mode)
    assert len(leaf_pin_violations(dense_pair, C, eps, mode)) >= 4, name


@pytest.mark.parametrize("which", ["dense_pair", "dense_lowrank_pair"])
def test_expanded_bases_span_the_far_field_of_the_exact_product(which, request):
    d = request.getfixturevalue(which)
    for eps, mode in ((1e-6, "sv"), (1e-4, "paper")):
        res = span_residuals(d, mmp.mmp(d.A, d.B, eps, mode), eps, mode)
        worst = max(max(a, b) for a, b in res.values())
        assert worst <= 2.0, (eps, mode, res)


@pytest.mark.parametrize("name", NONLEAF_MUTANTS)
def test_planted_nonleaf_gram_mistakes_break_the_span_pin(dense_pair, dense_lowrank_pair, name):
    # in sv mode at eps = 1e-6 a missing or transposed non-leaf term leaves parts of
    # the product's far field outside the new transfer bases
    eps, mode = 1e-6, "sv"
    worst = 0.0
    for d in (dense_pair, dense_lowrank_pair):
        res = span_residuals(d, mutant(name).mmp(d.A, d.B, eps, mode), eps, mode)
        worst = max(worst, max(max(a, b) for a, b in res.values()))
    assert worst > 4.0, (name, worst)
