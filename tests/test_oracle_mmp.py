"""Pins for oracle.mmp: the structure-preserving product with change of bases.

* mode "full" keeps every eigenvector, so every projection in Sec. III-IV is exact
  and C must equal the dense product A B to rounding: this fixes every step that is
  not the truncation (cases 1-4, collects, projections, merges, the top-down split);
* the truncated product must stay within a multiple of its threshold (the paper's
  tables show eps_rel / sqrt(eps_trunc) between 0.08 and 0.81, Sec. VI);
* the algorithm must not depend on the choice of input bases (all Grams are
  invariant under V -> V Q), which catches a transposed or conjugated operand;
* the new bases are orthonormal and keep A's partition (Sec. III);
* a planted mistake (a Gram term dropped) breaks the accuracy pin.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import basis as Bs
from oracle import h2, mmp
from paper_1908_05218_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_full_mode_is_the_exact_product(cube2x2_pair):
    _, _, A, B = cube2x2_pair
    C = mmp.mmp(A, B, 0.0, Bs.FULL)
    assert rel(h2.to_dense(C), h2.to_dense(A) @ h2.to_dense(B)) < 1e-13


def test_full_mode_with_rotated_bases_and_complex_kernel():
    w = inputs.workload_sphere(640, radius=1.5, wavenumber=2 * math.pi)
    A = h2.rotate_bases(h2.build(w.points, w.kernel, 20, 1.0, 1e-5), seed=1)
    B = h2.rotate_bases(h2.build(w.points, w.kernel, 20, 1.0, 1e-3), seed=2)
    C = mmp.mmp(A, B, 0.0, Bs.FULL)
    assert rel(h2.to_dense(C), h2.to_dense(A) @ h2.to_dense(B)) < 1e-13


@pytest.mark.parametrize("mode,eps,bound", [("paper", 1e-2, 1.0), ("paper", 1e-4, 1.0),
                                            ("sv", 1e-2, 1.0), ("sv", 1e-4, 1.0)])
def test_truncated_product_error_within_bound(cube2x2_pair, mode, eps, bound):
    _, _, A, B = cube2x2_pair
    C = mmp.mmp(A, B, eps, mode)
    ref = h2.to_dense(A) @ h2.to_dense(B)
    err = rel(h2.to_dense(C), ref)
    scale = math.sqrt(eps) if mode == "paper" else eps
    assert err <= bound * scale, err
    assert err > 0.0
    # Eq. error with exact H^2 matvecs agrees with the dense error within a factor
    x = inputs.standard_normal((ref.shape[0], 4), seed=1)
    y_ref = h2.matvec(A, h2.matvec(B, x))
    e2 = np.linalg.norm(h2.matvec(C, x) - y_ref) / np.linalg.norm(y_ref)
    assert e2 <= 3 * bound * scale


def test_error_trend_matches_the_papers_tables(cube2x2_pair):
    # Sec. VI tables: eps_rel / sqrt(eps_trunc) stays inside [0.078, 0.81]
    tab = json.load(open(GOLDEN))
    ratios = []
    for name, t in (("bus", tab["bus"]), ("slab", tab["slab"]), ("cube", tab["cube"])):
        for key, vals in t.items():
            if key.startswith("1e"):
                ratios += [v / math.sqrt(float(key)) for v in vals]
    lo, hi = min(ratios), max(ratios)
    assert 0.07 < lo < 0.08 and 0.8 < hi < 0.82
    _, _, A, B = cube2x2_pair
    ref = h2.to_dense(A) @ h2.to_dense(B)
    for eps in (1e-2, 1e-4):
        r = rel(h2.to_dense(mmp.mmp(A, B, eps, "paper")), ref) / math.sqrt(eps)
        assert lo / 4 < r < hi * 4


def test_result_does_not_depend_on_input_bases(cube2x2_pair):
    _, _, A, B = cube2x2_pair
    C1 = h2.to_dense(mmp.mmp(A, B, 1e-4, "paper"))
    C2 = h2.to_dense(mmp.mmp(h2.rotate_bases(A, 3), h2.rotate_bases(B, 4), 1e-4, "paper"))
    assert rel(C2, C1) < 1e-11


def test_new_bases_orthonormal_and_structure_kept(cube2x2_pair):
    _, _, A, B = cube2x2_pair
    st = {}
    C = mmp.mmp(A, B, 1e-4, "paper", stats=st)
    assert C.part is A.part
    assert set(C.S) == {(l, t, s) for l in range(A.L + 1) for (t, s, k) in A.part.blocks[l] if k == "R"}
    assert set(C.Fb) == set(A.Fb)
    for l in range(st["l_min"], A.L + 1):
        for t in range(1 << l):
            for col in (False, True):
                v = h2.expand_basis(C, l, t, col)
                np.testing.assert_allclose(v.T @ v, np.eye(v.shape[1]), atol=1e-12)


def test_ranks_monotone_in_eps(cube2x2_pair):
    _, _, A, B = cube2x2_pair
    ranks = {}
    for eps in (1e-2, 1e-3, 1e-4):
        st = {}
        mmp.mmp(A, B, eps, "paper", stats=st)
        ranks[eps] = st
    L = A.L
    for a, b in ((1e-2, 1e-3), (1e-3, 1e-4)):
        # leaf Grams do not depend on eps: per-cluster monotonicity is exact there
        assert all(x <= y for x, y in zip(ranks[a]["ranks_r"][L], ranks[b]["ranks_r"][L]))
        assert all(x <= y for x, y in zip(ranks[a]["ranks_c"][L], ranks[b]["ranks_c"][L]))
        for l in range(ranks[a]["l_min"], L):
            assert sum(ranks[a]["ranks_r"][l]) <= sum(ranks[b]["ranks_r"][l])


def test_new_row_rank_at_least_old_rank(cube2x2_pair):
    # G3 (Eq. Gr3L) is kept: each normalised eigenvalue of Vr Vr^H is 1/sqrt(k) > eps
    _, _, A, B = cube2x2_pair
    st = {}
    mmp.mmp(A, B, 1e-3, "paper", stats=st)
    L = A.L
    assert all(st["ranks_r"][L][t] >= A.kr[(L, t)] for t in range(1 << L))
    assert all(st["ranks_c"][L][t] >= B.kc[(L, t)] for t in range(1 << L))


def test_planted_mistake_breaks_the_accuracy_pin(cube2x2_pair, monkeypatch):
    # drop the case-2 Gram term (Eq. Gr2L) in the oracle: nestedness is lost and the
    # accuracy pin fails, showing that the pin sees the Gram terms
    _, _, A, B = cube2x2_pair
    ref = h2.to_dense(A) @ h2.to_dense(B)
    orig = Bs.normalized_sum

    def drop_second(grams, dim, dtype, *rest):
        return orig([grams[0], None, grams[2]], dim, dtype, *rest)

    monkeypatch.setattr(mmp.Bs, "normalized_sum", drop_second)
    err = rel(h2.to_dense(mmp.mmp(A, B, 1e-4, "paper")), ref)
    assert err > 1.0 * math.sqrt(1e-4)


def test_formatted_product_keeps_input_bases_and_is_exact_with_complete_bases(cube2x2_pair):
    # the comparison method ("Existing" row of the cube-array table): C's bases are
    # A's row and B's column bases.  With complete bases (a full-mode product as input:
    # square leaf bases and transfers) every projection is the identity -> exact.
    _, _, A, B = cube2x2_pair
    Cf = mmp.mmp(A, B, 0.0, Bs.FULL)
    D = mmp.mmp(Cf, Cf, 0.0, Bs.FORMATTED)
    ref = h2.to_dense(Cf) @ h2.to_dense(Cf)
    assert rel(h2.to_dense(D), ref) < 1e-12
    E = mmp.mmp(A, B, 0.0, Bs.FORMATTED)
    L = A.L
    assert all(E.kr[(L, t)] == A.kr[(L, t)] for t in range(1 << L))
    assert all(E.kc[(L, t)] == B.kc[(L, t)] for t in range(1 << L))
    np.testing.assert_array_equal(E.Vr[0], A.Vr[0])


def test_formatted_product_is_less_accurate_than_change_of_bases(cube2x2_pair):
    # Sec. VI, Table relErr_cube: the formatted product's error exceeds the proposed
    # product's at every eps_trunc
    _, _, A, B = cube2x2_pair
    ref = h2.to_dense(A) @ h2.to_dense(B)
    e_fmt = rel(h2.to_dense(mmp.mmp(A, B, 0.0, Bs.FORMATTED)), ref)
    e_new = rel(h2.to_dense(mmp.mmp(A, B, 1e-2, "paper")), ref)
    assert e_fmt > e_new
