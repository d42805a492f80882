"""The structure-preserving H^2 matrix-matrix product C = A B with change of
cluster bases (Ma & Jiao), written step by step in the paper's order and notation.

TEST INFRASTRUCTURE ONLY.  Plain float64 / complex128 loops over blocks and
triples; library matmuls and numpy.linalg.eigh are the only primitives.

Notation: i, j, k are clusters of one level; a product A_ij B_jk is a "triple";
the target (i, k) of a triple is, in C (which keeps A's partition, Sec. III), an
inadmissible leaf block F, an admissible block R, a non-leaf block NL, or a
sub-block of an admissible block of a coarser level (SUB, the "blue" blocks of
Fig. 3(c)).  Triples with both factors NL are not computed on their level: their
four children triples are computed one level down (Sec. IV-A).

Leaf level (Sec. III):
  B_j            cluster-basis products, leaf and nested (Sec. III-D, Eq. nonleafproduct)
  F targets      exact dense products, R factors expanded (Sec. III-A)
  row Grams      Eq. Gr1L (per case-1 product with R/SUB target), Eq. Gr2L (every F
                 block of row i in A), Eq. Gr3L; columns: Eq. case1-ch, case2-ch, case3-ch
  new bases      normalised sum, eigen-decomposition, truncation (oracle.basis)
  P, collects    Eq. leafproj, Eq. Fcollect, R-block images of Eq. nonleafA / nonleafB
  couplings      Eq. leafcoup_simple, summed over j per target
Non-leaf level l (Sec. IV, steps 1-6 of Sec. IV-E):
  1-2 collected NL blocks of A and B from the children's images (Eq. nonleafA/B)
  3   merged coupling M_ik of R/SUB targets from the children's sums (Eq. nonleafA
      first form, Eq. NL_col)
  4   transfer Grams Eq. case1-ch-nl (per target), case2-ch-nl (every NL block of
      row i in A), case3-ch-nl, and the column counterparts; new stacked transfer
      matrices E^C = [T^C_1; T^C_2]
  5   nested projections Eq. nonleafproj, NL collect Eq. NLcollect
  6   couplings Eq. nonleafcoup_simple (case-1 once per target, on M)
Post-processing (Sec. IV-E, last paragraph): couplings of NL targets are held and
split top-down into the children blocks of C.

Readings (where the paper is silent, garbled or ambiguous):
  * truncation and normalisation: see oracle.basis;
  * Eq. Gr1L is taken as printed (one Gram term per product F_ij F_jk), Eq.
    case1-ch-nl per merged target;
  * Eq. Gr2L / case2-ch-nl sum over every F (leaf) / NL (non-leaf) block of row i of
    A, whether or not a case-2 partner exists on that level, and their column
    counterparts over every block of column k of B;
  * Eq. case3_coll writes V^A_{j,r}: read as A's column basis V^A_{j,c}, as in
    Eq. Fcollect and in B_j;
  * Eq. nonleafcoup writes V where transfer matrices are meant: Eq.
    nonleafcoup_simple is followed;
  * the case-4 products and the R-block images use B_j of A's column basis and B's
    row basis (Sec. III-D);
  * the bottom-up traversal stops at l_min, the coarsest level holding an admissible
    block; clusters above it get rank 0 in C.

Mode "formatted" is the comparison method of Sec. VI (Table relErr_cube, row
"Existing"; Sec. I): the cluster bases of C are not changed but taken from A (rows)
and B (columns), every product is projected onto them, and no Gram matrix or
eigen-decomposition is formed.

Pins: tests/test_oracle_mmp.py — mode "full" (no truncation) reproduces the exact
dense product to rounding, which fixes every non-truncation step; the truncated
product stays within a multiple of its bound; results do not depend on unitary
changes of the input bases; new bases are orthonormal; ranks grow as eps shrinks.
"""
from __future__ import annotations

import numpy as np

from . import basis as Bs
from .h2 import H2, expand_basis
from .tree import F, NL, R

SUB = "SUB"


def _h(x):
    return x.conj().T


def target_class(part, l: int, i: int, k: int) -> str:
    """Class of (i, k) of level l in C (which has A's partition)."""
    kind = part.kind[l].get((i, k))
    if kind is not None:
        return kind
    for lv in range(l - 1, -1, -1):
        kk = part.kind[lv].get((i >> (l - lv), k >> (l - lv)))
        if kk == R:
            return SUB
        if kk is not None:
            break
    raise AssertionError(f"pair {(l, i, k)} is neither a block nor inside an admissible block")


def triples(part, l: int):
    """All (i, j, k, kind_A, kind_B) with (i, j) and (j, k) blocks of level l."""
    rows = {}
    for (j, k, kb) in part.blocks[l]:
        rows.setdefault(j, []).append((k, kb))
    out = []
    for (i, j, ka) in part.blocks[l]:
        for (k, kb) in rows.get(j, []):
            out.append((i, j, k, ka, kb))
    return out


def l_min(part) -> int:
    for l in range(part.L + 1):
        if any(kind == R for (_, _, kind) in part.blocks[l]):
            return l
    return part.L


def basis_products(A: H2, Bm: H2) -> dict:
    """B_j = (V^A_{j,c})^T V^B_{j,r} on every cluster (Sec. III-D, Eq. nonleafproduct)."""
    L = A.L
    Bj = {}
    for j in range(1 << L):
        Bj[(L, j)] = A.Vc[j].T @ Bm.Vr[j]
    for l in range(L - 1, -1, -1):
        for j in range(1 << l):
            ka1 = A.kc[(l + 1, 2 * j)]
            kb1 = Bm.kr[(l + 1, 2 * j)]
            Ta, Tb = A.Ec[(l, j)], Bm.Er[(l, j)]
            Bj[(l, j)] = (Ta[:ka1].T @ Bj[(l + 1, 2 * j)] @ Tb[:kb1]
                          + Ta[ka1:].T @ Bj[(l + 1, 2 * j + 1)] @ Tb[kb1:])
    return Bj


def mmp(A: H2, Bm: H2, eps: float, mode: str = Bs.PAPER, cap: int | None = None,
        stats: dict | None = None, norm: str = Bs.FRO) -> H2:
    part = A.part
    assert Bm.part.blocks == part.blocks, "A and B must share one block partition"
    tree = part.tree
    L = tree.L
    dtype = np.result_type(A.dtype, Bm.dtype)
    C = H2(part, dtype)
    lmin = l_min(part)
    margins = {}             # (level, cluster, column side) -> truncation margin
    Bj = basis_products(A, Bm)

    def denseA(i, j, kind):           # leaf block of A as a full matrix (Sec. III-A)
        if kind == F:
            return A.Fb[(i, j)]
        return A.Vr[i] @ A.S[(L, i, j)] @ A.Vc[j].T

    def denseB(j, k, kind):
        if kind == F:
            return Bm.Fb[(j, k)]
        return Bm.Vr[j] @ Bm.S[(L, j, k)] @ Bm.Vc[k].T

    # ------------------------------------------------------------ leaf level, Sec. III
    trip = triples(part, L)
    cls = {(i, k): target_class(part, L, i, k) for (i, _, k, _, _) in trip}
    for (t, s, kind) in part.blocks[L]:
        if kind == F:
            C.Fb[(t, s)] = np.zeros((tree.size[L][t], tree.size[L][s]), dtype=dtype)
    # Sec. III-A: products whose target is an F block of C, computed exactly
    for (i, j, k, ka, kb) in trip:
        if cls[(i, k)] == F:
            C.Fb[(i, k)] += denseA(i, j, ka) @ denseB(j, k, kb)

    # Sec. III-C: Gram matrices of the new leaf row and column bases
    formatted = mode == Bs.FORMATTED
    G1r = {i: [] for i in range(1 << L)}
    G1c = {k: [] for k in range(1 << L)}
    for (i, j, k, ka, kb) in ([] if formatted else trip):
        if ka == F and kb == F and cls[(i, k)] in (R, SUB):
            X = A.Fb[(i, j)] @ Bm.Fb[(j, k)]
            G1r[i].append(X @ _h(X))                       # Eq. Gr1L
            G1c[k].append(X.T @ X.conj())                  # Eq. case1-ch
    Vn_r, Vn_c = {}, {}
    for i in ([] if formatted else range(1 << L)):
        n_i = tree.size[L][i]
        g1 = sum(G1r[i]) if G1r[i] else None
        g2 = None
        for (ii, j, kind) in part.blocks[L]:
            if ii == i and kind == F:
                Y = A.Fb[(i, j)] @ Bm.Vr[j]
                g2 = Y @ _h(Y) if g2 is None else g2 + Y @ _h(Y)   # Eq. Gr2L
        g3 = A.Vr[i] @ _h(A.Vr[i])                                  # Eq. Gr3L
        G = Bs.normalized_sum([g1, g2, g3], n_i, dtype, norm)
        Vn_r[i], lam = Bs.truncated_eigvecs(G, eps, mode, cap)
        margins[(L, i, False)] = _margin(lam, eps, mode)
    for k in ([] if formatted else range(1 << L)):
        n_k = tree.size[L][k]
        g1 = sum(G1c[k]) if G1c[k] else None
        g2 = None
        for (j, kk, kind) in part.blocks[L]:
            if kk == k and kind == F:
                Y = A.Vc[j].T @ Bm.Fb[(j, k)]
                g2 = Y.T @ Y.conj() if g2 is None else g2 + Y.T @ Y.conj()   # Eq. case2-ch
        g3 = Bm.Vc[k] @ _h(Bm.Vc[k])                                          # Eq. case3-ch
        G = Bs.normalized_sum([g1, g2, g3], n_k, dtype, norm)
        Vn_c[k], lam = Bs.truncated_eigvecs(G, eps, mode, cap)
        margins[(L, k, True)] = _margin(lam, eps, mode)
    if formatted:                          # the existing formatted product keeps the bases
        Vn_r = {i: A.Vr[i] for i in range(1 << L)}
        Vn_c = {k: Bm.Vc[k] for k in range(1 << L)}
    C.Vr, C.Vc = Vn_r, Vn_c
    for t in range(1 << L):
        C.kr[(L, t)] = Vn_r[t].shape[1]
        C.kc[(L, t)] = Vn_c[t].shape[1]

    # Eq. leafproj: projections of the old bases onto the new ones
    PA = {(L, i): _h(Vn_r[i]) @ A.Vr[i] for i in range(1 << L)}
    PB = {(L, k): Bm.Vc[k].T @ Vn_c[k].conj() for k in range(1 << L)}
    # Eq. Fcollect and the R-block images of Eq. nonleafA / nonleafB: every block of A
    # expressed in (new row basis of C, row basis of B); of B in (column basis of A,
    # new column basis of C)
    Ahat, Bhat = {}, {}
    for (i, j, kind) in part.blocks[L]:
        if kind == F:
            Ahat[(L, i, j)] = _h(Vn_r[i]) @ A.Fb[(i, j)] @ Bm.Vr[j]
        else:
            Ahat[(L, i, j)] = PA[(L, i)] @ A.S[(L, i, j)] @ Bj[(L, j)]
    for (j, k, kind) in part.blocks[L]:
        if kind == F:
            Bhat[(L, j, k)] = A.Vc[j].T @ Bm.Fb[(j, k)] @ Vn_c[k].conj()
        else:
            Bhat[(L, j, k)] = Bj[(L, j)] @ Bm.S[(L, j, k)] @ PB[(L, k)]

    # Eq. leafcoup_simple: couplings of R and SUB targets, summed over j
    Ssum = {}
    for (i, j, k, ka, kb) in trip:
        c = cls[(i, k)]
        if c not in (R, SUB):
            continue
        if ka == F and kb == F:                                            # case-1
            s = _h(Vn_r[i]) @ A.Fb[(i, j)] @ Bm.Fb[(j, k)] @ Vn_c[k].conj()
        elif ka == F and kb == R:                                          # case-2
            s = Ahat[(L, i, j)] @ Bm.S[(L, j, k)] @ PB[(L, k)]
        elif ka == R and kb == F:                                          # case-3
            s = PA[(L, i)] @ A.S[(L, i, j)] @ Bhat[(L, j, k)]
        else:                                                              # case-4
            s = PA[(L, i)] @ A.S[(L, i, j)] @ Bj[(L, j)] @ Bm.S[(L, j, k)] @ PB[(L, k)]
        key = (L, i, k)
        Ssum[key] = s if key not in Ssum else Ssum[key] + s
    for (i, k) in {(i, k) for (i, _, k, _, _) in trip}:
        if cls[(i, k)] == R:
            C.S[(L, i, k)] = Ssum[(L, i, k)]

    # ---------------------------------------------------- non-leaf levels, Sec. IV
    H = {}                                   # couplings held by NL targets of C
    for l in range(L - 1, lmin - 1, -1):
        trip = triples(part, l)
        cls = {(i, k): target_class(part, l, i, k) for (i, _, k, _, _) in trip}
        kCr = lambda t: C.kr[(l + 1, t)]      # noqa: E731  (children ranks of C)
        kCc = lambda t: C.kc[(l + 1, t)]      # noqa: E731

        # steps 1-2: collected NL blocks from the children's images, Eq. nonleafA/B
        AcollC, BcollC = {}, {}
        for (i, j, kind) in part.blocks[l]:
            if kind != NL:
                continue
            AcollC[(i, j)] = np.block([[Ahat[(l + 1, 2 * i + a, 2 * j + b)] for b in (0, 1)]
                                       for a in (0, 1)])
            BcollC[(i, j)] = np.block([[Bhat[(l + 1, 2 * i + a, 2 * j + b)] for b in (0, 1)]
                                       for a in (0, 1)])
        # step 3: merged couplings of R/SUB targets that NL x NL products reach
        M = {}
        for (i, j, k, ka, kb) in trip:
            if ka == NL and kb == NL and cls[(i, k)] in (R, SUB) and (i, k) not in M:
                blocks = []
                for a in (0, 1):
                    row = []
                    for b in (0, 1):
                        key = (l + 1, 2 * i + a, 2 * k + b)
                        row.append(Ssum.get(key, np.zeros((kCr(2 * i + a), kCc(2 * k + b)),
                                                          dtype=dtype)))
                    blocks.append(row)
                M[(i, k)] = np.block(blocks)

        # step 4: transfer Grams and the new stacked transfer matrices
        En_r, En_c = {}, {}
        if formatted:
            En_r = {i: A.Er[(l, i)] for i in range(1 << l)}
            En_c = {k: Bm.Ec[(l, k)] for k in range(1 << l)}
        for i in ([] if formatted else range(1 << l)):
            dim = kCr(2 * i) + kCr(2 * i + 1)
            g1 = None
            for (ii, k), m in M.items():
                if ii == i:
                    g1 = m @ _h(m) if g1 is None else g1 + m @ _h(m)        # Eq. case1-ch-nl
            g2 = None
            for (ii, j, kind) in part.blocks[l]:
                if ii == i and kind == NL:
                    Y = AcollC[(i, j)] @ Bm.Er[(l, j)]
                    g2 = Y @ _h(Y) if g2 is None else g2 + Y @ _h(Y)       # Eq. case2-ch-nl
            Pch = _blkdiag(PA[(l + 1, 2 * i)], PA[(l + 1, 2 * i + 1)])
            W = Pch @ A.Er[(l, i)]
            g3 = W @ _h(W)                                                 # Eq. case3-ch-nl
            G = Bs.normalized_sum([g1, g2, g3], dim, dtype, norm)
            En_r[i], lam = Bs.truncated_eigvecs(G, eps, mode, cap)
            margins[(l, i, False)] = _margin(lam, eps, mode)
        for k in ([] if formatted else range(1 << l)):
            dim = kCc(2 * k) + kCc(2 * k + 1)
            g1 = None
            for (i, kk), m in M.items():
                if kk == k:
                    g1 = m.T @ m.conj() if g1 is None else g1 + m.T @ m.conj()
            g2 = None
            for (j, kk, kind) in part.blocks[l]:
                if kk == k and kind == NL:
                    Y = A.Ec[(l, j)].T @ BcollC[(j, k)]
                    g2 = Y.T @ Y.conj() if g2 is None else g2 + Y.T @ Y.conj()
            Pch = _blkdiag(PB[(l + 1, 2 * k)], PB[(l + 1, 2 * k + 1)])
            W = Pch.T @ Bm.Ec[(l, k)].conj()
            g3 = W @ _h(W)
            G = Bs.normalized_sum([g1, g2, g3], dim, dtype, norm)
            En_c[k], lam = Bs.truncated_eigvecs(G, eps, mode, cap)
            margins[(l, k, True)] = _margin(lam, eps, mode)
        for t in range(1 << l):
            C.Er[(l, t)] = En_r[t]
            C.Ec[(l, t)] = En_c[t]
            C.kr[(l, t)] = En_r[t].shape[1]
            C.kc[(l, t)] = En_c[t].shape[1]

        # step 5: nested projections (Eq. nonleafproj) and NL collects (Eq. NLcollect)
        for i in range(1 << l):
            Pch = _blkdiag(PA[(l + 1, 2 * i)], PA[(l + 1, 2 * i + 1)])
            PA[(l, i)] = _h(En_r[i]) @ Pch @ A.Er[(l, i)]
        for k in range(1 << l):
            Pch = _blkdiag(PB[(l + 1, 2 * k)], PB[(l + 1, 2 * k + 1)])
            PB[(l, k)] = Bm.Ec[(l, k)].T @ Pch @ En_c[k].conj()
        for (i, j, kind) in part.blocks[l]:
            if kind == NL:
                Ahat[(l, i, j)] = _h(En_r[i]) @ AcollC[(i, j)] @ Bm.Er[(l, j)]
                Bhat[(l, i, j)] = A.Ec[(l, i)].T @ BcollC[(i, j)] @ En_c[j].conj()
            elif kind == R:
                Ahat[(l, i, j)] = PA[(l, i)] @ A.S[(l, i, j)] @ Bj[(l, j)]
                Bhat[(l, i, j)] = Bj[(l, i)] @ Bm.S[(l, i, j)] @ PB[(l, j)]

        # step 6: couplings, Eq. nonleafcoup_simple
        for (i, k), m in M.items():                                        # case-1
            Ssum[(l, i, k)] = _h(En_r[i]) @ m @ En_c[k].conj()
        for (i, j, k, ka, kb) in trip:
            if ka == NL and kb == NL:
                continue
            if ka == NL and kb == R:                                       # case-2
                s = Ahat[(l, i, j)] @ Bm.S[(l, j, k)] @ PB[(l, k)]
            elif ka == R and kb == NL:                                     # case-3
                s = PA[(l, i)] @ A.S[(l, i, j)] @ Bhat[(l, j, k)]
            else:                                                          # case-4
                s = PA[(l, i)] @ A.S[(l, i, j)] @ Bj[(l, j)] @ Bm.S[(l, j, k)] @ PB[(l, k)]
            key = (l, i, k)
            if cls[(i, k)] == NL:
                H[key] = s if key not in H else H[key] + s
            else:
                Ssum[key] = s if key not in Ssum else Ssum[key] + s
        for (i, k) in {(i, k) for (i, _, k, _, _) in trip}:
            if cls[(i, k)] == R:
                C.S[(l, i, k)] = Ssum[(l, i, k)]

    # levels above l_min hold no admissible block: rank 0 bases there
    for l in range(lmin - 1, -1, -1):
        for t in range(1 << l):
            C.Er[(l, t)] = np.zeros((C.kr[(l + 1, 2 * t)] + C.kr[(l + 1, 2 * t + 1)], 0), dtype=dtype)
            C.Ec[(l, t)] = np.zeros((C.kc[(l + 1, 2 * t)] + C.kc[(l + 1, 2 * t + 1)], 0), dtype=dtype)
            C.kr[(l, t)] = 0
            C.kc[(l, t)] = 0
    for l in range(lmin, L + 1):
        for (t, s, kind) in part.blocks[l]:
            if kind == R and (l, t, s) not in C.S:
                C.S[(l, t, s)] = np.zeros((C.kr[(l, t)], C.kc[(l, s)]), dtype=dtype)

    # post-processing: split the couplings held by NL targets top-down
    for l in range(lmin, L):
        for (i, k, kind) in part.blocks[l]:
            if kind != NL or (l, i, k) not in H:
                continue
            X = C.Er[(l, i)] @ H[(l, i, k)] @ C.Ec[(l, k)].T
            r1 = C.kr[(l + 1, 2 * i)]
            c1 = C.kc[(l + 1, 2 * k)]
            for a in (0, 1):
                for b in (0, 1):
                    Xab = X[(slice(0, r1), slice(r1, None))[a], (slice(0, c1), slice(c1, None))[b]]
                    ca, cb = 2 * i + a, 2 * k + b
                    child = part.kind[l + 1][(ca, cb)]
                    if child == R:
                        C.S[(l + 1, ca, cb)] = C.S[(l + 1, ca, cb)] + Xab
                    elif child == NL:
                        key = (l + 1, ca, cb)
                        H[key] = Xab if key not in H else H[key] + Xab
                    else:
                        C.Fb[(ca, cb)] = C.Fb[(ca, cb)] + C.Vr[ca] @ Xab @ C.Vc[cb].T
    if stats is not None:
        stats["l_min"] = lmin
        stats["ranks_r"] = {l: [C.kr[(l, t)] for t in range(1 << l)] for l in range(L + 1)}
        stats["ranks_c"] = {l: [C.kc[(l, t)] for t in range(1 << l)] for l in range(L + 1)}
        stats["margins"] = margins
    return C


def _margin(lam, eps, mode) -> float:
    """Distance of the nearest eigenvalue to the truncation threshold, in units of
    lambda_1 (how far rounding would have to move the rank decision)."""
    if mode in (Bs.FULL, Bs.FORMATTED) or len(lam) == 0 or not lam[0] > 0:
        return float("inf")
    return float(np.min(np.abs(lam / lam[0] - Bs.threshold(eps, mode))))


def _blkdiag(a, b):
    out = np.zeros((a.shape[0] + b.shape[0], a.shape[1] + b.shape[1]),
                   dtype=np.result_type(a.dtype, b.dtype))
    out[:a.shape[0], :a.shape[1]] = a
    out[a.shape[0]:, a.shape[1]:] = b
    return out
