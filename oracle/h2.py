"""H^2 representation, construction, exact matvec and dense expansion (oracle).

TEST INFRASTRUCTURE ONLY.

Representation (Sec. II): an admissible block is R_ts = V_t S_ts V_s^T; leaf
clusters store their bases V, non-leaf clusters store the stacked transfer matrix
E_t = [T_t1; T_t2] so that V_t = blkdiag(V_t1, V_t2) E_t (the nested property);
inadmissible blocks exist on the leaf level only and are stored densely.  Row and
column bases are kept apart (V_r, V_c), as in Sec. III where the row basis of A and
the column basis of B are distinct objects.  Everything is stored in tree order.

Construction.  The paper builds its input matrices with a method it cites but does
not describe (Sec. V-A, Sec. VI); this oracle takes the plain nested far-field
compression as its reading: the row basis of a leaf t spans the dominant left
singular vectors of K(t, far(t)), where far(t) holds every column index of the
admissible blocks of t and of all its ancestors; a non-leaf t compresses
[V_t1^H K(t1, far(t)); V_t2^H K(t2, far(t))] the same way, which yields its transfer
matrix; singular vectors with sigma / sigma_1 > eps_h2 are kept.  Column bases are
built the same way from K^T.  Couplings are S_ts = V_t^H K(t, s) conj(V_s), dense
blocks are K(t, s).

Large inputs (far_sample set): the far field of a cluster is read only at a
deterministic sample of each partner block, at most far_sample points taken at an
even stride in tree order; couplings and dense blocks stay exact.  This is the
reading of the cited construction for N beyond what the exact far field allows (its
cost is L N^2 kernel entries); the product is checked against the product of the
matrices built here, so the construction's accuracy does not enter that check.

Matvec (Sec. VI, Eq. error: the reference solution is computed with exact H^2
matrix-vector products): forward transform with the column bases, coupling, backward
transform with the row bases, plus the dense near field.

Pins: tests/test_oracle_h2.py (to_dense(H) x == matvec(H, x) to 1e-13, to_dense
against the dense kernel within the construction tolerance, orthonormal bases,
and the exact special case where the far field has full rank).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import basis as B
from . import kernels
from .tree import NL, R, F, Partition, build_partition, build_tree


@dataclass
class H2:
    part: Partition
    dtype: type
    Vr: dict = field(default_factory=dict)      # leaf t -> (|t|, k)
    Vc: dict = field(default_factory=dict)
    Er: dict = field(default_factory=dict)      # (l, t), l < L -> (k_t1 + k_t2, k_t)
    Ec: dict = field(default_factory=dict)
    kr: dict = field(default_factory=dict)      # (l, t) -> row rank
    kc: dict = field(default_factory=dict)
    S: dict = field(default_factory=dict)       # (l, t, s) -> (kr_t, kc_s), R blocks
    Fb: dict = field(default_factory=dict)      # (t, s) -> dense, leaf F blocks

    @property
    def tree(self):
        return self.part.tree

    @property
    def L(self):
        return self.part.tree.L


def expand_basis(h: H2, l: int, t: int, col: bool = False) -> np.ndarray:
    """V_t as an explicit |t| x k matrix (nested property, Sec. II)."""
    if l == h.L:
        return (h.Vc if col else h.Vr)[t]
    E = (h.Ec if col else h.Er)[(l, t)]
    v1 = expand_basis(h, l + 1, 2 * t, col)
    v2 = expand_basis(h, l + 1, 2 * t + 1, col)
    k1 = v1.shape[1]
    return np.concatenate([v1 @ E[:k1], v2 @ E[k1:]], axis=0)


def far_field(part: Partition, l: int, t: int, col: bool, index=None) -> list:
    """(level, cluster) pairs of the admissible partners of t and of its ancestors."""
    if index is None:
        index = admissible_partners(part, col)
    out = []
    for lv in range(l, -1, -1):
        tt = t >> (l - lv)
        out += [(lv, b) for b in index[lv].get(tt, [])]
    return out


def admissible_partners(part: Partition, col: bool) -> list:
    """Per level: cluster -> partners s of its admissible blocks (t, s) (or (s, t))."""
    out = []
    for lv in range(part.L + 1):
        d = {}
        for (a, b, kind) in part.blocks[lv]:
            if kind == R:
                if col:
                    d.setdefault(b, []).append(a)
                else:
                    d.setdefault(a, []).append(b)
        out.append(d)
    return out


def _far_indices(tree, pairs, sample=None) -> np.ndarray:
    if not pairs:
        return np.zeros(0, dtype=np.int64)
    out = []
    for (lv, s) in pairs:
        n = tree.size[lv][s]
        if sample is None or n <= sample:
            out.append(np.arange(tree.start[lv][s], tree.start[lv][s] + n))
        else:       # sample points at an even stride in tree order
            out.append(tree.start[lv][s] + (np.arange(sample) * n) // sample)
    return np.concatenate(out)


def build(points: np.ndarray, spec, leaf_size: int, eta: float, eps_h2: float,
          far_sample: int | None = None) -> H2:
    """Nested far-field compression of the kernel matrix (reading stated above);
    far_sample: None (exact far field) or the most points read per partner block."""
    tree = build_tree(points, leaf_size)
    part = build_partition(tree, eta)
    dtype = np.complex128 if kernels.is_complex(spec) else np.float64
    h = H2(part, dtype)
    pts = np.asarray(points, dtype=np.float64)[tree.perm]     # tree order
    n = tree.n

    def K(rows, cols):
        same = rows[:, None] == cols[None, :]
        return kernels.kernel_matrix(spec, pts[rows], pts[cols], same).astype(dtype)

    L = tree.L
    cache = {}

    def expanded(l, t, col):
        key = (l, t, col)
        if key not in cache:
            if l == L:
                cache[key] = (h.Vc if col else h.Vr)[t]
            else:
                E = (h.Ec if col else h.Er)[(l, t)]
                v1, v2 = expanded(l + 1, 2 * t, col), expanded(l + 1, 2 * t + 1, col)
                k1 = v1.shape[1]
                cache[key] = np.concatenate([v1 @ E[:k1], v2 @ E[k1:]], axis=0)
        return cache[key]

    for col in (False, True):
        index = admissible_partners(part, col)
        V = h.Vc if col else h.Vr
        E = h.Ec if col else h.Er
        rk = h.kc if col else h.kr
        for l in range(L, -1, -1):
            for t in range(1 << l):
                rows = np.arange(tree.start[l][t], tree.start[l][t] + tree.size[l][t])
                far = _far_indices(tree, far_field(part, l, t, col, index), far_sample)
                if l == L:
                    w = K(rows, far) if not col else K(far, rows).T
                else:
                    v1 = expanded(l + 1, 2 * t, col)
                    v2 = expanded(l + 1, 2 * t + 1, col)
                    n1 = v1.shape[0]
                    kf = K(rows, far) if not col else K(far, rows).T
                    w = np.concatenate([v1.conj().T @ kf[:n1], v2.conj().T @ kf[n1:]], axis=0)
                g = w @ w.conj().T
                u, _ = B.truncated_eigvecs(g, eps_h2, B.SV) if far.size else (
                    np.zeros((w.shape[0], 0), dtype=dtype), None)
                if l == L:
                    V[t] = u.astype(dtype)
                else:
                    E[(l, t)] = u.astype(dtype)
                rk[(l, t)] = u.shape[1]
    for l in range(L + 1):
        for (t, s, kind) in part.blocks[l]:
            rows = np.arange(tree.start[l][t], tree.start[l][t] + tree.size[l][t])
            cols = np.arange(tree.start[l][s], tree.start[l][s] + tree.size[l][s])
            if kind == R:
                vt = expanded(l, t, False)
                vs = expanded(l, s, True)
                h.S[(l, t, s)] = vt.conj().T @ K(rows, cols) @ vs.conj()
            elif kind == F:
                h.Fb[(t, s)] = K(rows, cols)
    assert n == tree.n
    return h


def to_dense_tree(h: H2) -> np.ndarray:
    """Dense matrix in tree order: R blocks expanded through the nested bases."""
    tree = h.tree
    out = np.zeros((tree.n, tree.n), dtype=h.dtype)
    for l in range(h.L + 1):
        for (t, s, kind) in h.part.blocks[l]:
            rt, rs = tree.range(l, t), tree.range(l, s)
            if kind == R:
                out[rt, rs] = expand_basis(h, l, t) @ h.S[(l, t, s)] @ expand_basis(h, l, s, True).T
            elif kind == F:
                out[rt, rs] = h.Fb[(t, s)]
    return out


def to_dense(h: H2) -> np.ndarray:
    """Dense matrix in user order."""
    d = to_dense_tree(h)
    p = h.tree.perm
    out = np.zeros_like(d)
    out[np.ix_(p, p)] = d
    return out


def matvec(h: H2, x: np.ndarray) -> np.ndarray:
    """y = H x in user order, x of shape (N,) or (N, nrhs); exact H^2 arithmetic."""
    tree = h.tree
    L = h.L
    squeeze = x.ndim == 1
    X = x.reshape(tree.n, -1)
    dtype = np.result_type(h.dtype, X.dtype)
    xt = X[tree.perm].astype(dtype)
    nrhs = X.shape[1]
    # forward transform: xhat_s = V_s^T x_s with the column bases
    xh = {}
    for t in range(1 << L):
        xh[(L, t)] = h.Vc[t].T @ xt[tree.range(L, t)]
    for l in range(L - 1, -1, -1):
        for t in range(1 << l):
            E = h.Ec[(l, t)]
            xh[(l, t)] = E.T @ np.concatenate([xh[(l + 1, 2 * t)], xh[(l + 1, 2 * t + 1)]], axis=0)
    # coupling
    yh = {(l, t): np.zeros((h.kr[(l, t)], nrhs), dtype=dtype)
          for l in range(L + 1) for t in range(1 << l)}
    yt = np.zeros((tree.n, nrhs), dtype=dtype)
    for l in range(L + 1):
        for (t, s, kind) in h.part.blocks[l]:
            if kind == R:
                yh[(l, t)] += h.S[(l, t, s)] @ xh[(l, s)]
            elif kind == F:
                yt[tree.range(l, t)] += h.Fb[(t, s)] @ xt[tree.range(l, s)]
    # backward transform with the row bases
    for l in range(L):
        for t in range(1 << l):
            E = h.Er[(l, t)]
            z = E @ yh[(l, t)]
            k1 = h.kr[(l + 1, 2 * t)]
            yh[(l + 1, 2 * t)] += z[:k1]
            yh[(l + 1, 2 * t + 1)] += z[k1:]
    for t in range(1 << L):
        yt[tree.range(L, t)] += h.Vr[t] @ yh[(L, t)]
    y = np.zeros_like(yt)
    y[tree.perm] = yt
    return y[:, 0] if squeeze else y


def rotate_bases(h: H2, seed: int) -> H2:
    """The same matrix with every cluster basis multiplied by a random unitary.

    V_t -> V_t Q_t on the leaves, E_t -> blkdiag(Q_t1, Q_t2)^H E_t Q_t on non-leaf
    clusters and S_ts -> Q_t^H S_ts conj(Q_s); to_dense is unchanged.  Used to pin
    that the product does not depend on the choice of input bases.
    """
    rng = np.random.default_rng(seed)
    L = h.L
    cplx = np.iscomplexobj(np.zeros(1, dtype=h.dtype))

    def unitary(k):
        a = rng.standard_normal((k, k))
        if cplx:
            a = a + 1j * rng.standard_normal((k, k))
        q, _ = np.linalg.qr(a)
        return q.astype(h.dtype)

    out = H2(h.part, h.dtype, kr=dict(h.kr), kc=dict(h.kc), Fb=dict(h.Fb))
    for col in (False, True):
        rk = h.kc if col else h.kr
        Q = {(l, t): unitary(rk[(l, t)]) for l in range(L + 1) for t in range(1 << l)}
        Vin, Vout = (h.Vc, out.Vc) if col else (h.Vr, out.Vr)
        Ein, Eout = (h.Ec, out.Ec) if col else (h.Er, out.Er)
        for t in range(1 << L):
            Vout[t] = Vin[t] @ Q[(L, t)]
        for l in range(L):
            for t in range(1 << l):
                k1 = rk[(l + 1, 2 * t)]
                E = Ein[(l, t)]
                top = Q[(l + 1, 2 * t)].conj().T @ E[:k1]
                bot = Q[(l + 1, 2 * t + 1)].conj().T @ E[k1:]
                Eout[(l, t)] = np.concatenate([top, bot], axis=0) @ Q[(l, t)]
        if col:
            Qc = Q
        else:
            Qr = Q
    for (l, t, s), S in h.S.items():
        out.S[(l, t, s)] = Qr[(l, t)].conj().T @ S @ Qc[(l, s)].conj()
    return out
