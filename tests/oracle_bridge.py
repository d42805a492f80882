"""Test helper: packs an oracle H^2 matrix into the h2_import layout (include/h2.h)."""
import numpy as np

from oracle.tree import F, R


def pack(h):
    from paper_1908_05218_gb300.h2 import Packed
    L = h.L
    blocks = h.part.blocks
    kr = np.array([h.kr[(l, t)] for l in range(L + 1) for t in range(1 << l)], dtype=np.int32)
    kc = np.array([h.kc[(l, t)] for l in range(L + 1) for t in range(1 << l)], dtype=np.int32)

    dt = np.complex128 if np.issubdtype(h.dtype, np.complexfloating) else np.float64

    def cat(mats):
        mats = [np.asarray(m, dtype=dt).ravel() for m in mats]
        return np.concatenate(mats) if mats else np.zeros(0, dtype=dt)

    vr = cat(h.Vr[t] for t in range(1 << L))
    vc = cat(h.Vc[t] for t in range(1 << L))
    er = cat(h.Er[(l, t)] for l in range(L) for t in range(1 << l))
    ec = cat(h.Ec[(l, t)] for l in range(L) for t in range(1 << l))
    s = cat(h.S[(l, t, u)] for l in range(L + 1) for (t, u, k) in blocks[l] if k == R)
    f = cat(h.Fb[(t, u)] for (t, u, k) in blocks[L] if k == F)
    return Packed(kr, kc, vr, vc, er, ec, s, f)


def ranks(h):
    L = h.L
    kr = np.array([h.kr[(l, t)] for l in range(L + 1) for t in range(1 << l)], dtype=np.int32)
    kc = np.array([h.kc[(l, t)] for l in range(L + 1) for t in range(1 << l)], dtype=np.int32)
    return kr, kc


def unpack(packed, part):
    """The inverse of pack: an oracle H2 on the partition `part` from packed arrays (a
    library-built matrix read into the oracle's representation)."""
    from oracle.h2 import H2
    tree = part.tree
    L = tree.L
    dt = np.complex128 if np.iscomplexobj(packed.vr) else np.float64
    h = H2(part, dt)
    node = lambda l, t: (1 << l) - 1 + t  # noqa: E731
    for l in range(L + 1):
        for t in range(1 << l):
            h.kr[(l, t)] = int(packed.kr[node(l, t)])
            h.kc[(l, t)] = int(packed.kc[node(l, t)])
    off = {"vr": 0, "vc": 0, "er": 0, "ec": 0, "s": 0, "f": 0}

    def take(name, rows, cols):
        a = getattr(packed, name)
        o = off[name]
        off[name] = o + rows * cols
        return np.asarray(a[o:o + rows * cols], dtype=dt).reshape(rows, cols)

    for t in range(1 << L):
        h.Vr[t] = take("vr", tree.size[L][t], h.kr[(L, t)])
    for t in range(1 << L):
        h.Vc[t] = take("vc", tree.size[L][t], h.kc[(L, t)])
    for l in range(L):
        for t in range(1 << l):
            h.Er[(l, t)] = take("er", h.kr[(l + 1, 2 * t)] + h.kr[(l + 1, 2 * t + 1)], h.kr[(l, t)])
    for l in range(L):
        for t in range(1 << l):
            h.Ec[(l, t)] = take("ec", h.kc[(l + 1, 2 * t)] + h.kc[(l + 1, 2 * t + 1)], h.kc[(l, t)])
    for l in range(L + 1):
        for (t, s, kind) in part.blocks[l]:
            if kind == R:
                h.S[(l, t, s)] = take("s", h.kr[(l, t)], h.kc[(l, s)])
    for (t, s, kind) in part.blocks[L]:
        if kind == F:
            h.Fb[(t, s)] = take("f", tree.size[L][t], tree.size[L][s])
    return h
