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
