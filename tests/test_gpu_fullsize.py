"""Full-size GPU checks: configs 1, 2 and 5 of the product, in the benchmark's launch
configuration.  Where the oracle cannot finish in seconds (N = 65,536 and 1,048,576),
properties that hold at any size are checked: the error against the exact product
A(Bx) (Eq. error) within the truncation bound, mixed precision within 2 max(eps, 2e-5)
of float64 and no less accurate against A(Bx), orthonormal nested bases, A's partition
kept, leaf ranks monotone in eps.
"""
import math

import numpy as np
import pytest

from paper_1908_05218_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_1908_05218_gb300 import h2
    return h2


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def eq_error(lib, A, B, C, n, seed=1):
    import torch
    x = torch.from_numpy(inputs.standard_normal((n, 4), seed=seed)).cuda()
    y_ref = A.matvec(B.matvec(x))
    return float(torch.linalg.norm(C.matvec(x) - y_ref) / torch.linalg.norm(y_ref)), x


def test_config1_uniform_1024_against_oracle_and_dense(lib):
    # N = 1024 uniform in the unit cube, seed 0, 1/(4 pi r), leaf 32, eta 1, nested bases
    # at 1e-8, C = A x A with eps = 1e-6, checked against the dense product
    from oracle import h2 as oh2
    from oracle import mmp as ommp
    from oracle_bridge import pack
    w = inputs.workload_uniform(1024, seed=0)
    A = oh2.build(w.points, w.kernel, 32, 1.0, 1e-8)
    C = ommp.mmp(A, A, 1e-6, "paper")
    ga = lib.h2_import(w.points, 32, 1.0, pack(A))
    gc = ga.mmp(ga, 1e-6)
    d = gc.to_dense().cpu().numpy()
    dense = oh2.to_dense(A) @ oh2.to_dense(A)
    ref = oh2.to_dense(C)
    assert np.max(np.abs(d - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert rel(d, dense) < math.sqrt(1e-6)


def test_config2_cube_array_65536_properties(lib):
    wa = inputs.workload_cube_array(4, 4, 4096)
    wb = inputs.workload_cube_array(4, 4, 4096, kernel="invr2")
    n = wa.points.shape[0]
    A = lib.h2_build(wa.points, wa.kernel, 32, 1.0, 1e-4)
    B = lib.h2_build(wb.points, wb.kernel, 32, 1.0, 1e-4)
    res = {}
    for eps, cap in ((1e-4, 48), (1e-6, 96)):
        C64 = A.mmp(B, eps, precision=lib.FP64, rank_cap=cap)
        e64, x = eq_error(lib, A, B, C64, n)
        assert e64 < math.sqrt(eps), (eps, e64)
        Cm = A.mmp(B, eps, precision=lib.MIXED_FP32, rank_cap=cap)
        em, _ = eq_error(lib, A, B, Cm, n)
        assert em < 1.2 * e64 + 1e-6
        diff = float((Cm.matvec(x) - C64.matvec(x)).norm() / C64.matvec(x).norm())
        # within 2 eps of float64; float32 Gram sums resolve eigenvalues to ~1e-7 of
        # lambda_1, so below eps = 2e-5 the mixed product tracks float64 to ~2e-5
        assert diff < 2 * max(eps, 2e-5), (eps, diff)
        assert C64.info()["cap_hits"] == 0 and Cm.info()["cap_hits"] == 0
        res[eps] = C64
    # A's partition is kept
    for l in range(A.info()["levels"]):
        for u, v in zip(A.level_blocks(l), res[1e-4].level_blocks(l)):
            np.testing.assert_array_equal(u, v)
    # leaf ranks grow as eps shrinks (leaf Grams do not depend on eps)
    p4, p6 = res[1e-4].export(), res[1e-6].export()
    nl = (len(p4.kr) + 1) // 2
    assert np.all(p4.kr[-nl:] <= p6.kr[-nl:]) and np.all(p4.kc[-nl:] <= p6.kc[-nl:])
    # new bases orthonormal: leaf bases and stacked transfers (row side)
    perm = A.tree_perm()
    L = int(round(math.log2(nl)))
    leaf_sizes = np.full(nl, n // nl)
    off = 0
    for t in range(nl):
        k = p4.kr[nl - 1 + t]
        V = p4.vr[off: off + leaf_sizes[t] * k].reshape(leaf_sizes[t], k)
        off += leaf_sizes[t] * k
        np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-12)
    off = 0
    for l in range(L):
        for t in range(1 << l):
            k = p4.kr[(1 << l) - 1 + t]
            k1 = p4.kr[(1 << (l + 1)) - 1 + 2 * t]
            k2 = p4.kr[(1 << (l + 1)) - 1 + 2 * t + 1]
            E = p4.er[off: off + (k1 + k2) * k].reshape(k1 + k2, k)
            off += (k1 + k2) * k
            np.testing.assert_allclose(E.T @ E, np.eye(k), atol=1e-12)
    assert len(perm) == n


def test_config5_cube_array_1m_mixed(lib):
    # the benchmark's workload and launch configuration: N = 1,048,576, the BF16 split
    # product (the headline) and the float32 one; both within the truncation bound
    # against A(Bx), and within 2 eps of each other
    wa = inputs.workload_cube_array(16, 16, 4096)
    wb = inputs.workload_cube_array(16, 16, 4096, kernel="invr2")
    n = wa.points.shape[0]
    A = lib.h2_build(wa.points, wa.kernel, 32, 1.0, 1e-4)
    B = lib.h2_build(wb.points, wb.kernel, 32, 1.0, 1e-4)
    ys = {}
    for p in (lib.MIXED_BF16X3, lib.MIXED_FP32):
        C = A.mmp(B, 1e-4, precision=p, autotune=True)
        C = A.mmp(B, 1e-4, precision=p, autotune=True, out=C)
        err, x = eq_error(lib, A, B, C, n)
        assert err < math.sqrt(1e-4), err
        info = C.info()
        assert info["cap_hits"] == 0 and info["n"] == n
        assert max(info["max_rank_row"]) <= 48
        ys[p] = C.matvec(x)
        C.destroy()
    yb, yf = ys[lib.MIXED_BF16X3], ys[lib.MIXED_FP32]
    assert float((yb - yf).norm() / yf.norm()) < 2e-4
