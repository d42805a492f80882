"""GPU parity: the CUDA path against the CPU oracle, through the C ABI.

Tolerances (float64 path): the structure and the ranks must match exactly; every
entry of the dense product (or of C x for N too large to expand) agrees with the
oracle's to 1e-12 of the largest entry.  The two sides sum in different orders and
decompose with different eigensolvers, so each cluster's kept subspace agrees only to
u lambda_1 / (lambda_k - lambda_k+1), u = 2^-53, and the directions near the threshold
carry ~sqrt(thr) of the content: the attainable agreement is ~u / sqrt(thr), which
passes 1e-12 only for thresholds thr >= 1e-8; below, the bound is 20 u / sqrt(thr)
(sv mode at eps = 1e-5: thr = 1e-10, measured 8.9e-11).
Mixed precisions: within 2 eps of the oracle, no less accurate against the exact
product, and equal ranks wherever the oracle's decision is clear of the threshold by
more than what float32 Gram matrices can move (1e-5 lambda_1).  The BF16 split
couplings (H2_MIXED_BF16X3) carry relative errors up to ~2^-16, and the non-leaf Gram
matrices are built from them: eigenvalues move by up to ~4e-5 lambda_1, so ranks are
compared where the decision is clear by 1e-4 lambda_1.
"""
import math

import numpy as np
import pytest

from oracle import h2 as oh2
from oracle import mmp as ommp
from oracle.tree import build_partition, build_tree
from paper_1908_05218_gb300 import inputs

from oracle_bridge import pack, ranks

pytestmark = pytest.mark.gpu

TOL = 1e-12     # float64: element-wise, relative to the largest entry
MIXED_MARGIN = 1e-5
BF16_MARGIN = 1e-4
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32x3": 2, "bf16x3": 3}   # h2_precision values


def fp64_tol(eps, mode):
    """Element-wise float64 bound (module docstring): 1e-12, or 20 u / sqrt(thr) when the
    truncation threshold thr lies below 1e-8."""
    thr = {"paper": eps, "sv": eps * eps}.get(mode)
    if thr is None or thr >= 1e-8:
        return TOL
    return max(TOL, 20 * 2.0 ** -53 / math.sqrt(thr))


def assert_entries_close(got, ref, tol=TOL):
    """Every entry of got within tol * max|ref| of ref."""
    scale = float(np.max(np.abs(ref)))
    err = float(np.max(np.abs(got - ref)))
    assert err <= tol * scale, f"max entry difference {err:.3e} = {err / scale:.3e} of max|ref|"


def clear_rank_mismatches(gpu_export, stats, L, margin=MIXED_MARGIN):
    """Clusters (level, t, column side) whose GPU rank differs from the oracle's although
    the oracle's decision is clear of the threshold by `margin` (of lambda_1)."""
    bad = []
    for (l, t, col), m in stats["margins"].items():
        if m <= margin:
            continue
        node = (1 << l) - 1 + t
        got = (gpu_export.kc if col else gpu_export.kr)[node]
        want = (stats["ranks_c"] if col else stats["ranks_r"])[l][t]
        if got != want:
            bad.append((l, t, col, int(got), int(want)))
    return bad


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


CASES = {
    # name: (workload factory, leaf, eta, eps_h2)
    "cubes_1024": (lambda: inputs.workload_cube_array(2, 2, 256), 32, 1.0, 1e-4),
    "cubes_2048_invr2": (lambda: inputs.workload_cube_array(2, 2, 512, kernel="invr2"), 32, 1.0, 1e-4),
    "uniform_1000_ragged": (lambda: inputs.workload_uniform(1000, seed=5), 32, 1.0, 1e-6),
    "sphere_700_ragged": (lambda: inputs.Workload("s", inputs.fibonacci_sphere(700, 2.0), inputs.laplace_spec(0.1), 0.1), 20, 1.5, 1e-5),
}

_cache = {}


def oracle_case(name):
    if name not in _cache:
        fac, leaf, eta, e = CASES[name]
        w = fac()
        _cache[name] = (w, leaf, eta, oh2.build(w.points, w.kernel, leaf, eta, e))
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_structure_is_bit_exact(lib, name):
    w, leaf, eta, A = oracle_case(name)
    g = lib.h2_import(w.points, leaf, eta, pack(A))
    np.testing.assert_array_equal(g.tree_perm(), A.tree.perm)
    for l in range(A.L + 1):
        t, s, k = g.level_blocks(l)
        ob = A.part.blocks[l]
        assert len(t) == len(ob)
        kinds = {"R": 0, "F": 1, "NL": 2}
        assert list(zip(t.tolist(), s.tolist(), k.tolist())) == [(a, b, kinds[c]) for (a, b, c) in ob]


@pytest.mark.parametrize("nx,ppc,leaf", [(2, 1280, 32), (2, 5120, 32), (4, 1024, 32), (2, 1000, 20)])
def test_structure_on_grid_geometries_is_bit_exact(lib, nx, ppc, leaf):
    # panel centroids on a grid: many admissibility tests hold with equality in exact
    # arithmetic, so the library's host rounding must be the oracle's (no fused
    # multiply-add contraction on the host, also where FMA is baseline)
    w = inputs.workload_cube_array(nx, nx, ppc)
    g = lib.h2_build(w.points, w.kernel, leaf, 1.0, 1e-2)
    tree = build_tree(w.points, leaf)
    part = build_partition(tree, 1.0)
    np.testing.assert_array_equal(g.tree_perm(), tree.perm)
    kinds = {"R": 0, "F": 1, "NL": 2}
    for l in range(tree.L + 1):
        t, s, k = g.level_blocks(l)
        assert list(zip(t.tolist(), s.tolist(), k.tolist())) == [(a, b, kinds[c]) for (a, b, c) in part.blocks[l]], l


@pytest.mark.parametrize("name", list(CASES))
def test_import_export_roundtrip_and_matvec(lib, name):
    import torch
    w, leaf, eta, A = oracle_case(name)
    p = pack(A)
    g = lib.h2_import(w.points, leaf, eta, p)
    e = g.export()
    for f in ("kr", "kc", "vr", "vc", "er", "ec", "s", "f"):
        np.testing.assert_array_equal(getattr(e, f), getattr(p, f))
    # in place: arrays of the right size are written, not replaced; a wrong one is replaced
    sz = g.export_sizes()
    o = lib.Packed(np.full(sz[0], -7, np.int32), np.full(sz[0], -7, np.int32),
                   *[np.full(sz[i], np.nan) for i in range(1, 6)], np.zeros(3))
    keep = [o.kr, o.vr, o.s]
    o2 = g.export(out=o)
    assert o2 is o and o.kr is keep[0] and o.vr is keep[1] and o.s is keep[2]
    for f in ("kr", "kc", "vr", "vc", "er", "ec", "s", "f"):
        np.testing.assert_array_equal(getattr(o, f), getattr(p, f))
    x = inputs.standard_normal((w.points.shape[0], 3), seed=2)
    y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert_entries_close(y, oh2.matvec(A, x), 1e-13)
    y1 = g.matvec(torch.from_numpy(x[:, 1].copy()).cuda()).cpu().numpy()
    assert_entries_close(y1, oh2.matvec(A, x[:, 1]), 1e-13)
    assert_entries_close(g.to_dense().cpu().numpy(), oh2.to_dense(A), 1e-13)


@pytest.mark.parametrize("name,mode,eps,norm", [("cubes_1024", "paper", 1e-4, "fro"), ("cubes_1024", "sv", 1e-4, "fro"),
                                                ("cubes_2048_invr2", "paper", 1e-2, "fro"),
                                                ("uniform_1000_ragged", "paper", 1e-6, "fro"),
                                                ("sphere_700_ragged", "sv", 1e-3, "fro"),
                                                ("uniform_1000_ragged", "full", 0.0, "fro"),
                                                ("cubes_1024", "paper", 1e-4, "spectral"),
                                                ("sphere_700_ragged", "sv", 1e-3, "spectral")])
def test_product_matches_oracle(lib, name, mode, eps, norm):
    w, leaf, eta, A = oracle_case(name)
    # B: a different matrix on the same tree (other kernel), bases rotated so that
    # row and column bases differ
    wb = inputs.Workload("b", w.points, inputs.inv_r2_spec(w.spacing) if w.kernel.kind == 0 else inputs.laplace_spec(w.spacing), w.spacing)
    key = name + "_B"
    if key not in _cache:
        _cache[key] = oh2.rotate_bases(oh2.build(wb.points, wb.kernel, leaf, eta, 1e-4), seed=7)
    B = _cache[key]
    st = {}
    C = ommp.mmp(A, B, eps, mode, stats=st, norm=norm)
    ga = lib.h2_import(w.points, leaf, eta, pack(A))
    gb = lib.h2_import(w.points, leaf, eta, pack(B))
    gc = ga.mmp(gb, eps, trunc=mode, rank_cap=64 if mode != "full" else 0, norm=norm)
    info = gc.info()
    assert info["cap_hits"] == 0
    ckr, ckc = ranks(C)
    e = gc.export()
    np.testing.assert_array_equal(e.kr[: len(ckr)], ckr)
    np.testing.assert_array_equal(e.kc[: len(ckc)], ckc)
    d_gpu = gc.to_dense().cpu().numpy()
    d_orc = oh2.to_dense(C)
    assert_entries_close(d_gpu, d_orc, fp64_tol(eps, mode))
    if mode == "full":
        assert_entries_close(d_gpu, oh2.to_dense(A) @ oh2.to_dense(B))


def test_product_is_deterministic_and_reusable(lib):
    w, leaf, eta, A = oracle_case("cubes_1024")
    ga = lib.h2_import(w.points, leaf, eta, pack(A))
    c1 = ga.mmp(ga, 1e-4)
    d1 = c1.to_dense().cpu().numpy()
    c2 = ga.mmp(ga, 1e-4, out=c1)      # in place
    assert c2 is c1
    d2 = c1.to_dense().cpu().numpy()
    np.testing.assert_array_equal(d1, d2)
    assert_entries_close(d1, oh2.to_dense(ommp.mmp(A, A, 1e-4)))
    with pytest.raises(lib.H2Error) as ei:
        ga.mmp(ga, 1e-4, out=ga)       # the output must not be an operand
    assert ei.value.code == lib.H2_EINVAL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_products_of_products(lib, prec):
    # a product's output as an operand of later products (powers, solver iterations):
    # D = (A A) A against the oracle's chain, and an output rewritten in place and then
    # used again as an operand gives what fresh handles give
    w, leaf, eta, A = oracle_case("cubes_1024")
    p = lib.FP64 if prec == "fp64" else lib.MIXED_FP32
    ga = lib.h2_import(w.points, leaf, eta, pack(A))
    c = ga.mmp(ga, 1e-4, precision=p)
    d = c.mmp(ga, 1e-4, precision=p)
    C = ommp.mmp(A, A, 1e-4)
    D = ommp.mmp(C, A, 1e-4)
    if prec == "fp64":
        assert_entries_close(d.to_dense().cpu().numpy(), oh2.to_dense(D))
    else:
        assert rel(d.to_dense().cpu().numpy(), oh2.to_dense(D)) < 4e-4
    # c rewritten in place with another product, then an operand again
    ga.mmp(c, 1e-4, precision=p)                # c as the right operand too
    c3 = ga.mmp(ga, 1e-3, precision=p, out=c)   # in place: A A at another threshold
    assert c3 is c
    e1 = c.mmp(ga, 1e-4, precision=p).to_dense().cpu().numpy()
    f = ga.mmp(ga, 1e-3, precision=p)
    e2 = f.mmp(ga, 1e-4, precision=p).to_dense().cpu().numpy()
    np.testing.assert_array_equal(e1, e2)


def test_structure_mismatch_is_rejected(lib):
    w, leaf, eta, A = oracle_case("cubes_1024")
    w2, leaf2, eta2, A2 = oracle_case("uniform_1000_ragged")
    ga = lib.h2_import(w.points, leaf, eta, pack(A))
    gb = lib.h2_import(w2.points, leaf2, eta2, pack(A2))
    with pytest.raises(lib.H2Error) as ei:
        ga.mmp(gb, 1e-4)
    assert ei.value.code == lib.H2_ESTRUCT


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("name,mode,eps", [("cubes_1024", "paper", 1e-4), ("cubes_2048_invr2", "paper", 1e-3),
                                           ("uniform_1000_ragged", "paper", 1e-4), ("sphere_700_ragged", "sv", 1e-2)])
def test_mixed_product_within_2eps_of_oracle(lib, name, mode, eps, prec):
    # products in float32 (CUDA cores), as three TF32 products (tensor cores), or with the
    # couplings as three BF16 split products on the tensor cores; float32 accumulation;
    # float64 rank decisions and bases: the result must stay within 2 eps of the float64
    # oracle and be no less accurate against the exact product A B
    w, leaf, eta, A = oracle_case(name)
    st = {}
    C = ommp.mmp(A, A, eps, mode, stats=st)
    ga = lib.h2_import(w.points, leaf, eta, pack(A))
    gc = ga.mmp(ga, eps, precision=PRECISIONS[prec], trunc=mode)
    d_gpu = gc.to_dense().cpu().numpy()
    d_orc = oh2.to_dense(C)
    exact = oh2.to_dense(A) @ oh2.to_dense(A)
    assert rel(d_gpu, d_orc) < 2 * eps
    assert rel(d_gpu, exact) < 1.2 * rel(d_orc, exact) + 1e-6
    margin = BF16_MARGIN if prec == "bf16x3" else MIXED_MARGIN
    assert clear_rank_mismatches(gc.export(), st, A.L, margin) == []


def test_fp64_rank_bounds_do_not_change_results(lib):
    # the same product twice, the second time re-using the cached plan and output
    w, leaf, eta, A = oracle_case("sphere_700_ragged")
    ga = lib.h2_import(w.points, leaf, eta, pack(A))
    c1 = ga.mmp(ga, 1e-5, trunc="sv")
    c1 = ga.mmp(ga, 1e-5, trunc="sv", out=c1)
    d1 = c1.to_dense().cpu().numpy()
    C = ommp.mmp(A, A, 1e-5, "sv")
    assert_entries_close(d1, oh2.to_dense(C), fp64_tol(1e-5, "sv"))


@pytest.mark.parametrize("name,prec", [("cubes_1024", "fp64"), ("cubes_2048_invr2", "fp64"),
                                       ("uniform_1000_ragged", "mixed")])
def test_formatted_product_matches_oracle(lib, name, prec):
    # the comparison method of Sec. VI (fixed bases): float64 parity with the oracle,
    # mixed within 2 max(eps, 2e-5) with eps = 1e-4 as the scale
    w, leaf, eta, A = oracle_case(name)
    C = ommp.mmp(A, A, 0.0, "formatted")
    ga = lib.h2_import(w.points, leaf, eta, pack(A))
    gc = ga.mmp(ga, 0.0, trunc=lib.TRUNC_FORMATTED,
                precision=lib.FP64 if prec == "fp64" else lib.MIXED_FP32)
    d = gc.to_dense().cpu().numpy()
    e = gc.export()
    ckr, ckc = ranks(C)
    np.testing.assert_array_equal(e.kr, ckr)
    np.testing.assert_array_equal(e.kc, ckc)
    if prec == "fp64":
        assert_entries_close(d, oh2.to_dense(C))
    else:
        assert rel(d, oh2.to_dense(C)) < 2e-4


def test_batched_products_equal_single_products(lib):
    # independent instances of uneven size (config-4 style: stretched boxes)
    import torch
    hs = []
    for i, n in enumerate((700, 1500, 2600)):
        pts = inputs.stretched_box(n, seed=i)
        hs.append(lib.h2_build(pts, inputs.laplace_spec(n ** (-1 / 3)), 32, 1.0, 1e-4))
    cs = lib.h2_mmp_batched(hs, hs, 1e-4, precision=lib.MIXED_FP32)
    for h, c in zip(hs, cs):
        single = h.mmp(h, 1e-4, precision=lib.MIXED_FP32)
        x = torch.ones((h.n, 2), dtype=torch.float64, device="cuda")
        assert torch.equal(c.matvec(x), single.matvec(x))
    cs2 = lib.h2_mmp_batched(hs, hs, 1e-4, precision=lib.MIXED_FP32, outs=cs)
    assert all(a is b for a, b in zip(cs, cs2))


@pytest.mark.parametrize("n", [700, 2600])
def test_mixed_product_is_deterministic_with_odd_leaf_sizes(lib, n):
    # leaf clusters of 21 points give odd Gram dimensions; three runs must agree bit
    # for bit (fixed summation orders, no shared scratch between clusters)
    pts = inputs.stretched_box(n, seed=1)
    h = lib.h2_build(pts, inputs.laplace_spec(n ** (-1 / 3)), 32, 1.0, 1e-4)
    ex = [h.mmp(h, 1e-4, precision=lib.MIXED_FP32).export() for _ in range(3)]
    for e in ex[1:]:
        for f in ("kr", "kc", "vr", "vc", "er", "ec", "s", "f"):
            np.testing.assert_array_equal(getattr(e, f), getattr(ex[0], f))


@pytest.mark.parametrize("precision,trunc", [("mixed", "paper"), ("fp64", "paper"), ("mixed", "formatted"),
                                             ("bf16x3", "paper")])
def test_batched_graph_and_replay_equal_single(lib, precision, trunc):
    # instances of uneven size in one captured graph, one branch per product (the
    # repeated instance shares its plan with the first and gets its own slice of the
    # work space); the second call replays the graph.  Every result equals its single
    # product bit for bit (the tensor-core coupling pass included).
    import torch
    prec = {"mixed": lib.MIXED_FP32, "fp64": lib.FP64, "bf16x3": lib.MIXED_BF16X3}[precision]
    specs = [(900, 11, "box"), (1700, 12, "box"), (900, 11, "box"), (1200, 13, "uniform")]
    hs = []
    for n, seed, kind in specs:
        pts = inputs.stretched_box(n, seed=seed) if kind == "box" else inputs.workload_uniform(n, seed=seed).points
        hs.append(lib.h2_build(pts, inputs.laplace_spec(n ** (-1 / 3)), 32, 1.0, 1e-4))
    singles = [h.mmp(h, 1e-4, precision=prec, trunc=trunc) for h in hs]
    n0 = lib.kernel_launches()
    cs = lib.h2_mmp_batched(hs, hs, 1e-4, precision=prec, trunc=trunc)
    n1 = lib.kernel_launches()
    cs2 = lib.h2_mmp_batched(hs, hs, 1e-4, precision=prec, trunc=trunc, outs=cs)
    n2 = lib.kernel_launches()
    assert all(a is b for a, b in zip(cs, cs2))
    # the replay counts the kernels of the captured program
    assert n2 - n1 == n1 - n0 > 0
    for h, c, s in zip(hs, cs2, singles):
        x = torch.from_numpy(inputs.standard_normal((h.n, 3), seed=5)).cuda()
        assert torch.equal(c.matvec(x), s.matvec(x))
        assert c.info()["cap_hits"] == s.info()["cap_hits"]


def test_allocation_failure_during_a_product_leaves_the_library_usable(lib):
    # a product that needs a new program and a new output is refused at its 1st, 2nd,
    # ... device allocation until it gets through: every refused attempt fails with
    # H2_ENOMEM and leaves the library usable (what a refused attempt already built, such
    # as its cached program, is reused by the next one); the product that finally runs
    # equals one made without refusals, and an earlier product is unchanged
    import torch
    w, leaf, eta, A = oracle_case("cubes_1024")
    ga = lib.h2_import(w.points, leaf, eta, pack(A))
    ref = ga.mmp(ga, 1e-4, precision=lib.MIXED_FP32)
    x = torch.from_numpy(inputs.standard_normal((ga.n, 2), seed=3)).cuda()
    y_ref = ref.matvec(x)
    refused = 0
    c = None
    for k in range(0, 32):
        lib.set_alloc_limit(k)
        try:
            c = ga.mmp(ga, 1e-4, precision=lib.MIXED_FP32, rank_cap=40)
            break
        except lib.H2Error as e:
            assert e.code == lib.H2_ENOMEM
            refused += 1
        finally:
            lib.set_alloc_limit(-1)
    assert c is not None and refused >= 4
    assert c.info()["cap_hits"] == 0
    c2 = ga.mmp(ga, 1e-4, precision=lib.MIXED_FP32, rank_cap=40)
    assert torch.equal(c.matvec(x), c2.matvec(x))
    assert torch.equal(ga.mmp(ga, 1e-4, precision=lib.MIXED_FP32).matvec(x), y_ref)


def test_batched_instances_match_the_oracle(lib):
    # two instances of different size in one h2_mmp_batched call, each against the
    # oracle's product of the same matrices
    cases = [("uniform_1000_ragged", "paper", 1e-4), ("cubes_2048_invr2", "paper", 1e-3)]
    gs, orc = [], []
    for name, mode, eps in cases:
        w, leaf, eta, A = oracle_case(name)
        gs.append(lib.h2_import(w.points, leaf, eta, pack(A)))
        orc.append(oh2.to_dense(ommp.mmp(A, A, 1e-4, "paper")))
    cs = lib.h2_mmp_batched(gs, gs, 1e-4)
    for c, d in zip(cs, orc):
        assert_entries_close(c.to_dense().cpu().numpy(), d)
    cs = lib.h2_mmp_batched(gs, gs, 1e-4, outs=cs)        # the captured graph, replayed
    for c, d in zip(cs, orc):
        assert_entries_close(c.to_dense().cpu().numpy(), d)


@pytest.fixture(scope="module")
def big_case():
    # N = 20,480 on the 2x2 cube array (1024 leaves of 20 points, L = 10): levels with
    # 1024 and 2048 eigen tasks and ~10^5 segments per launch, the launch
    # configuration of the large workloads.  The oracle reads the far field at 16
    # points per partner block (an exact far field costs L N^2 kernel entries).
    wa = inputs.workload_cube_array(2, 2, 5120)
    wb = inputs.workload_cube_array(2, 2, 5120, kernel="invr2")
    A = oh2.build(wa.points, wa.kernel, 32, 1.0, 1e-4, far_sample=16)
    B = oh2.build(wb.points, wb.kernel, 32, 1.0, 1e-4, far_sample=16)
    st = {}
    C = ommp.mmp(A, B, 1e-4, "paper", stats=st)
    x = inputs.standard_normal((wa.points.shape[0], 4), seed=1)
    return wa, wb, A, B, C, st, x


def test_n20480_float64_product_matches_the_oracle(lib, big_case):
    import torch
    wa, wb, A, B, C, st, x = big_case
    ga = lib.h2_import(wa.points, 32, 1.0, pack(A))
    gb = lib.h2_import(wb.points, 32, 1.0, pack(B))
    gc = ga.mmp(gb, 1e-4)
    e = gc.export()
    ckr, ckc = ranks(C)
    np.testing.assert_array_equal(e.kr, ckr)
    np.testing.assert_array_equal(e.kc, ckc)
    y = gc.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert_entries_close(y, oh2.matvec(C, x))


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
def test_n20480_mixed_product_against_the_oracle(lib, big_case, prec):
    import torch
    wa, wb, A, B, C, st, x = big_case
    ga = lib.h2_import(wa.points, 32, 1.0, pack(A))
    gb = lib.h2_import(wb.points, 32, 1.0, pack(B))
    gm = ga.mmp(gb, 1e-4, precision=PRECISIONS[prec])
    ym = gm.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = oh2.matvec(C, x)
    y_exact = oh2.matvec(A, oh2.matvec(B, x))
    assert rel(ym, yo) < 2e-4
    assert rel(ym, y_exact) < 1.2 * rel(yo, y_exact)
    margin = BF16_MARGIN if prec == "bf16x3" else MIXED_MARGIN
    assert clear_rank_mismatches(gm.export(), st, A.L, margin) == []


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("n", [700, 2600])
def test_tensor_core_product_is_deterministic_and_tracks_float32(lib, n, prec):
    # the tensor-core products (3xTF32 everywhere, or the BF16 split couplings): reruns
    # bit for bit equal (fixed accumulation order), and close to the CUDA-core float32
    # products: Gram matrices agree to ~1e-6 (3xTF32) or ~4e-5 (BF16 split), so ranks may
    # differ only where an eigenvalue lies that close to the threshold (at most 2 % of the
    # clusters); such a flip moves C by the content of one near-threshold direction, so
    # C x agrees within 2 eps
    import torch
    pts = inputs.stretched_box(n, seed=1)
    h = lib.h2_build(pts, inputs.laplace_spec(n ** (-1 / 3)), 32, 1.0, 1e-4)
    t1 = h.mmp(h, 1e-4, precision=PRECISIONS[prec])
    t2 = h.mmp(h, 1e-4, precision=PRECISIONS[prec])
    f = h.mmp(h, 1e-4, precision=lib.MIXED_FP32)
    e1, e2, ef = t1.export(), t2.export(), f.export()
    for k in ("kr", "kc", "vr", "vc", "er", "ec", "s", "f"):
        np.testing.assert_array_equal(getattr(e1, k), getattr(e2, k))
    differ = int(np.sum(e1.kr != ef.kr) + np.sum(e1.kc != ef.kc))
    assert differ <= 0.02 * (len(e1.kr) + len(e1.kc)), differ
    x = torch.from_numpy(inputs.standard_normal((n, 3), seed=2)).cuda()
    yt, yf = t1.matvec(x), f.matvec(x)
    assert float(torch.linalg.norm(yt - yf) / torch.linalg.norm(yf)) < 2e-4


def test_bf16_split_couplings_run_on_the_tensor_cores(lib):
    # H2_MIXED_BF16X3: the coupling pass of every level whose tiles fit, and the dense
    # leaf products F F, run on the tensor-core kernel (trace kind "tc"); the
    # executed-flop counter covers the CUDA-core rest
    w, leaf, eta, A = oracle_case("cubes_2048_invr2")
    ga = lib.h2_import(w.points, leaf, eta, pack(A))
    ga.trace_enable(True)
    c = ga.mmp(ga, 1e-3, precision=lib.MIXED_BF16X3)
    kinds, levels, ms, fl, names = c.trace_read()
    ga.trace_enable(False)
    tc_levels = {int(lv) for k, lv, nm in zip(kinds, levels, names) if k == "tc" and nm == "coup"}
    assert A.L in tc_levels and len(tc_levels) >= 3
    assert [int(lv) for k, lv, nm in zip(kinds, levels, names) if k == "tc" and nm == "leaf_dense"] == [A.L]
    assert all(nm in ("coup", "leaf_dense") for k, nm in zip(kinds, names) if k == "tc")
    assert c.trace_flops() > 0 and c.info()["cap_hits"] == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_autotuned_products_equal_fixed_ones(lib, prec):
    # h2_opts.autotune: the first products of a program try the candidate launch
    # configurations of every GEMM and mixed eigen launch group and then keep the
    # fastest; every candidate sums each output in the same order, so all products equal
    # the untuned one
    w, leaf, eta, A = oracle_case("cubes_2048_invr2")
    ga = lib.h2_import(w.points, leaf, eta, pack(A))
    p = PRECISIONS[prec]
    ref = ga.mmp(ga, 1e-4, precision=p).export()
    c = None
    for _ in range(5):
        c = ga.mmp(ga, 1e-4, precision=p, autotune=True, out=c)
        e = c.export()
        for f in ("kr", "kc", "vr", "vc", "er", "ec", "s", "f"):
            np.testing.assert_array_equal(getattr(e, f), getattr(ref, f))


# ---------------------------------------------------------------- complex kernels
# The Helmholtz kernel exp(-j k r) / (4 pi r) (Sec. VI-B, scattering): complex matrices,
# complex float64 and mixed (complex float32) products on the GPU against the complex128
# oracle.
ZCASES = {
    # name: (points, leaf, eta, eps_h2 of A, eps_h2 of B, wavenumber)
    "sphere_640": (lambda: inputs.fibonacci_sphere(640, 1.5), 20, 1.0, 1e-5, 1e-3, 2 * math.pi),
    "sphere_2048_4lambda": (lambda: inputs.fibonacci_sphere(2048, 4.0), 64, 1.0, 1e-3, 1e-3, 2 * math.pi),
}


def zcase(name):
    key = "z_" + name
    if key not in _cache:
        fac, leaf, eta, ea, eb, k = ZCASES[name]
        pts = fac()
        n = pts.shape[0]
        h = math.sqrt(4 * math.pi * float(np.max(np.linalg.norm(pts, axis=1))) ** 2 / n)
        spec = inputs.helmholtz_spec(h, k)
        A = oh2.rotate_bases(oh2.build(pts, spec, leaf, eta, ea), seed=1)
        B = oh2.rotate_bases(oh2.build(pts, spec, leaf, eta, eb), seed=2)
        _cache[key] = (pts, leaf, eta, spec, A, B)
    return _cache[key]


@pytest.mark.parametrize("name", list(ZCASES))
def test_complex_import_export_matvec_and_dense(lib, name):
    import torch
    pts, leaf, eta, spec, A, B = zcase(name)
    p = pack(A)
    g = lib.h2_import(pts, leaf, eta, p)
    assert g.is_complex and g.info()["is_complex"]
    e = g.export()
    for f in ("kr", "kc", "vr", "vc", "er", "ec", "s", "f"):
        np.testing.assert_array_equal(getattr(e, f), getattr(p, f))
    x = inputs.standard_normal((pts.shape[0], 3), seed=2) + 1j * inputs.standard_normal((pts.shape[0], 3), seed=3)
    y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert_entries_close(y, oh2.matvec(A, x), 1e-13)
    assert_entries_close(g.to_dense().cpu().numpy(), oh2.to_dense(A), 1e-13)


@pytest.mark.parametrize("name,mode,eps,norm", [("sphere_640", "full", 0.0, "fro"), ("sphere_640", "paper", 1e-3, "fro"),
                                                ("sphere_640", "sv", 1e-3, "fro"), ("sphere_640", "paper", 1e-4, "spectral"),
                                                ("sphere_2048_4lambda", "paper", 1e-3, "fro"),
                                                ("sphere_2048_4lambda", "sv", 1e-2, "fro")])
def test_complex_product_matches_oracle(lib, name, mode, eps, norm):
    pts, leaf, eta, spec, A, B = zcase(name)
    st = {}
    C = ommp.mmp(A, B, eps, mode, stats=st, norm=norm)
    ga = lib.h2_import(pts, leaf, eta, pack(A))
    gb = lib.h2_import(pts, leaf, eta, pack(B))
    gc = ga.mmp(gb, eps, trunc=mode, rank_cap=128 if mode == "full" else 96, norm=norm)
    assert gc.is_complex and gc.info()["cap_hits"] == 0
    ckr, ckc = ranks(C)
    e = gc.export()
    np.testing.assert_array_equal(e.kr, ckr)
    np.testing.assert_array_equal(e.kc, ckc)
    d_gpu = gc.to_dense().cpu().numpy()
    assert_entries_close(d_gpu, oh2.to_dense(C), fp64_tol(eps, mode))
    if mode == "full":
        assert_entries_close(d_gpu, oh2.to_dense(A) @ oh2.to_dense(B))


def test_complex_build_approximates_the_helmholtz_kernel(lib):
    # h2_build with the Helmholtz kernel: the library's own complex construction
    from oracle import kernels
    import torch
    pts = inputs.fibonacci_sphere(2048, 4.0)
    spec = inputs.helmholtz_spec(math.sqrt(4 * math.pi * 16.0 / 2048), 2 * math.pi)
    g = lib.h2_build(pts, spec, 64, 1.0, 1e-4)
    assert g.is_complex
    K = kernels.dense(spec, pts)
    x = inputs.standard_normal((2048, 2), seed=4) + 1j * inputs.standard_normal((2048, 2), seed=5)
    y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, K @ x) < 1e-3
    c = g.mmp(g, 1e-3)
    y2 = c.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = g.matvec(g.matvec(torch.from_numpy(x).cuda())).cpu().numpy()
    assert rel(y2, ref) < math.sqrt(1e-3)
    with pytest.raises(lib.H2Error) as ei:
        g.mmp(g, 1e-3, precision=lib.MIXED_TF32X3)
    assert ei.value.code == lib.H2_EUNSUPPORTED


@pytest.mark.parametrize("name,mode,eps", [("sphere_640", "paper", 1e-3), ("sphere_640", "sv", 1e-3),
                                           ("sphere_2048_4lambda", "paper", 1e-3),
                                           ("sphere_2048_4lambda", "sv", 1e-2)])
def test_complex_mixed_product_against_the_oracle(lib, name, mode, eps):
    # complex float32 products (float2 operands and sums) with the float64 Hermitian
    # eigen-decomposition of the (float32) Gram sums: within 2 eps of the complex128
    # oracle, no less accurate against the exact product, equal ranks wherever the
    # oracle's decision is clear of the threshold, and reruns bitwise equal
    pts, leaf, eta, spec, A, B = zcase(name)
    st = {}
    C = ommp.mmp(A, B, eps, mode, stats=st)
    ga = lib.h2_import(pts, leaf, eta, pack(A))
    gb = lib.h2_import(pts, leaf, eta, pack(B))
    gm = ga.mmp(gb, eps, trunc=mode, rank_cap=96, precision=lib.MIXED_FP32)
    assert gm.is_complex and gm.info()["cap_hits"] == 0
    d_gpu = gm.to_dense().cpu().numpy()
    d_orc = oh2.to_dense(C)
    exact = oh2.to_dense(A) @ oh2.to_dense(B)
    assert rel(d_gpu, d_orc) < 2 * eps
    assert rel(d_gpu, exact) < 1.2 * rel(d_orc, exact) + 1e-6
    assert clear_rank_mismatches(gm.export(), st, A.L) == []
    e1 = gm.export()
    gm2 = ga.mmp(gb, eps, trunc=mode, rank_cap=96, precision=lib.MIXED_FP32)
    e2 = gm2.export()
    for f in ("kr", "kc", "vr", "vc", "er", "ec", "s", "f"):
        np.testing.assert_array_equal(getattr(e1, f), getattr(e2, f))
