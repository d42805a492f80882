"""CPU tests of the library's host construction (h2_build_packed: the steps of h2_build
without a GPU), read back into the oracle's representation.

The paper cites but does not describe its construction; what it must deliver is an H^2
matrix on the library's partition that approximates the kernel matrix to about eps_H2,
with orthonormal leaf bases and transfers (nested bases, Sec. II), and for the symmetric
kernels (1/(4 pi r), 1/r^2, and the complex-symmetric exp(-j k r)/(4 pi r)) column bases
equal to row bases, R = V S V^T.
"""
import math

import numpy as np
import pytest

from oracle import h2 as oh2
from oracle import kernels
from oracle.tree import build_partition, build_tree
from paper_1908_05218_gb300 import inputs

from oracle_bridge import unpack


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1908_05218_gb300 import h2
    return h2


CASES = {
    "cubes_laplace": (lambda: inputs.workload_cube_array(2, 2, 512), 32, 1e-4),
    "uniform_invr2": (lambda: inputs.Workload("u", inputs.uniform_cube(1500, seed=4), inputs.inv_r2_spec(1500 ** (-1 / 3)),
                                              1500 ** (-1 / 3)), 32, 1e-3),
    "sphere_helmholtz_4lambda": (lambda: inputs.workload_sphere(2048), 64, 1e-4),
    "sphere_helmholtz_1e-3": (lambda: inputs.workload_sphere(2048), 64, 1e-3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_host_construction_approximates_the_kernel(lib, name):
    fac, leaf, eps = CASES[name]
    w = fac()
    p = lib.build_packed(w.points, w.kernel, leaf, 1.0, eps)
    part = build_partition(build_tree(w.points, leaf), 1.0)
    h = unpack(p, part)
    K = kernels.dense(w.kernel, w.points)
    err = np.linalg.norm(oh2.to_dense(h) - K) / np.linalg.norm(K)
    assert err <= 2 * eps, err
    assert np.iscomplexobj(p.vr) == (w.kernel.kind == 2)
    # symmetric kernels: column bases are the row bases
    np.testing.assert_array_equal(p.kr, p.kc)
    np.testing.assert_array_equal(p.vr, p.vc)
    np.testing.assert_array_equal(p.er, p.ec)
    # orthonormal leaf bases and transfers: every expanded basis is orthonormal
    for l in range(h.L + 1):
        for t in range(1 << l):
            v = oh2.expand_basis(h, l, t)
            np.testing.assert_allclose(v.conj().T @ v, np.eye(v.shape[1]), atol=1e-10)
