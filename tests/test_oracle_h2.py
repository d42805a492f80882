"""Pins for oracle.h2 and oracle.kernels: representation, matvec, construction."""
import math

import numpy as np
import pytest

from oracle import h2, kernels
from paper_1908_05218_gb300 import inputs


def test_kernel_entries_match_the_formulas():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 2.0]])
    y = np.array([[3.0, 0.0, 4.0], [0.0, 0.0, 0.0]])
    lap = inputs.laplace_spec(0.1)
    k = kernels.kernel_matrix(lap, x, y)
    assert k[0, 0] == pytest.approx(1 / (4 * math.pi * 5.0), rel=1e-15)
    assert k[1, 1] == pytest.approx(1 / (4 * math.pi * 3.0), rel=1e-15)
    assert k[0, 1] == lap.diag == pytest.approx(1 / (2 * math.pi * 0.1))
    inv = inputs.inv_r2_spec(0.5)
    assert kernels.kernel_matrix(inv, x, y)[0, 0] == pytest.approx(1 / 25.0, rel=1e-15)
    hel = inputs.helmholtz_spec(0.1, 2 * math.pi)
    v = kernels.kernel_matrix(hel, x, y)[1, 1]
    r = 3.0
    assert v == pytest.approx(complex(math.cos(2 * math.pi * r), -math.sin(2 * math.pi * r)) / (4 * math.pi * r), rel=1e-14)
    assert kernels.kernel_matrix(hel, x, y)[0, 1] == pytest.approx(complex(hel.diag, -2 * math.pi / (4 * math.pi)))


@pytest.fixture(scope="module")
def small_cube():
    w = inputs.workload_cube_array(2, 2, 256)
    return w, h2.build(w.points, w.kernel, 32, 1.0, 1e-6)


def test_matvec_equals_dense_product(small_cube):
    w, A = small_cube
    x = np.random.default_rng(2).standard_normal((w.points.shape[0], 3))
    D = h2.to_dense(A)
    np.testing.assert_allclose(h2.matvec(A, x), D @ x, rtol=0, atol=1e-13 * np.abs(D @ x).max())
    np.testing.assert_allclose(h2.matvec(A, x[:, 0]), D @ x[:, 0], atol=1e-13 * np.abs(D @ x).max())


def test_construction_accuracy_and_orthonormal_bases(small_cube):
    w, A = small_cube
    K = kernels.dense(w.kernel, w.points)
    err = np.linalg.norm(h2.to_dense(A) - K) / np.linalg.norm(K)
    assert err < 1e-5
    for l in range(A.L + 1):
        for t in range(1 << l):
            for col in (False, True):
                v = h2.expand_basis(A, l, t, col)
                np.testing.assert_allclose(v.T @ v, np.eye(v.shape[1]), atol=1e-12)
    assert A.part.blocks[A.L]
    assert any(k == "R" for l in range(A.L) for (_, _, k) in A.part.blocks[l])


def test_exact_when_far_field_is_kept_in_full():
    # eps_h2 below rounding keeps every singular vector: the representation is exact
    w = inputs.workload_uniform(300, seed=4)
    A = h2.build(w.points, w.kernel, 16, 1.0, 1e-30)
    K = kernels.dense(w.kernel, w.points)
    assert np.linalg.norm(h2.to_dense(A) - K) / np.linalg.norm(K) < 1e-13


def test_complex_kernel_roundtrip():
    w = inputs.workload_sphere(512, radius=1.0, wavenumber=2 * math.pi)
    A = h2.build(w.points, w.kernel, 32, 1.0, 1e-6)
    K = kernels.dense(w.kernel, w.points)
    assert A.dtype == np.complex128
    assert np.linalg.norm(h2.to_dense(A) - K) / np.linalg.norm(K) < 1e-5
    x = np.random.default_rng(0).standard_normal(512) + 1j * np.random.default_rng(1).standard_normal(512)
    D = h2.to_dense(A)
    np.testing.assert_allclose(h2.matvec(A, x), D @ x, atol=1e-13 * np.abs(D @ x).max())


def test_rotated_bases_represent_the_same_matrix(small_cube):
    _, A = small_cube
    Ar = h2.rotate_bases(A, seed=9)
    np.testing.assert_allclose(h2.to_dense(Ar), h2.to_dense(A), atol=1e-13 * np.abs(h2.to_dense(A)).max())
    assert not np.allclose(Ar.Vr[0], A.Vr[0])


def test_far_field_sampling_reduces_to_exact_and_keeps_accuracy():
    # far_sample at least the largest cluster: every partner is read whole, so the
    # result is the exact construction bit for bit; a small sample keeps the
    # construction accuracy within a factor 2 of the exact far field
    from oracle import kernels
    w = inputs.workload_cube_array(2, 2, 256)
    ex = h2.build(w.points, w.kernel, 32, 1.0, 1e-4)
    same = h2.build(w.points, w.kernel, 32, 1.0, 1e-4, far_sample=w.points.shape[0])
    np.testing.assert_array_equal(h2.to_dense(same), h2.to_dense(ex))
    smp = h2.build(w.points, w.kernel, 32, 1.0, 1e-4, far_sample=16)
    pts = w.points
    K = kernels.kernel_matrix(w.kernel, pts, pts, np.eye(len(pts), dtype=bool))
    e_ex = np.linalg.norm(h2.to_dense(ex) - K) / np.linalg.norm(K)
    e_smp = np.linalg.norm(h2.to_dense(smp) - K) / np.linalg.norm(K)
    assert e_smp < 2 * e_ex + 1e-12 and e_ex < 1e-3
