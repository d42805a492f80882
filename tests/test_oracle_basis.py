"""Pins for oracle.basis: normalised Gram sum and truncated eigenvectors (Sec. III-C)."""
import numpy as np
import pytest

from oracle import basis as Bs


def _spd_with_spectrum(lam, seed=0, cplx=False):
    rng = np.random.default_rng(seed)
    n = len(lam)
    a = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    q, _ = np.linalg.qr(a)
    return (q * np.asarray(lam)) @ q.conj().T, q


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("mode,eps,expect", [("paper", 1e-3, 4), ("sv", 1e-3, 6), ("sv", 1e-1, 3),
                                             ("paper", 0.5, 1), ("full", 0.0, 8)])
def test_rank_follows_the_threshold(cplx, mode, eps, expect):
    lam = [2.0, 1.0, 0.5, 1e-2, 1.5e-3, 1e-5, 1e-7, 0.0]      # sorted, known spectrum
    g, q = _spd_with_spectrum(lam, cplx=cplx)
    u, got = Bs.truncated_eigvecs(g, eps, mode)
    assert u.shape[1] == expect
    np.testing.assert_allclose(got, lam, atol=1e-14)
    np.testing.assert_allclose(u.conj().T @ u, np.eye(expect), atol=1e-13)
    # span = the leading eigenvectors: same projector
    p_ref = q[:, :expect] @ q[:, :expect].conj().T
    np.testing.assert_allclose(u @ u.conj().T, p_ref, atol=1e-10)


def test_threshold_is_strict():
    g, _ = _spd_with_spectrum([1.0, 1e-2, 1e-4])
    u, _ = Bs.truncated_eigvecs(g, 1e-2 * (1 + 1e-9), "paper")
    assert u.shape[1] == 1
    u, _ = Bs.truncated_eigvecs(g, 1e-2 * (1 - 1e-9), "paper")
    assert u.shape[1] == 2


def test_normalized_sum_is_scale_free_and_skips_zeros():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((5, 3))
    b = rng.standard_normal((5, 2))
    ga, gb = a @ a.T, b @ b.T
    s1 = Bs.normalized_sum([ga, gb, np.zeros((5, 5)), None], 5, np.float64)
    s2 = Bs.normalized_sum([1e8 * ga, 1e-8 * gb], 5, np.float64)
    np.testing.assert_allclose(s1, s2, rtol=1e-13)
    assert abs(np.linalg.norm(Bs.normalized_sum([ga], 5, np.float64)) - 1.0) < 1e-14
    # each normalised component is seen: a tiny Gram still contributes its span
    u, _ = Bs.truncated_eigvecs(Bs.normalized_sum([1e12 * ga, 1e-12 * gb], 5, np.float64), 1e-6, "paper")
    assert u.shape[1] == 5


def test_zero_matrix_gives_rank_zero():
    u, _ = Bs.truncated_eigvecs(np.zeros((4, 4)), 1e-3, "paper")
    assert u.shape == (4, 0)


def test_sign_convention():
    g, _ = _spd_with_spectrum([3.0, 2.0, 1.0], seed=5)
    u, _ = Bs.truncated_eigvecs(g, 1e-3, "paper")
    for c in range(3):
        p = np.argmax(np.abs(u[:, c]))
        assert u[p, c] > 0


def test_spectral_normalisation_divides_by_the_largest_eigenvalue():
    # components with known spectra: the spectral-norm reading divides each by its
    # largest eigenvalue, the default by the root of the sum of squared eigenvalues
    ga, qa = _spd_with_spectrum([4.0, 1.0, 0.0, 0.0, 0.0], seed=3)
    gb, qb = _spd_with_spectrum([0.5, 0.5, 0.25, 0.0, 0.0], seed=4)
    s = Bs.normalized_sum([ga, gb], 5, np.float64, Bs.SPECTRAL)
    np.testing.assert_allclose(s, ga / 4.0 + gb / 0.5, atol=1e-14)
    f = Bs.normalized_sum([ga, gb], 5, np.float64)
    np.testing.assert_allclose(f, ga / np.sqrt(17.0) + gb / np.sqrt(0.5625), atol=1e-14)
