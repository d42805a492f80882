"""New cluster bases from normalised Gram sums (oracle; test infrastructure only).

Sec. III-C (leaf level) and Sec. IV-C (non-leaf level): each of a cluster's three Gram
matrices is scaled to unit norm, the scaled matrices are added, and the new basis (or
the new stacked transfer matrix) is made of the eigenvectors of that sum whose
eigenvalue, relative to the largest one, lies above the truncation threshold.

Readings taken here:
  * "normalised" = divided by the Frobenius norm (the default; the spectral norm on
    request, norm="spectral"); a Gram matrix that is exactly zero is left out of the
    sum;
  * the summed G is Hermitian positive semi-definite, so its SVD is its eigen-
    decomposition; the k-th vector is kept when lambda_k / lambda_1 > threshold with
    threshold = eps (mode "paper": the normalised singular values of G itself, the
    literal statement), eps**2 (mode "sv": the singular values of the stacked
    contributions, i.e. the square roots of lambda), or every vector (mode "full",
    used to pin the product: it makes every projection exact);
  * the eigen-decomposition is numpy.linalg.eigh (a library primitive); each kept
    vector is scaled to unit norm by eigh and its sign fixed so that its entry of
    largest magnitude (first such index) is real and positive.

Pins: tests/test_oracle_basis.py (orthonormality, the truncation bound lambda_{k+1}
<= thr * lambda_1 on the summed matrix, a hand-made matrix with known spectrum, and
rank monotonicity in eps).
"""
from __future__ import annotations

import numpy as np

PAPER, SV, FULL, FORMATTED = "paper", "sv", "full", "formatted"
FRO, SPECTRAL = "fro", "spectral"


def normalized_sum(grams, dim: int, dtype, norm: str = FRO) -> np.ndarray:
    """G = sum of G_m / ||G_m|| over the nonzero G_m (Sec. III-C, normalised sum);
    ||.|| is the Frobenius norm, or the spectral norm for norm="spectral"."""
    g = np.zeros((dim, dim), dtype=dtype)
    for gm in grams:
        if gm is None:
            continue
        nrm = np.linalg.norm(gm) if norm == FRO else np.linalg.norm(gm, 2)
        if nrm > 0.0:
            g = g + gm / nrm
    return g


def threshold(eps: float, mode: str) -> float:
    if mode == PAPER:
        return eps
    if mode == SV:
        return eps * eps
    if mode == FULL:
        return -np.inf
    raise ValueError(mode)


def fix_signs(u: np.ndarray) -> np.ndarray:
    u = u.copy()
    for c in range(u.shape[1]):
        col = u[:, c]
        p = int(np.argmax(np.abs(col)))
        a = col[p]
        if a != 0:
            u[:, c] = col * (np.conj(a) / abs(a))
    return u


def truncated_eigvecs(g: np.ndarray, eps: float, mode: str, cap: int | None = None):
    """Eigenvectors of the Hermitian PSD g whose eigenvalue exceeds thr * lambda_1.

    Returns (U, lam): U has orthonormal columns ordered by decreasing eigenvalue.
    """
    n = g.shape[0]
    if n == 0:
        return np.zeros((0, 0), dtype=g.dtype), np.zeros(0)
    lam, u = np.linalg.eigh(g)
    lam = lam[::-1]
    u = u[:, ::-1]
    if mode == FULL:
        k = n
    else:
        thr = threshold(eps, mode)
        lam1 = lam[0]
        if not lam1 > 0.0:
            k = 0
        else:
            k = int(np.sum(lam > thr * lam1))
    if cap is not None:
        k = min(k, cap)
    return fix_signs(u[:, :k]), lam
