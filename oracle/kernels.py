"""Kernel functions evaluated on point sets (oracle; test infrastructure only).

The paper's matrices come from capacitance extraction (static 1/r kernel) and
volume integral equations (oscillatory kernel) (Sec. VI).  The synthetic stand-ins:
  kind 0: 1/(4 pi r), self term = spec.diag
  kind 1: 1/r^2,      self term = spec.diag
  kind 2: exp(-j k r)/(4 pi r), self term = spec.diag + j spec.diag_im
A pair of distinct points at distance zero also takes the self term.
Pin: tests/test_oracle_h2.py checks entries against the formulas written out with
math.* on scalar pairs.
"""
from __future__ import annotations

import math

import numpy as np


def is_complex(spec) -> bool:
    return spec.kind == 2


def kernel_matrix(spec, x: np.ndarray, y: np.ndarray, same: np.ndarray | None = None) -> np.ndarray:
    """K(x_a, y_b) for rows x (m,3) and columns y (n,3).

    `same` (m, n) bool marks entries that are diagonal entries of the full matrix
    (same point); they get the self term.
    """
    d = x[:, None, :] - y[None, :, :]
    r = np.sqrt(d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2])
    zero = r == 0.0
    if same is not None:
        zero = zero | same
    rs = np.where(zero, 1.0, r)
    if spec.kind == 0:
        k = 1.0 / (4.0 * math.pi * rs)
        return np.where(zero, spec.diag, k)
    if spec.kind == 1:
        k = 1.0 / (rs * rs)
        return np.where(zero, spec.diag, k)
    if spec.kind == 2:
        k = np.exp(-1j * spec.wavenumber * rs) / (4.0 * math.pi * rs)
        return np.where(zero, spec.diag + 1j * spec.diag_im, k)
    raise ValueError(f"unknown kernel kind {spec.kind}")


def dense(spec, points: np.ndarray) -> np.ndarray:
    """The full N x N kernel matrix in user order."""
    n = points.shape[0]
    return kernel_matrix(spec, points, points, np.eye(n, dtype=bool))
