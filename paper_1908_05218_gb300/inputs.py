"""Seeded synthetic workloads: point clouds and kernel specifications.

This module holds the geometry generators shared by the CUDA path, the tests and
the CPU oracle.  It contains none of the product algorithm's arithmetic: it only
draws points (numpy PCG64 generators with fixed seeds) and states which kernel
function and diagonal value a workload uses.

The paper measures on capacitance-extraction and volume-integral-equation matrices
that are not available here (Sec. VI).  The generators below stand in for them with
the same kind of geometry: clustered surface points on arrays of unit cubes (the
capacitance-like case), a volume point cloud, a sphere surface for the oscillatory
kernel, and randomly stretched boxes for batches of uneven problems.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# kernel kinds; the numeric codes are part of the C ABI (include/h2.h)
LAPLACE = 0      # 1 / (4 pi r)
INV_R2 = 1       # 1 / r^2
HELMHOLTZ = 2    # exp(-j k r) / (4 pi r)


@dataclass(frozen=True)
class KernelSpec:
    kind: int
    diag: float            # value placed on the diagonal (r = 0)
    wavenumber: float = 0.0
    diag_im: float = 0.0


@dataclass(frozen=True)
class Workload:
    name: str
    points: np.ndarray     # (N, 3) float64, user order
    kernel: KernelSpec
    spacing: float         # mean spacing h used for the diagonal


def laplace_spec(h: float) -> KernelSpec:
    """1/(4 pi r) with the self term 1/(2 pi h) for mean spacing h."""
    return KernelSpec(LAPLACE, 1.0 / (2.0 * math.pi * h))


def inv_r2_spec(h: float) -> KernelSpec:
    """1/r^2 with the self term 1/h^2."""
    return KernelSpec(INV_R2, 1.0 / (h * h))


def helmholtz_spec(h: float, k: float) -> KernelSpec:
    """exp(-jkr)/(4 pi r) with self term 1/(2 pi h) - j k / (4 pi)."""
    return KernelSpec(HELMHOLTZ, 1.0 / (2.0 * math.pi * h), k, -k / (4.0 * math.pi))


def uniform_cube(n: int, seed: int = 0) -> np.ndarray:
    """n points uniform in the unit cube."""
    rng = np.random.default_rng(seed)
    return rng.random((n, 3))


def cube_array_surface(nx: int, ny: int, pts_per_cube: int = 4096, gap: float = 0.5,
                       seed: int = 0) -> np.ndarray:
    """Panel centroids on the six faces of an nx x ny array of unit cubes.

    Cube (a, b) occupies [a(1+gap), a(1+gap)+1] x [b(1+gap), b(1+gap)+1] x [0, 1].
    Each face carries a g x g grid of panel centroids, g = ceil(sqrt(pts/6)); a
    seeded permutation keeps pts_per_cube of the 6 g^2 centroids of each cube.
    """
    g = int(math.ceil(math.sqrt(pts_per_cube / 6.0)))
    c = (np.arange(g) + 0.5) / g
    u, v = np.meshgrid(c, c, indexing="ij")
    u = u.ravel()
    v = v.ravel()
    zero = np.zeros_like(u)
    one = np.ones_like(u)
    faces = [np.stack(f, axis=1) for f in (
        (zero, u, v), (one, u, v), (u, zero, v), (u, one, v), (u, v, zero), (u, v, one))]
    unit = np.concatenate(faces, axis=0)
    rng = np.random.default_rng(seed)
    out = []
    for a in range(nx):
        for b in range(ny):
            keep = rng.permutation(unit.shape[0])[:pts_per_cube]
            p = unit[np.sort(keep)].copy()
            p[:, 0] += a * (1.0 + gap)
            p[:, 1] += b * (1.0 + gap)
            out.append(p)
    return np.concatenate(out, axis=0)


def fibonacci_sphere(n: int, radius: float) -> np.ndarray:
    """n nearly uniform points on a sphere (golden-angle spiral)."""
    i = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = math.pi * (3.0 - math.sqrt(5.0)) * i
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def stretched_box(n: int, seed: int) -> np.ndarray:
    """n points uniform in a box with sides (1, s2, s3), s log-uniform in [1, 8]."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(0.0, math.log(8.0), size=2))
    return rng.random((n, 3)) * np.array([1.0, s[0], s[1]])


# ---------------------------------------------------------------- named workloads

def workload_uniform(n: int = 1024, seed: int = 0) -> Workload:
    """Points uniform in the unit cube with the Laplace kernel (volume spacing)."""
    h = n ** (-1.0 / 3.0)
    return Workload(f"uniform_cube_N{n}", uniform_cube(n, seed), laplace_spec(h), h)


def workload_batch(count: int = 48, n_min: int = 4096, n_max: int = 131072, seed: int = 0) -> list:
    """Independent instances of uneven size: instance i has N_i log-uniform in
    [n_min, n_max] and points uniform in a box with sides (1, s2, s3), s log-uniform in
    [1, 8] (seed seed + i), with the Laplace kernel at the box's volume spacing."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        s = np.exp(rng.uniform(0.0, math.log(8.0), size=2))
        pts = rng.random((n, 3)) * np.array([1.0, s[0], s[1]])
        h = (s[0] * s[1] / n) ** (1.0 / 3.0)
        out.append(Workload(f"box_{i}_N{n}", pts, laplace_spec(h), h))
    return out


def workload_cube_array(nx: int, ny: int, pts_per_cube: int = 4096, kernel: str = "laplace",
                        seed: int = 0) -> Workload:
    """Capacitance-like surface points on an nx x ny array of unit cubes."""
    pts = cube_array_surface(nx, ny, pts_per_cube, seed=seed)
    n = pts.shape[0]
    h = math.sqrt(6.0 * nx * ny / n)
    spec = laplace_spec(h) if kernel == "laplace" else inv_r2_spec(h)
    return Workload(f"cube_array_{nx}x{ny}_{kernel}_N{n}", pts, spec, h)


def workload_sphere(n: int, radius: float = 4.0, wavenumber: float = 2.0 * math.pi) -> Workload:
    pts = fibonacci_sphere(n, radius)
    h = math.sqrt(4.0 * math.pi * radius * radius / n)
    return Workload(f"sphere_N{n}", pts, helmholtz_spec(h, wavenumber), h)


def standard_normal(shape, seed: int) -> np.ndarray:
    """Seeded N(0,1) test vectors (the error metric's x)."""
    return np.random.default_rng(seed).standard_normal(shape)
