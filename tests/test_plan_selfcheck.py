"""Host-only checks of the product and matvec programs (no GPU).

h2_plan_selfcheck builds, for a point set, the program of C = A A in every truncation
mode, three precisions (float64, float32, BF16 split with the tensor-core coupling pass
and its operand tiles) and two rank caps, plus the matvec programs, and validates every
access of every segment and eigen task against the live allocations of its region.
The geometries cover leaf sizes that are not multiples of four (storage caps round
up), ragged trees and η ≠ 1.  h2_plan_digest hashes a program: the host builds it
with all its threads, and the program must not depend on their number.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1908_05218_gb300 import inputs


@pytest.fixture(scope="module")
def lib():
    from paper_1908_05218_gb300 import h2
    h2.load()
    return h2


@pytest.mark.parametrize("name,points,leaf,eta", [
    ("sphere_700", lambda: inputs.fibonacci_sphere(700, 2.0), 20, 1.5),
    ("uniform_777_leaf13", lambda: inputs.uniform_cube(777, 3), 13, 1.0),
    ("stretched_2600", lambda: inputs.stretched_box(2600, seed=1), 32, 1.0),
    ("cubes_1024", lambda: inputs.workload_cube_array(2, 2, 256).points, 32, 1.0),
    ("uniform_300_leaf7", lambda: inputs.uniform_cube(300, 9), 7, 0.7),
])
def test_every_program_stays_inside_its_allocations(lib, name, points, leaf, eta):
    assert lib.plan_selfcheck(points(), leaf, eta, 1e-4) == 26


def test_selfcheck_rejects_bad_arguments(lib):
    with pytest.raises(lib.H2Error):
        lib.plan_selfcheck(np.zeros((10, 3)), 8, 1.0, 2.0)


def test_program_cost_per_point_stays_bounded(lib):
    # Sec. V: at constant rank the product costs O(N).  On the cube array (1024 points
    # per cube) N goes from 16,384 to 65,536; the share of boundary clusters still falls
    # (pre-asymptotic), so the cost per point may rise a little, but far less than
    # the factor 4 of an O(N^2) method or of pairs emitted quadratically.
    per = []
    for nx in (4, 8):
        w = inputs.workload_cube_array(nx, nx, 1024)
        fl, sg, it = lib.plan_stats(w.points, 32, 1.0, 1e-4)
        n = w.points.shape[0]
        per.append((fl / n, sg / n, it / n))
    for a, b in zip(per[0], per[1]):
        assert b / a < 1.5, (per, b / a)


def test_allocation_failure_is_reported_cleanly(lib):
    # the first device allocation of h2_build is refused: the call fails with
    # H2_ENOMEM before any device work, and the limit is lifted afterwards
    pts = inputs.uniform_cube(500, 1)
    lib.set_alloc_limit(0)
    try:
        with pytest.raises(lib.H2Error) as e:
            lib.h2_build(pts, inputs.laplace_spec(500 ** (-1 / 3)), 32, 1.0, 1e-4)
        assert e.value.code == 2 and "allocation limit" in str(e.value)
    finally:
        lib.set_alloc_limit(-1)


def test_program_size_follows_the_truncation_rule(lib):
    # the paper and sv rules differ only in the threshold the eigen step applies, so
    # they share one program; the full rule keeps every eigenvector (larger caps, more
    # work); the formatted product keeps A's and B's bases and skips the Gram sums and
    # eigen-decompositions altogether (fewer segments and flops)
    w = inputs.workload_cube_array(2, 2, 1024)
    st = {t: lib.plan_stats(w.points, 32, 1.0, 1e-4, t) for t in ("paper", "sv", "full", "formatted")}
    assert st["paper"] == st["sv"]
    assert st["full"][0] > st["paper"][0]
    assert st["formatted"][0] < st["paper"][0] and st["formatted"][1] < st["paper"][1]


_DIGEST_CHILD = """
import sys
sys.path.insert(0, {root!r})
from paper_1908_05218_gb300 import h2, inputs
pts = inputs.workload_cube_array(4, 4, 1024).points
print(" ".join(str(h2.plan_digest(pts, 32, 1.0, 1e-4, p, t)) for p in (0, 1, 3) for t in ("paper", "formatted")))
"""


def test_program_does_not_depend_on_the_host_thread_count(lib):
    # N = 16,384: the launch groups are large enough for the parallel emission (each
    # thread writes a contiguous range of its loop, appended in index order)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = []
    for nt in ("1", "3", "8"):
        env = dict(os.environ, OMP_NUM_THREADS=nt)
        r = subprocess.run([sys.executable, "-c", _DIGEST_CHILD.format(root=root)], env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        out.append(r.stdout.split())
    assert out[0] == out[1] == out[2]
    assert len(set(out[0])) == len(out[0])  # the precisions and truncation modes differ


def test_digest_rejects_bad_arguments(lib):
    pts = inputs.uniform_cube(300, 9)
    with pytest.raises(lib.H2Error):
        lib.plan_digest(pts, 7, 0.7, 1e-4, precision=9)
    with pytest.raises(lib.H2Error):
        lib.plan_digest(pts, 7, 0.7, 1.5)
