"""Host-only checks of the product and matvec programs (no GPU).

h2_plan_selfcheck builds, for a point set, the program of C = A A in every truncation
mode, both precisions and two rank caps, plus the matvec programs, and validates every
access of every segment and eigen task against the live allocations of its region.
The geometries cover leaf sizes that are not multiples of four (storage caps round
up), ragged trees and η ≠ 1.
"""
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
    assert lib.plan_selfcheck(points(), leaf, eta, 1e-4) == 18


def test_selfcheck_rejects_bad_arguments(lib):
    with pytest.raises(lib.H2Error):
        lib.plan_selfcheck(np.zeros((10, 3)), 8, 1.0, 2.0)
