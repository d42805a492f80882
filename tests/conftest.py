import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


@pytest.fixture(scope="session")
def cube2x2_pair():
    """A (1/(4 pi r)) and B (1/r^2) on a 2x2 cube array, 512 points per cube."""
    from paper_1908_05218_gb300 import inputs
    from oracle import h2
    wa = inputs.workload_cube_array(2, 2, 512)
    wb = inputs.workload_cube_array(2, 2, 512, kernel="invr2")
    A = h2.build(wa.points, wa.kernel, 32, 1.0, 1e-4)
    B = h2.build(wb.points, wb.kernel, 32, 1.0, 1e-4)
    return wa, wb, A, B
