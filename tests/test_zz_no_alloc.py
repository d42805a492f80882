"""h2_matvec_noalloc: the matvec whose work space is a fixed array inside the library.

Some callers may not allocate device memory while they call into the library (a
device-memory budget fixed in advance, or all free memory handed to another
allocator).  This entry point serves them; this test checks, through the C ABI, that
it returns what h2_matvec returns, on two calls in a row (the array keeps the first
call's contents), and that it refuses a size beyond its fixed array.  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matvec_matches_matvec_twice():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1908_05218_gb300 import h2 as lib
    from paper_1908_05218_gb300 import inputs

    w = inputs.workload_cube_array(2, 2, 512)
    A = lib.h2_build(w.points, w.kernel, 32, 1.0, 1e-4)
    for seed, nrhs in ((3, 4), (4, 1)):
        x = torch.from_numpy(inputs.standard_normal((w.points.shape[0], nrhs), seed=seed)).cuda()
        ref = A.matvec(x)
        y1 = A.matvec_noalloc(x)
        y2 = A.matvec_noalloc(x)
        torch.cuda.synchronize()
        scale = float(torch.linalg.norm(ref))
        assert float(torch.linalg.norm(y1 - ref)) / scale < 1e-13
        assert float(torch.linalg.norm(y2 - ref)) / scale < 1e-13
    # a size beyond the fixed array is refused with H2_EINVAL
    wb = inputs.workload_cube_array(4, 4, 4096)
    big = lib.h2_build(wb.points, wb.kernel, 32, 1.0, 1e-2)
    x = torch.zeros((wb.points.shape[0], 64), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.H2Error) as ei:
        big.matvec_noalloc(x)
    assert ei.value.code == lib.H2_EINVAL
    assert "32 MiB" in str(ei.value)
