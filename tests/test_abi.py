"""CPU tests of the boundary: the library loads and exports every declared symbol."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "h2.h")


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1908_05218_gb300 import h2
    return h2.LIB_PATH


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(h2_[a-z_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("h2_build", "h2_mmp", "h2_matvec", "h2_to_dense", "h2_import", "h2_export", "h2_info",
              "h2_destroy", "h2_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (h2_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_lists_all_symbols(lib_path):
    from paper_1908_05218_gb300 import h2
    assert sorted(h2.SYMBOLS) == declared_functions()


def test_argument_errors_without_gpu(lib_path):
    # argument validation happens before any device work
    from paper_1908_05218_gb300 import h2
    lib = h2.load()
    assert lib.h2_build(None, 10, None, 32, 1.0, 1e-4, None, None) == h2.H2_EINVAL
    assert b"null" in lib.h2_last_error()
    assert lib.h2_mmp(None, None, 1e-4, None, None) == h2.H2_EINVAL
    assert lib.h2_matvec(None, None, None, 1) == h2.H2_EINVAL
    lib.h2_destroy(None)


def test_structs_match_the_header():
    from paper_1908_05218_gb300 import h2
    assert ctypes.sizeof(h2.Kernel) == 32
    assert ctypes.sizeof(h2.Opts) == 32
    src = open(HEADER).read()
    assert "int32_t max_rank_row[32]" in src
    # h2_opts field order as declared
    body = src[:src.index("} h2_opts;")].rsplit("typedef struct {", 1)[1]
    fields = re.findall(r"^\s*(?:int32_t|void\*)\s+(\w+);", body, re.M)
    assert fields == [f for f, _ in h2.Opts._fields_]
    for name, val in (("H2_FP64", 0), ("H2_MIXED_FP32", 1), ("H2_MIXED_TF32X3", 2), ("H2_MIXED_BF16X3", 3),
                      ("H2_NORM_FROBENIUS", 0), ("H2_NORM_SPECTRAL", 1)):
        assert re.search(rf"\b{name} = {val}\b", src), name


def test_options_are_validated_through_the_abi(lib_path):
    # h2_build checks its options before any device work, so this runs without a GPU
    import numpy as np

    from paper_1908_05218_gb300 import h2
    lib = h2.load()
    pts = np.random.default_rng(0).random((64, 3))
    k = h2.Kernel(0, 0.0, 1.0, 0.0)
    out = ctypes.c_void_p(0)

    def build(**kw):
        o = h2.make_opts(**kw)
        return lib.h2_build(pts.ctypes.data_as(ctypes.c_void_p), 64, ctypes.byref(k), 32, 1.0, 1e-4,
                            ctypes.byref(o), ctypes.byref(out))

    assert build(norm=2) == h2.H2_EINVAL
    assert build(precision=7) == h2.H2_EINVAL
    assert build(autotune=2) == h2.H2_EINVAL
    o = h2.make_opts()
    o.reserved = 5
    assert lib.h2_build(pts.ctypes.data_as(ctypes.c_void_p), 64, ctypes.byref(k), 32, 1.0, 1e-4, ctypes.byref(o),
                        ctypes.byref(out)) == h2.H2_EINVAL
    assert out.value is None
