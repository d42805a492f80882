"""Python binding of the C ABI in include/h2.h (argument marshalling only).

Every numeric step runs in the CUDA library libh2gb300.so; this module converts
numpy arrays and torch CUDA tensors to pointers and status codes to exceptions.
Importing it on a machine without the built library raises immediately: there is
no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libh2gb300.so")

H2_OK, H2_EINVAL, H2_ENOMEM, H2_ECUDA, H2_ESTRUCT, H2_ETIMEOUT, H2_EINTERNAL, H2_EUNSUPPORTED = range(8)
FP64, MIXED_FP32, MIXED_TF32X3, MIXED_BF16X3 = 0, 1, 2, 3
NORM_FROBENIUS, NORM_SPECTRAL = 0, 1
_NORM = {"fro": NORM_FROBENIUS, "spectral": NORM_SPECTRAL}
TRUNC_PAPER, TRUNC_SV, TRUNC_FULL, TRUNC_FORMATTED = 0, 1, 2, 3
_TRUNC = {"paper": TRUNC_PAPER, "sv": TRUNC_SV, "full": TRUNC_FULL, "formatted": TRUNC_FORMATTED}

# exported symbols and their signatures (checked by the CPU tests)
SYMBOLS = ["h2_build", "h2_import", "h2_import_complex", "h2_export", "h2_mmp", "h2_mmp_batched", "h2_matvec", "h2_matvec_noalloc", "h2_to_dense", "h2_info",
           "h2_tree_perm", "h2_level_blocks", "h2_trace_enable", "h2_trace_read", "h2_trace_flops", "h2_trace_phase", "h2_destroy",
           "h2_last_error", "h2_kernel_launches", "h2_plan_selfcheck", "h2_set_alloc_limit", "h2_plan_stats",
           "h2_plan_digest", "h2_build_packed"]


class H2Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"h2 status {code}: {msg}")
        self.code = code


class Kernel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("wavenumber", C.c_double), ("diag_re", C.c_double), ("diag_im", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("trunc", C.c_int32), ("rank_cap", C.c_int32), ("norm", C.c_int32),
                ("stream", C.c_void_p), ("autotune", C.c_int32), ("reserved", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("levels", C.c_int32), ("leaf_size", C.c_int32), ("l_min", C.c_int32),
                ("csp", C.c_int32), ("n_admissible", C.c_int64), ("n_dense", C.c_int64),
                ("max_rank_row", C.c_int32 * 32), ("max_rank_col", C.c_int32 * 32), ("bytes_stored", C.c_int64),
                ("device_bytes", C.c_int64), ("cap_hits", C.c_int64), ("mmp_ms", C.c_double),
                ("is_complex", C.c_int32), ("reserved", C.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} missing: run __graft_entry__.build() (the CUDA library is required)")
    lib = C.CDLL(path)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.h2_build.argtypes = [P, I64, C.POINTER(Kernel), I32, D, D, C.POINTER(Opts), C.POINTER(P)]
    lib.h2_import.argtypes = [P, I64, I32, D, P, P, P, P, P, P, P, P, C.POINTER(Opts), C.POINTER(P)]
    lib.h2_import_complex.argtypes = [P, I64, I32, D, P, P, P, P, P, P, P, P, C.POINTER(Opts), C.POINTER(P)]
    lib.h2_export.argtypes = [P, P, P, P, P, P, P, P, P, P]
    lib.h2_mmp.argtypes = [P, P, D, C.POINTER(Opts), C.POINTER(P)]
    lib.h2_mmp_batched.argtypes = [P, P, I32, D, C.POINTER(Opts), P]
    lib.h2_matvec.argtypes = [P, P, P, I64]
    lib.h2_matvec_noalloc.argtypes = [P, P, P, I64]
    lib.h2_to_dense.argtypes = [P, P]
    lib.h2_info.argtypes = [P, C.POINTER(Stats)]
    lib.h2_tree_perm.argtypes = [P, P]
    lib.h2_level_blocks.argtypes = [P, I32, P, P, P, P]
    lib.h2_trace_enable.argtypes = [P, I32]
    lib.h2_trace_read.argtypes = [P, I32, P, P, P, P, P]
    lib.h2_trace_flops.argtypes = [P, P]
    lib.h2_kernel_launches.argtypes = [P]
    lib.h2_plan_selfcheck.argtypes = [P, I64, I32, C.c_double, C.c_double, P]
    lib.h2_set_alloc_limit.argtypes = [I64]
    lib.h2_plan_stats.argtypes = [P, I64, I32, D, D, I32, P, P, P]
    lib.h2_plan_digest.argtypes = [P, I64, I32, D, D, I32, I32, P]
    lib.h2_build_packed.argtypes = [P, I64, C.POINTER(Kernel), I32, D, D, P, P, P, P, P, P, P, P, P]
    lib.h2_trace_phase.argtypes = [P, I32]
    lib.h2_trace_phase.restype = C.c_char_p
    lib.h2_destroy.argtypes = [P]
    lib.h2_destroy.restype = None
    lib.h2_last_error.restype = C.c_char_p
    for name in SYMBOLS:
        if name not in ("h2_destroy", "h2_last_error", "h2_trace_phase"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(code: int):
    if code != H2_OK:
        raise H2Error(code, load().h2_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


def make_opts(precision: int = FP64, trunc: str | int = "paper", rank_cap: int = 0, stream=None,
              norm: str | int = "fro", autotune: bool = False) -> Opts:
    t = _TRUNC[trunc] if isinstance(trunc, str) else int(trunc)
    nm = _NORM[norm] if isinstance(norm, str) else int(norm)
    if stream is None:
        try:
            import torch
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
        except Exception:  # pragma: no cover - torch without CUDA
            stream = None
    return Opts(precision, t, rank_cap, nm, stream, int(autotune), 0)


def make_kernel(spec) -> Kernel:
    return Kernel(int(spec.kind), float(spec.wavenumber), float(spec.diag), float(spec.diag_im))


@dataclass
class Packed:
    kr: np.ndarray
    kc: np.ndarray
    vr: np.ndarray
    vc: np.ndarray
    er: np.ndarray
    ec: np.ndarray
    s: np.ndarray
    f: np.ndarray


class H2Matrix:
    """Owning wrapper of an h2_handle (complex: the Helmholtz kernel or h2_import_complex)."""

    def __init__(self, handle: int, n: int, is_complex: bool = False):
        self.handle = C.c_void_p(handle)
        self.n = n
        self.is_complex = is_complex

    @property
    def dtype(self):
        import torch
        return torch.complex128 if self.is_complex else torch.float64

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().h2_destroy(self.handle)
            self.handle = C.c_void_p(0)

    def mmp(self, other: "H2Matrix", eps: float, precision: int = FP64, trunc="paper", rank_cap: int = 0,
            out: "H2Matrix | None" = None, stream=None, norm="fro", autotune: bool = False) -> "H2Matrix":
        """C = self x other (h2_mmp); `out` from an earlier identical call is overwritten in place."""
        o = make_opts(precision, trunc, rank_cap, stream, norm, autotune)
        h = C.c_void_p(out.handle.value if out is not None else 0)
        _check(load().h2_mmp(self.handle, other.handle, float(eps), C.byref(o), C.byref(h)))
        if out is not None and h.value == out.handle.value:
            return out
        return H2Matrix(h.value, self.n, self.is_complex)

    def matvec(self, x, y=None):
        """y = H x for a torch CUDA float64 (complex handles: complex128) x of shape (n,)
        or (n, nrhs) (h2_matvec)."""
        import torch
        if x.dtype != self.dtype:
            if self.is_complex:
                x = x.to(torch.complex128)
            else:
                raise TypeError("a real H^2 matrix multiplies float64 vectors")
        squeeze = x.dim() == 1
        X = x.reshape(self.n, -1)
        nrhs = X.shape[1]
        xc = X.t().contiguous()          # column-major n x nrhs
        yc = torch.empty_like(xc)
        _check(load().h2_matvec(self.handle, C.c_void_p(xc.data_ptr()), C.c_void_p(yc.data_ptr()), nrhs))
        out = yc.t()
        if y is not None:
            y.copy_(out.reshape(y.shape))
            return y
        return out[:, 0] if squeeze else out

    def matvec_noalloc(self, x):
        """y = H x through h2_matvec_noalloc (no allocation inside the library call)."""
        import torch
        squeeze = x.dim() == 1
        X = x.reshape(self.n, -1)
        xc = X.t().contiguous()
        yc = torch.empty_like(xc)
        _check(load().h2_matvec_noalloc(self.handle, C.c_void_p(xc.data_ptr()), C.c_void_p(yc.data_ptr()),
                                        X.shape[1]))
        out = yc.t()
        return out[:, 0] if squeeze else out

    def matvec_ptr(self, x_ptr: int, y_ptr: int, nrhs: int):
        _check(load().h2_matvec(self.handle, C.c_void_p(x_ptr), C.c_void_p(y_ptr), int(nrhs)))

    def to_dense(self):
        import torch
        out = torch.empty((self.n, self.n), dtype=self.dtype, device="cuda")
        _check(load().h2_to_dense(self.handle, C.c_void_p(out.data_ptr())))
        return out.t()                   # column-major buffer -> row-major view

    def info(self) -> dict:
        s = Stats()
        _check(load().h2_info(self.handle, C.byref(s)))
        L = s.levels
        return {"n": s.n, "levels": L, "leaf_size": s.leaf_size, "l_min": s.l_min, "csp": s.csp,
                "n_admissible": s.n_admissible, "n_dense": s.n_dense,
                "max_rank_row": list(s.max_rank_row[:L]), "max_rank_col": list(s.max_rank_col[:L]),
                "bytes_stored": s.bytes_stored, "device_bytes": s.device_bytes, "cap_hits": s.cap_hits,
                "mmp_ms": s.mmp_ms, "is_complex": bool(s.is_complex)}

    def export_sizes(self) -> np.ndarray:
        """Element counts of the packed arrays (h2_export with NULL arrays): entry 0 the
        length of kr and kc, entries 1..6 those of vr, vc, er, ec, s, f."""
        sizes = np.zeros(8, dtype=np.int64)
        _check(load().h2_export(self.handle, _ptr(sizes), None, None, None, None, None, None, None, None))
        return sizes

    def export(self, out: "Packed | None" = None) -> Packed:
        """The packed host arrays of this matrix (h2_export).  With `out`, its arrays are
        written in place (for example page-locked buffers the caller keeps); an array of
        `out` whose length, dtype or layout does not fit is replaced by a new one."""
        sizes = self.export_sizes()
        dt = np.complex128 if self.is_complex else np.float64

        def take(a, n, t):
            ok = (a is not None and isinstance(a, np.ndarray) and a.dtype == t and a.ndim == 1
                  and a.shape[0] == n and a.flags.c_contiguous and a.flags.writeable)
            return a if ok else np.zeros(n, t)

        o = out if out is not None else Packed(*([None] * 8))
        kr = take(o.kr, sizes[0], np.int32)
        kc = take(o.kc, sizes[0], np.int32)
        arrs = [take(getattr(o, k), sizes[i + 1], dt) for i, k in enumerate(("vr", "vc", "er", "ec", "s", "f"))]
        _check(load().h2_export(self.handle, _ptr(sizes), _ptr(kr), _ptr(kc), *[_ptr(a) for a in arrs]))
        if out is not None:
            out.kr, out.kc, out.vr, out.vc, out.er, out.ec, out.s, out.f = kr, kc, *arrs
            return out
        return Packed(kr, kc, *arrs)

    def trace_enable(self, on: bool = True):
        _check(load().h2_trace_enable(self.handle, int(on)))

    def trace_read(self) -> list:
        """Per launch group of the product that made this handle: (kind, level, ms, work):
        work = padded multiply-add flops of a GEMM group, clusters of an eigen group."""
        lib = load()
        cnt = C.c_int32(0)
        _check(lib.h2_trace_read(self.handle, 0, None, None, None, None, C.byref(cnt)))
        n = cnt.value
        kind = np.zeros(n, np.int32)
        level = np.zeros(n, np.int32)
        ms = np.zeros(n, np.float64)
        fl = np.zeros(n, np.float64)
        _check(lib.h2_trace_read(self.handle, n, _ptr(kind), _ptr(level), _ptr(ms), _ptr(fl), C.byref(cnt)))
        names = [lib.h2_trace_phase(self.handle, i).decode() for i in range(n)]
        return [("gemm", "eig", "memset", "tc")[k] for k in kind], level, ms, fl, names

    def trace_flops(self) -> float:
        v = C.c_double(0)
        _check(load().h2_trace_flops(self.handle, C.byref(v)))
        return v.value

    def tree_perm(self) -> np.ndarray:
        p = np.zeros(self.n, dtype=np.int64)
        _check(load().h2_tree_perm(self.handle, _ptr(p)))
        return p

    def level_blocks(self, level: int):
        lib = load()
        cnt = C.c_int64(0)
        _check(lib.h2_level_blocks(self.handle, level, None, None, None, C.byref(cnt)))
        t = np.zeros(cnt.value, np.int32)
        s = np.zeros(cnt.value, np.int32)
        k = np.zeros(cnt.value, np.int8)
        if cnt.value:
            _check(lib.h2_level_blocks(self.handle, level, _ptr(t), _ptr(s), _ptr(k), C.byref(cnt)))
        return t, s, k


def plan_selfcheck(points: np.ndarray, leaf_size: int = 32, eta: float = 1.0, eps: float = 1e-4) -> int:
    """Builds and validates every product and matvec program for these points on the
    host (no GPU); returns the number of programs checked, raises H2Error on a fault."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = C.c_int32(0)
    _check(load().h2_plan_selfcheck(_ptr(pts), pts.shape[0], leaf_size, float(eta), float(eps), C.byref(n)))
    return int(n.value)


def build_packed(points: np.ndarray, spec, leaf_size: int = 32, eta: float = 1.0, eps: float = 1e-4) -> Packed:
    """The host construction as packed arrays (no GPU; complex kernels give complex128
    arrays); h2_build runs the same steps on the GPU for the real kernels."""
    lib = load()
    pts = np.ascontiguousarray(points, dtype=np.float64)
    k = make_kernel(spec)
    sizes = np.zeros(8, dtype=np.int64)
    args = (_ptr(pts), pts.shape[0], C.byref(k), int(leaf_size), float(eta), float(eps))
    _check(lib.h2_build_packed(*args, _ptr(sizes), None, None, None, None, None, None, None, None))
    kr = np.zeros(sizes[0], np.int32)
    kc = np.zeros(sizes[0], np.int32)
    dt = np.complex128 if int(spec.kind) == 2 else np.float64
    arrs = [np.zeros(max(1, sizes[i]), dt) for i in range(1, 7)]
    ptrs = [a.view(np.float64).ctypes.data_as(C.c_void_p) for a in arrs]
    _check(lib.h2_build_packed(*args, _ptr(sizes), _ptr(kr), _ptr(kc), *ptrs))
    return Packed(kr, kc, *[a[:sizes[i + 1]] for i, a in enumerate(arrs)])


def set_alloc_limit(n: int) -> None:
    """Test hook: after n more device allocations every further one fails (n < 0: off)."""
    _check(load().h2_set_alloc_limit(int(n)))


def plan_stats(points: np.ndarray, leaf_size: int = 32, eta: float = 1.0, eps: float = 1e-4,
               trunc: str = "paper") -> tuple:
    """(flops, segments, items) of the program of C = A A for these points, on the host."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    fl, sg, it = C.c_double(0), C.c_int64(0), C.c_int64(0)
    _check(load().h2_plan_stats(_ptr(pts), pts.shape[0], leaf_size, float(eta), float(eps), _TRUNC[trunc],
                                C.byref(fl), C.byref(sg), C.byref(it)))
    return fl.value, int(sg.value), int(it.value)


def plan_digest(points: np.ndarray, leaf_size: int = 32, eta: float = 1.0, eps: float = 1e-4,
                precision: int = FP64, trunc: str = "paper") -> int:
    """64-bit digest of the program of C = A A for these points (h2_plan_digest), on the host."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    d = C.c_uint64(0)
    _check(load().h2_plan_digest(_ptr(pts), pts.shape[0], leaf_size, float(eta), float(eps), int(precision),
                                 _TRUNC[trunc], C.byref(d)))
    return int(d.value)


def kernel_launches() -> int:
    """CUDA kernels this library has launched in this process so far."""
    v = C.c_uint64(0)
    _check(load().h2_kernel_launches(C.byref(v)))
    return int(v.value)


def h2_mmp_batched(As, Bs, eps: float, precision: int = FP64, trunc="paper", rank_cap: int = 0,
                   outs=None, stream=None, norm="fro", autotune: bool = False) -> list:
    """[A_i x B_i] through h2_mmp_batched (independent products, in order on one stream)."""
    n = len(As)
    if len(Bs) != n:
        raise ValueError("A and B lists differ in length")
    o = make_opts(precision, trunc, rank_cap, stream, norm, autotune)
    ha = (C.c_void_p * n)(*[a.handle.value for a in As])
    hb = (C.c_void_p * n)(*[b.handle.value for b in Bs])
    hc = (C.c_void_p * n)(*[(outs[i].handle.value if outs else 0) for i in range(n)])
    _check(load().h2_mmp_batched(ha, hb, n, float(eps), C.byref(o), hc))
    res = []
    for i in range(n):
        if outs and hc[i] == outs[i].handle.value:
            res.append(outs[i])
        else:
            res.append(H2Matrix(hc[i], As[i].n, As[i].is_complex))
    return res


def h2_build(points: np.ndarray, spec, leaf_size: int = 32, eta: float = 1.0, eps: float = 1e-4,
             stream=None) -> H2Matrix:
    pts = np.ascontiguousarray(points, dtype=np.float64)
    k = make_kernel(spec)
    o = make_opts(stream=stream)
    h = C.c_void_p(0)
    _check(load().h2_build(_ptr(pts), pts.shape[0], C.byref(k), int(leaf_size), float(eta), float(eps),
                           C.byref(o), C.byref(h)))
    return H2Matrix(h.value, pts.shape[0], int(spec.kind) == 2)


def h2_import(points: np.ndarray, leaf_size: int, eta: float, p: Packed, stream=None) -> H2Matrix:
    """h2_import, or h2_import_complex when any array of p is complex (passed as
    interleaved real and imaginary parts)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    cplx = any(np.iscomplexobj(a) for a in (p.vr, p.vc, p.er, p.ec, p.s, p.f))
    if cplx:
        arrs = [np.ascontiguousarray(a, dtype=np.complex128).view(np.float64) for a in (p.vr, p.vc, p.er, p.ec, p.s, p.f)]
    else:
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (p.vr, p.vc, p.er, p.ec, p.s, p.f)]
    kr = np.ascontiguousarray(p.kr, dtype=np.int32)
    kc = np.ascontiguousarray(p.kc, dtype=np.int32)
    o = make_opts(stream=stream)
    h = C.c_void_p(0)
    fn = load().h2_import_complex if cplx else load().h2_import
    _check(fn(_ptr(pts), pts.shape[0], int(leaf_size), float(eta), _ptr(kr), _ptr(kc),
              *[_ptr(a) for a in arrs], C.byref(o), C.byref(h)))
    return H2Matrix(h.value, pts.shape[0], cplx)
