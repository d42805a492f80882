"""Benchmark of the H^2 matrix-matrix product C = A x B with change of bases.

One step = one full product (every phase of Sec. III-IV: basis products, dense
targets, Gram matrices, eigen-decompositions, projections, collects, couplings,
merges, the top-down split) on inputs resident in device memory.  The metric is
algorithmic throughput: (bytes of A + B + C at their actual ranks) / product time,
in GB/s, with the product time itself reported beside it.

  python bench.py [--gpus N --steps K --warmup W] [--workload cubes16x16|cubes4x4|batched48|sphere262k]
                  [--precision bf16x3|mixed|tf32x3|fp64] [--impl ours|reference] [--no-extras]

The headline precision is the BF16 split one (H2_MIXED_BF16X3: the coupling products on
the tensor cores as three BF16 products per split pair, the rest in float32, rank
decisions and bases in float64), the large-scale configuration's arithmetic.  Beside it
the line carries the same product in float32 (H2_MIXED_FP32), in float64 (the other arm
of the metric) and under the sv rule, each timed once after a warm-up, and an end-to-end
run for a caller with a new structure (program built inside the timed run).

--impl reference times the CPU oracle (the plain float64 restatement of the method)
on a bounded sample of the same geometry: the reference arm.
Multi-GPU: one product does not shard (every level exchanges neighbour blocks), so
N GPUs run N independent replicas; the value is the work of all replicas divided by
the slowest replica's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (nx, ny, points per cube, eps, description)
    "cubes16x16": (16, 16, 4096, 1e-4, "N=1,048,576 panel centroids on a 16x16 array of unit cubes"),
    "cubes4x4": (4, 4, 4096, 1e-4, "N=65,536 panel centroids on a 4x4 array of unit cubes"),
    "cubes2x2": (2, 2, 1024, 1e-4, "N=4,096 panel centroids on a 2x2 array of unit cubes"),
    "sample": (2, 2, 3072, 1e-4, "N=12,288 panel centroids on a 2x2 array of unit cubes"),
    "sample_ref": (2, 2, 2048, 1e-4, "N=8,192 panel centroids on a 2x2 array of unit cubes"),
}
# DRAM traffic of the float32 GEMM kernel (dram__bytes_read.sum + dram__bytes_write.sum)
# from one ncu capture of four of its launches -- the leaf level's dense targets, Gram
# pieces and case-1 Gram matrices of the N=65,536 cube-array product (BF16 split
# precision, the float32 kernel's share of it), 6.653 GB over 6.916e10 padded flops (2 m n
# k at the padded dims of their segments) -- valid only for the kernel source it was
# taken on (the hash of seg_gemm32_kernel's text).  A run's traffic per GEMM launch is
# that ratio times its own padded flops per GEMM launch.
TRAFFIC = {"kernel": "seg_gemm32_kernel", "src_sha256": "a6ae0b2f18ff361cf72fa4d4b5ee7b690290b40676dde85f96c615a0dbee48a5",
           "bytes": 6652807680.0, "padded_flops": 6.9159639040e10}
LEAF, ETA, EPS_H2 = 32, 1.0, 1e-4
# the variable-rank complex case: Fibonacci-sphere points, radius 4 wavelengths, Helmholtz
# kernel exp(-j k r) / (4 pi r) with k = 2 pi, leaf 64, eta 1, eps_trunc = eps_H2 = 1e-3,
# C = A A in complex float64
SPHERES = {
    # name: (points, leaf, eps, description)
    "sphere262k": (262144, 64, 1e-3, "N=262,144 points on a sphere of radius 4 wavelengths, Helmholtz kernel"),
    "sphere16k": (16384, 64, 1e-3, "N=16,384 points on a sphere of radius 4 wavelengths, Helmholtz kernel"),
    "sphere_sample": (4096, 64, 1e-3, "N=4,096 points on a sphere of radius 4 wavelengths, Helmholtz kernel"),
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """Samples nvidia-smi during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def reference_arm(args, sample="sample", threads=1):
    """The CPU oracle on a bounded sample of the workload (float64; its BLAS limited to
    `threads` host cores)."""
    nt = str(threads)
    env = dict(os.environ, OPENBLAS_NUM_THREADS=nt, OMP_NUM_THREADS=nt, MKL_NUM_THREADS=nt)
    t0 = time.time()
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-sample",
                          "--steps", str(args.steps), "--workload", sample], capture_output=True, text=True,
                         env=env)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    res = json.loads(out.stdout.strip().splitlines()[-1])
    res["wall_s"] = time.time() - t0
    return res


def oracle_sample(steps: int, sample: str = "sample"):
    """Child process: oracle product on N=12288 points of the cube-array geometry."""
    import numpy as np

    from oracle import h2 as oh2
    from oracle import mmp as ommp
    from paper_1908_05218_gb300 import inputs
    if sample in SPHERES:
        n, leaf, eps, _ = SPHERES[sample]
        wa = inputs.workload_sphere(n)
        A = oh2.build(wa.points, wa.kernel, leaf, ETA, eps)
        B = A
    else:
        nx, ny, ppc, eps, _ = WORKLOADS[sample]
        wa = inputs.workload_cube_array(nx, ny, ppc)
        wb = inputs.workload_cube_array(nx, ny, ppc, kernel="invr2")
        A = oh2.build(wa.points, wa.kernel, LEAF, ETA, EPS_H2)
        B = oh2.build(wb.points, wb.kernel, LEAF, ETA, EPS_H2)

    def size(h):
        n = sum(v.size for v in h.Vr.values()) + sum(v.size for v in h.Vc.values())
        n += sum(v.size for v in h.Er.values()) + sum(v.size for v in h.Ec.values())
        n += sum(v.size for v in h.S.values()) + sum(v.size for v in h.Fb.values())
        return (16 if np.iscomplexobj(next(iter(h.Fb.values()))) else 8) * n

    times = []
    C = None
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        C = ommp.mmp(A, B, eps, "paper")
        times.append(time.perf_counter() - t0)
    t = float(np.median(times))
    nbytes = size(A) + size(B) + size(C)
    print(json.dumps({"t": t, "bytes": nbytes, "n": int(wa.points.shape[0]), "steps": len(times)}))


def batched_main(args):
    """Config 4: 48 independent products A_i x A_i of uneven size (N_i log-uniform in
    [4096, 131072], points in stretched boxes), in chunks of 8 that fit the device
    memory together with their outputs.  Each chunk is one h2_mmp_batched call (one
    CUDA graph with a branch per product, captured once and replayed), timed against
    the same products one h2_mmp call at a time; the value is the bytes of all 48
    products over the sum of the chunks' times."""
    import torch

    from paper_1908_05218_gb300 import h2 as lib
    from paper_1908_05218_gb300 import inputs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    lib.load()
    prec = PRECISIONS[args.precision](lib)
    ws = inputs.workload_batch(48)
    eps, chunk = 1e-4, 8
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot_ms = tot_single = 0.0
    nbytes = 0
    nk = 0
    errs, ns = [], []
    build_s = 0.0
    with Clocks(0) as clk:
        for c0 in range(0, len(ws), chunk):
            part = ws[c0:c0 + chunk]
            t0 = time.time()
            hs = [lib.h2_build(w.points, w.kernel, LEAF, ETA, 1e-4) for w in part]
            build_s += time.time() - t0
            cs = lib.h2_mmp_batched(hs, hs, eps, precision=prec, trunc=args.trunc)
            for _ in range(args.warmup):
                cs = lib.h2_mmp_batched(hs, hs, eps, precision=prec, trunc=args.trunc, outs=cs)
            torch.cuda.synchronize()
            n0 = lib.kernel_launches()
            e0.record(stream)
            for _ in range(args.steps):
                cs = lib.h2_mmp_batched(hs, hs, eps, precision=prec, trunc=args.trunc, outs=cs)
            e1.record(stream)
            torch.cuda.synchronize()
            nk += lib.kernel_launches() - n0
            tot_ms += e0.elapsed_time(e1) / args.steps
            singles = [h.mmp(h, eps, precision=prec, trunc=args.trunc) for h in hs]
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                singles = [h.mmp(h, eps, precision=prec, trunc=args.trunc, out=c) for h, c in zip(hs, singles)]
            e1.record(stream)
            torch.cuda.synchronize()
            tot_single += e0.elapsed_time(e1) / args.steps
            for h, c, s_ in zip(hs, cs, singles):
                nbytes += 2 * h.info()["bytes_stored"] + c.info()["bytes_stored"]
                x = torch.from_numpy(inputs.standard_normal((h.n, 4), seed=1)).cuda()
                y = h.matvec(h.matvec(x))
                errs.append(float(torch.linalg.norm(c.matvec(x) - y) / torch.linalg.norm(y)))
                assert torch.equal(c.matvec(x), s_.matvec(x)), "merged and single products differ"
                ns.append(h.n)
            for h in singles + cs + hs:
                h.destroy()
            torch.cuda.empty_cache()
    print(json.dumps({
        "metric": "H2-MMP throughput, 48 independent products (bytes of A+A+C at actual ranks / batch time)",
        "value": nbytes / (tot_ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": "48 products A_i x A_i, N_i log-uniform in [4096, 131072] (total %d), points "
                               "uniform in boxes with sides (1, s2, s3), s log-uniform in [1, 8]; 1/(4 pi r), "
                               "leaf 32, eta 1, eps %g (%s rule)" % (sum(ns), eps, args.trunc),
                   "precision": args.precision,
                   "parallelism": "6 chunks of 8; per chunk one CUDA graph, one concurrent branch per product"},
        "ms_one_call_per_product": tot_single, "speedup_vs_one_call_per_product": tot_single / tot_ms,
        "gpu_launches_per_step": nk // args.steps, "max_rel_err_vs_exact_h2_matvecs": max(errs),
        "merged_equals_single": True, "n_min": min(ns), "n_max": max(ns), "build_s": build_s,
        "bytes_alg": nbytes, "clocks": clk.summary()}))


PRECISIONS = {"fp64": lambda lib: lib.FP64, "mixed": lambda lib: lib.MIXED_FP32,
              "tf32x3": lambda lib: lib.MIXED_TF32X3, "bf16x3": lambda lib: lib.MIXED_BF16X3}
DTYPES = {"fp64": "f64", "mixed": "f32+f64", "tf32x3": "tf32x3+f64", "bf16x3": "bf16x3+f32+f64"}
KERNELS = {"fp64": "seg_gemm_kernel<double>", "mixed": "seg_gemm32_kernel", "tf32x3": "seg_mma_tf32x3_kernel",
           "bf16x3": "seg_gemm32_kernel", "fp64c": "seg_zgemm_kernel", "mixedc": "seg_zgemm32_kernel"}


def trace_summary(C):
    """Per-kind, per-phase and per-level device times of the traced product of C."""
    kinds, levels, lms, lfl, lnames = C.trace_read()
    tot = {}
    for k, m_, f_ in zip(kinds, lms, lfl):
        tt = tot.setdefault(k, [0.0, 0.0, 0])
        tt[0] += m_
        tt[1] += f_
        tt[2] += 1
    by_phase, by_level, eig_by_level = {}, {}, {}
    for nm, m_ in zip(lnames, lms):
        by_phase[nm] = round(by_phase.get(nm, 0.0) + m_, 3)
    for lv, m_, kd in zip(levels, lms, kinds):
        by_level[int(lv)] = round(by_level.get(int(lv), 0.0) + m_, 3)
        if kd == "eig":
            eig_by_level[int(lv)] = round(eig_by_level.get(int(lv), 0.0) + m_, 3)
    return {"tot": tot, "phase_ms": {k: round(v[0], 3) for k, v in tot.items()}, "by_phase": by_phase,
            "by_level": dict(sorted(by_level.items())), "eig_by_level": dict(sorted(eig_by_level.items())),
            "executed_flops": C.trace_flops()}


def roofline(tr, precision):
    """Roofline entry of the GEMM kernel: multiply-add flops executed at the actual ranks
    (device counter) / the CUDA-event time of its launches, against the peak of the unit
    it runs on (float32 / float64 FMA lanes x 2 x max SM clock; for the 3xTF32 tensor-core
    kernel a third of the TF32 rate, half the measured dense BF16 rate)."""
    tot = tr["tot"]
    peaks, psrc = _peaks()
    clk_hz = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    if precision == "tf32x3":
        peak = 0.5 * float(peaks["bf16_tflops"]) / 3.0
        bound, peak_note = "tensor", f"TF32 = half the dense BF16 peak ({psrc}), / 3 products per split pair"
    elif precision in ("fp64", "fp64c"):
        peak = 152 * 2 * 2 * clk_hz / 1e12
        bound, peak_note = "alu", "152 SMs x 2 float64 FMA per clock x 2 flops x max SM clock"
    else:
        peak = 152 * 128 * 2 * clk_hz / 1e12
        bound, peak_note = "alu", "152 SMs x 128 float32 FMA lanes x 2 flops x max SM clock"
    gemm_ms = tot.get("gemm", [0.0])[0]
    fl = tr["executed_flops"]
    achieved = fl / (gemm_ms * 1e-3) / 1e12 if gemm_ms else 0.0
    dom = max(tot, key=lambda k: tot[k][0])
    traffic = None
    if precision in ("mixed", "bf16x3") and tot.get("gemm", [0, 0, 0])[2]:
        import hashlib
        src = open(os.path.join(ROOT, "paper_1908_05218_gb300", "csrc", "kernels.cu")).read()
        a = src.find("// ------------------------------------------------------------ segmented GEMM, float32")
        b = src.find("template <typename Acc>\nstatic void gemm_launch(")
        if a >= 0 and b > a and hashlib.sha256(src[a:b].encode()).hexdigest() == TRAFFIC["src_sha256"]:
            traffic = TRAFFIC["bytes"] / TRAFFIC["padded_flops"] * tot["gemm"][1] / tot["gemm"][2]
    eig = None
    if tot.get("eig", [0, 0, 0])[1]:
        e_ms, e_tasks, e_n = tot["eig"]
        eig = {"kernel": "eig_mixed_kept_kernel" if precision in ("mixed", "tf32x3", "bf16x3") else "eig_kernel",
               "bound": "latency", "ms_per_step": e_ms, "tasks_per_step": int(e_tasks), "launches_per_step": e_n,
               "sm_us_per_task": e_ms * 1e3 * 152 / e_tasks,
               "note": "one CTA per cluster basis: normalised Gram sum, Jacobi (barrier-separated "
                       "rotation steps), truncation; no throughput peak applies"}
    tc = None
    if tot.get("tc", [0, 0, 0])[2]:
        # the tensor-core coupling kernel (H2_MIXED_BF16X3): 2 m n k per item at the tile
        # dims of the plan (the device flop counter leaves it out), three BF16 products per
        # split pair against the dense BF16 peak
        t_ms, t_fl, t_n = tot["tc"]
        tpeak = float(peaks["bf16_tflops"]) / 3.0
        t_ach = t_fl / (t_ms * 1e-3) / 1e12 if t_ms else 0.0
        tc = {"kernel": "coup_tc_kernel", "bound": "tensor", "ms_per_step": t_ms, "launches_per_step": t_n,
              "flops_per_step": t_fl, "achieved": t_ach, "peak": tpeak, "unit": "TFLOP/s", "frac": t_ach / tpeak,
              "peak_note": f"dense BF16 ({psrc}) / 3 products per split pair",
              "note": "coupling sums: 2 m n k per item at the plan's padded dims / CUDA-event time"}
    return {"bound": bound, "kernel": KERNELS[precision], "dominant": dom, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak if peak else None, "traffic": traffic,
            "traffic_note": ("DRAM bytes per GEMM launch: bytes per padded flop of four captured launches "
                             "(N=65,536) x this run's padded flops per GEMM launch"
                             if traffic else "no DRAM capture of this kernel source at this precision"),
            "peak_note": peak_note, "launches_per_step": tot.get("gemm", [0, 0, 0])[2], "ms_per_step": gemm_ms,
            "executed_flops_per_step": fl, "eig": eig, "tc": tc,
            "note": "GEMM kernel: multiply-add flops executed at the actual ranks (device counter) / its "
                    "CUDA-event time"}


def side_arm(lib, A, B, eps, prec, trunc, x, y_ref, with_roofline=None, cap=None):
    """One more configuration of the same product: its first call (program built), one
    warm-up and one traced timed call; time, GB/s and Eq. error."""
    import torch
    kw = {} if cap is None else {"rank_cap": cap}
    try:
        t0 = time.time()
        C = A.mmp(B, eps, precision=prec, trunc=trunc, **kw)
        torch.cuda.synchronize()
        first = time.time() - t0
        C = A.mmp(B, eps, precision=prec, trunc=trunc, out=C, **kw)
        A.trace_enable(True)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        C = A.mmp(B, eps, precision=prec, trunc=trunc, out=C, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        tr = trace_summary(C)
        A.trace_enable(False)
        nbytes = A.info()["bytes_stored"] + B.info()["bytes_stored"] + C.info()["bytes_stored"]
        err = float(torch.linalg.norm(C.matvec(x) - y_ref) / torch.linalg.norm(y_ref))
        out = {"trunc": trunc, "precision": {0: "fp64", 1: "mixed", 2: "tf32x3", 3: "bf16x3"}.get(prec, prec), "ms": ms,
               "value": nbytes / (ms * 1e-3) / 1e9, "unit": "GB/s", "rel_err_vs_exact_h2_matvecs": err,
               "first_product_s_incl_plan": first, "warmup": 1, "steps": 1, "phase_ms": tr["phase_ms"],
               "max_rank_row": C.info()["max_rank_row"]}
        if with_roofline:
            out["roofline"] = roofline(tr, with_roofline)
        C.destroy()
        return out
    except Exception as e:  # reported, not fatal
        return {"error": str(e)[-300:]}


def _arrays(p):
    return (p.kr, p.kc, p.vr, p.vc, p.er, p.ec, p.s, p.f)


def _clear_cuda_error():
    """Clears the last-error state that a refused (non-sticky) host registration left in
    torch's CUDA runtime for this thread."""
    import ctypes
    try:
        ctypes.CDLL("libcudart.so.13").cudaGetLastError()
    except (OSError, AttributeError):
        pass


class PageLocked:
    """Page-locks the large arrays of packed matrices (cudaHostRegister through torch's
    CUDA runtime) for the duration of a `with` block, so that the host<->device copies of
    the end-to-end run go from and to pinned host memory, as a caller that keeps its
    matrices in pinned buffers has them.  Registration faults every page in, outside the
    timed region; an array the runtime refuses stays pageable (the library then pins it
    for the copy itself)."""
    MIN_BYTES = 64 << 20

    def __init__(self, *packs):
        self.arrays = [a for p in packs for a in _arrays(p) if a is not None and a.nbytes >= self.MIN_BYTES]
        self.ptrs = []
        self.bytes = 0

    def __enter__(self):
        import torch
        rt = torch.cuda.cudart()
        for a in self.arrays:
            if rt.cudaHostRegister(a.ctypes.data, a.nbytes, 0) == rt.cudaError.success:
                self.ptrs.append(a.ctypes.data)
                self.bytes += a.nbytes
            else:
                _clear_cuda_error()
        return self

    def __exit__(self, *exc):
        import torch
        rt = torch.cuda.cudart()
        torch.cuda.synchronize()
        for p in self.ptrs:
            if rt.cudaHostUnregister(p) != rt.cudaError.success:
                _clear_cuda_error()
        self.ptrs = []
        return False


def end_to_end(lib, wa, wb, pa, pbk, eps, prec, trunc, nbytes, c_sizes=None):
    """Through the public API with host buffers: h2_import of A and B from host arrays,
    h2_mmp, h2_export of C into host arrays; bytes counted from the arrays.  The arrays
    (A's and B's, and with c_sizes = C's packed sizes a set for C made beforehand) are
    page-locked before the timed region."""
    import numpy as np
    import torch
    h2d = sum(a.nbytes for a in _arrays(pa)) + sum(a.nbytes for a in _arrays(pbk))
    pc = None
    if c_sizes is not None:
        dt = pa.f.dtype
        pc = lib.Packed(np.empty(c_sizes[0], np.int32), np.empty(c_sizes[0], np.int32),
                        *[np.empty(int(c_sizes[i]), dt) for i in range(1, 7)])
    with PageLocked(pa, pbk, *([pc] if pc is not None else [])) as pin:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A2 = lib.h2_import(wa.points, LEAF, ETA, pa)
        B2 = lib.h2_import(wb.points, LEAF, ETA, pbk)
        C2 = A2.mmp(B2, eps, precision=prec, trunc=trunc)
        pc = C2.export(out=pc)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        pinned = pin.bytes
    d2h = sum(a.nbytes for a in _arrays(pc))
    for h in (C2, B2, A2):
        h.destroy()
    return {"value": nbytes / te / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "seconds": te, "steps": 1, "pinned_bytes": int(pinned)}


def sphere_main(args):
    """The variable-rank complex case (scattering, Sec. VI-B): C = A A for the Helmholtz
    kernel on a sphere on the GPU (mixed: complex float32 products with the float64
    Hermitian eigen step; or complex float64), against the oracle's complex128 product on
    a 4,096-point sample of the same geometry (one core).  With a mixed headline the
    line also carries the complex float64 product of the same matrices."""
    import torch

    from paper_1908_05218_gb300 import h2 as lib
    from paper_1908_05218_gb300 import inputs
    cpu = None
    if not args.no_cpu_baseline:
        try:
            cpu = reference_arm(argparse.Namespace(steps=1), "sphere_sample")
        except Exception as e:  # reported, not fatal
            cpu = {"error": str(e)[-300:]}
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    lib.load()
    n, leaf, eps, desc = SPHERES[args.workload]
    w = inputs.workload_sphere(n)
    t0 = time.time()
    A = lib.h2_build(w.points, w.kernel, leaf, ETA, eps)
    build_s = time.time() - t0
    stream = torch.cuda.current_stream()
    t0 = time.time()
    # (rank cap 128: ranks of the oscillatory kernel grow with the electrical size of the
    # coarse clusters)
    cap = 128
    # complex products run in float64 or complex float32 (the tensor-core splits are real
    # only): the split precisions take the complex float32 product
    if args.precision not in ("fp64", "mixed"):
        args.precision = "mixed"
    prec = PRECISIONS[args.precision](lib)
    C = A.mmp(A, eps, precision=prec, rank_cap=cap)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    for _ in range(args.warmup):
        C = A.mmp(A, eps, precision=prec, rank_cap=cap, out=C)
    A.trace_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with Clocks(0) as clk:
        n0 = lib.kernel_launches()
        e0.record(stream)
        for _ in range(args.steps):
            C = A.mmp(A, eps, precision=prec, rank_cap=cap, out=C)
        e1.record(stream)
        torch.cuda.synchronize()
        nk = lib.kernel_launches() - n0
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    tr = trace_summary(C)
    A.trace_enable(False)
    ia, ic = A.info(), C.info()
    nbytes = 2 * ia["bytes_stored"] + ic["bytes_stored"]
    x = torch.from_numpy(inputs.standard_normal((n, 4), seed=1) + 1j * inputs.standard_normal((n, 4), seed=2)).cuda()
    y_ref = A.matvec(A.matvec(x))
    err = float(torch.linalg.norm(C.matvec(x) - y_ref) / torch.linalg.norm(y_ref))
    roof = roofline(tr, "fp64c" if args.precision == "fp64" else "mixedc")
    ranks_C, cap_hits = ic["max_rank_row"], ic["cap_hits"]
    extras = {}
    if args.precision != "fp64" and not args.no_extras:
        C.destroy()
        C = None
        # the complex float64 product of the same matrices (one warm-up, one traced call)
        extras["fp64"] = side_arm(lib, A, A, eps, lib.FP64, "paper", x, y_ref, with_roofline="fp64c", cap=cap)
    cpu_line = None
    if cpu and "t" in cpu:
        cpu_line = {"value": cpu["bytes"] / cpu["t"] / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                    "sample": f"sphere of radius 4 wavelengths, N={cpu['n']}, one product A A, eps {eps}",
                    "seconds": cpu["t"]}
    elif cpu:
        cpu_line = {"error": cpu.get("error")}
    line = {
        "metric": "H2-MMP throughput, complex (bytes of A+A+C at actual ranks / product time)",
        "value": nbytes / (ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128" if args.precision == "fp64" else "c64+c128", "data": "synthetic",
        "config": {"workload": f"{desc}: exp(-j k r)/(4 pi r), k = 2 pi; leaf {leaf}, eta {ETA}, "
                               f"eps_trunc {eps} (paper rule), eps_H2 {eps}; rank cap {cap}; C = A A",
                   "precision": args.precision,
                   "inputs": "A, C together exceed L2 (no flush needed)", "parallelism": "replicas"},
        "mmp_s": ms * 1e-3, "rel_err_vs_exact_h2_matvecs": err, "ranks_C_max_row": ranks_C,
        "cap_hits": cap_hits, "bytes_alg": nbytes, "build_s": build_s, "first_product_s_incl_plan": setup_s,
        "phase_ms": tr["phase_ms"], "phase_ms_by_name": tr["by_phase"], "eig_ms_by_level": tr["eig_by_level"],
        "roofline": roof, "cpu_baseline": cpu_line, "gpu_launches": int(nk),
        "clocks": clk.summary()}
    line.update(extras)
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cubes16x16", choices=list(WORKLOADS) + ["batched48"] + list(SPHERES))
    ap.add_argument("--precision", default="bf16x3", choices=list(PRECISIONS))
    ap.add_argument("--trunc", default="paper", choices=["paper", "sv", "formatted"],
                    help="truncation rule; 'formatted' = fixed bases (the paper's comparison method)")
    ap.add_argument("--oracle-sample", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="h2_opts.autotune for the headline product (the warm-up products explore)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the sv-rule, float64 and new-structure end-to-end runs")
    args = ap.parse_args()

    if args.oracle_sample:
        oracle_sample(args.steps, args.workload if (args.workload.startswith("sample") or args.workload in SPHERES)
                      else "sample")
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload == "batched48":
        if args.impl == "reference" or world > 1:
            raise SystemExit("batched48 runs on one GPU, own implementation only")
        batched_main(args)
        return
    if args.workload in SPHERES:
        if args.impl == "reference" or world > 1:
            raise SystemExit("the sphere workloads run on one GPU, own implementation only")
        sphere_main(args)
        return
    nx, ny, ppc, eps, desc = WORKLOADS[args.workload]
    metric = "H2-MMP throughput (bytes of A+B+C at actual ranks / product time)"

    if args.impl == "reference":
        if rank != 0:
            return
        # (a smaller sample than the in-line CPU baseline, so that K steps stay within
        # a few minutes: about 8 s per step on one Neoverse-V2 core)
        r = reference_arm(args, "sample_ref")
        gbs = r["bytes"] / r["t"] / 1e9
        line = {"metric": metric, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus, "steps": r["steps"],
                "warmup": 0, "ms_per_step": r["t"] * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": f"cube array 2x2, 2048 points per cube (N={r['n']}), leaf {LEAF}, "
                                       f"eta {ETA}, eps {eps}, A: 1/(4 pi r), B: 1/r^2",
                           "sample_of": desc},
                "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                 "sample": f"N={r['n']} product, median of {r['steps']}"},
                "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    # CPU baseline first, in a child process started before any CUDA call
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = reference_arm(argparse.Namespace(steps=1))
            ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
            if ncores > 1 and not args.no_extras:
                ac = reference_arm(argparse.Namespace(steps=1), threads=ncores)
                ac["cores"] = ncores
                cpu["all_cores"] = ac
        except Exception as e:  # reported, not fatal
            cpu = {"error": str(e)[-300:]}

    import numpy as np
    import torch

    from paper_1908_05218_gb300 import h2 as lib
    from paper_1908_05218_gb300 import inputs, replicas

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib.load()
    prec = PRECISIONS[args.precision](lib)

    wa = inputs.workload_cube_array(nx, ny, ppc)
    wb = inputs.workload_cube_array(nx, ny, ppc, kernel="invr2")
    t0 = time.time()
    A = lib.h2_build(wa.points, wa.kernel, LEAF, ETA, EPS_H2)
    B = lib.h2_build(wb.points, wb.kernel, LEAF, ETA, EPS_H2)
    build_s = time.time() - t0
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(inputs.standard_normal((wa.points.shape[0], 4), seed=1)).cuda()
    y_ref = A.matvec(B.matvec(x))          # Eq. error: exact H^2 matvecs

    C = None
    at = bool(args.autotune)
    t0 = time.time()
    C = A.mmp(B, eps, precision=prec, trunc=args.trunc, out=C, autotune=at)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    for _ in range(args.warmup):
        C = A.mmp(B, eps, precision=prec, trunc=args.trunc, out=C, autotune=at)
    torch.cuda.synchronize()

    A.trace_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        n_launch0 = lib.kernel_launches()
        ev0.record(stream)
        for _ in range(args.steps):
            C = A.mmp(B, eps, precision=prec, trunc=args.trunc, out=C, autotune=at)
        ev1.record(stream)
        torch.cuda.synchronize()
        n_launch = lib.kernel_launches() - n_launch0
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / max(1, args.steps)
    ms = replicas.slowest(ms, dist, device="cuda")
    tr = trace_summary(C)
    A.trace_enable(False)

    ia, ib, ic = A.info(), B.info(), C.info()
    nbytes = ia["bytes_stored"] + ib["bytes_stored"] + ic["bytes_stored"]
    value = replicas.throughput(nbytes, world, ms)
    rel_err = float(torch.linalg.norm(C.matvec(x) - y_ref) / torch.linalg.norm(y_ref))
    roof = roofline(tr, args.precision)
    ranks_C = ic["max_rank_row"]
    cap_hits = ic["cap_hits"]
    c_sizes = C.export_sizes()
    C.destroy()

    extras = {}
    # end to end through the public API with host buffers: upload A and B from host
    # arrays, the product, download C (structure and program cached from the runs above)
    e2e = None
    if not args.no_e2e and rank == 0:
        pa, pbk = A.export(), B.export()
        e2e = end_to_end(lib, wa, wb, pa, pbk, eps, prec, args.trunc, nbytes, c_sizes)
    if rank == 0 and not args.no_extras:
        # the same product with the sv rule (thresholds eps^2: error ~ eps)
        extras["sv_rule"] = side_arm(lib, A, B, eps, prec, "sv", x, y_ref)
        # the float64 arm of the metric: the same product, every step in float64
        if args.precision != "fp64":
            extras["fp64"] = side_arm(lib, A, B, eps, lib.FP64, args.trunc, x, y_ref, with_roofline="fp64")
        # the float32 product (every small product on the CUDA cores)
        if args.precision not in ("fp64", "mixed"):
            extras["mixed_fp32"] = side_arm(lib, A, B, eps, lib.MIXED_FP32, args.trunc, x, y_ref, with_roofline="mixed")
    # end to end for a caller with a new structure: every handle is released first, so
    # that the tree, the partition and the product program are built inside the timed run
    e2e_cold = None
    if not args.no_e2e and rank == 0 and not args.no_extras:
        pa, pbk = A.export(), B.export()
        A.destroy()
        B.destroy()
        e2e_cold = end_to_end(lib, wa, wb, pa, pbk, eps, prec, args.trunc, nbytes, c_sizes)

    if rank == 0:
        cpu_line = None
        if cpu and "t" in cpu:
            cpu_line = {"value": cpu["bytes"] / cpu["t"] / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                        "sample": f"cube array 2x2, 3072 points per cube (N={cpu['n']}), one product, eps {eps}",
                        "seconds": cpu["t"]}
            if cpu.get("all_cores"):
                ac = cpu["all_cores"]
                cpu_line["all_cores"] = {"value": ac["bytes"] / ac["t"] / 1e9, "unit": "GB/s",
                                         "cores": ac["cores"], "seconds": ac["t"],
                                         "note": "the same oracle with every host core open to its BLAS"}
        elif cpu:
            cpu_line = {"error": cpu.get("error")}
        line = {
            "metric": metric, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": f"{desc}; leaf {LEAF}, eta {ETA}, eps_trunc {eps} ({args.trunc} rule), "
                                   f"eps_H2 {EPS_H2}; A: 1/(4 pi r), B: 1/r^2",
                       "precision": args.precision, "autotune": at,
                       "inputs": "A, B, C together exceed L2 (no flush needed)", "parallelism": "replicas"},
            "mmp_s": ms * 1e-3, "rel_err_vs_exact_h2_matvecs": rel_err,
            "ranks_C_max_row": ranks_C, "cap_hits": cap_hits,
            "bytes_alg": nbytes, "build_s": build_s, "first_product_s_incl_plan": setup_s,
            "plan_s": max(0.0, setup_s - ms * 1e-3),
            "phase_ms": tr["phase_ms"], "phase_ms_by_name": tr["by_phase"],
            "ms_by_level": tr["by_level"], "eig_ms_by_level": tr["eig_by_level"],
            "roofline": roof, "cpu_baseline": cpu_line, "e2e": e2e, "e2e_new_structure": e2e_cold,
            "gpu_launches": int(n_launch), "clocks": clk.summary(),
        }
        line.update(extras)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
