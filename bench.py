#!/usr/bin/env python3
"""Time-to-solution benchmark of the APLICUR hot path on one or more GB300s.

One step = one complete solve of the workload through the C ABI: the one-time sketch
S A, the CUR rank steps, the preconditioner builds and the warm-started
preconditioned LSQR phases, until the relative normal-equation residual
||A^T(b - A x) - mu x|| / ||A^T b|| <= 1e-8 (checked in FP64).  Inputs are resident
in HBM for `value`; `e2e` copies A and b from pinned host memory and x back inside the
timed region.  Under torchrun every rank solves its own replica (no collective on the
data path: the method does not shard).  `--impl reference` times the CPU oracle.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 rel. residual; SpMV HBM GB/s %peak; batched solves/s vs plain LSQR"
TOL = 1e-8
WORKLOADS = {
    # name: (generator, precision)
    "rbf_fp32_20000x20000": ("config3", "mixed"),
    "dense_fp64_2000x200": ("config1", "fp64"),
    "sparse_csr_200000x20000": ("config2", "fp64"),
}
DEFAULT_WORKLOAD = "rbf_fp32_20000x20000"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--maxit", type=int, default=200000)
    ap.add_argument("--no-spmv", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-sketch", action="store_true",
                    help="skip the sketching-operator leg (dense workloads)")
    ap.add_argument("--only-sketch", action="store_true",
                    help="run the sketching-operator leg alone and print it (1 GPU)")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the other configurations' time-to-tol legs")
    ap.add_argument("--only-headline", action="store_true",
                    help="time the headline workload only (no e2e, plain LSQR, legs, SpMV, "
                         "batched or CPU legs): the profiling runs under profiles/")
    ap.add_argument("--npts", type=int, default=0,
                    help="RBF points of a smaller RBF case (profiling; 0: the workload)")
    ap.add_argument("--precision", default="", choices=["", "fp64", "mixed", "df32"],
                    help="override the workload's arithmetic (profiling)")
    ap.add_argument("--batched-nprob", type=int, default=64,
                    help="problems of the batched workload (512 is the full configuration; a "
                         "full solve takes minutes, so the default line carries 64)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def aggregate(ms_local, steps, world, device=None):
    """Max over ranks of the timed region (ms) and the whole-job throughput: every rank
    solved `steps` replicas, so value = world * steps / max_ms."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * steps / (ms_max / 1000.0)


def make_workload(name, npts=0, precision=""):
    from paper_2604_05065_gb300 import workloads as wl
    gen, prec = WORKLOADS[name]
    if npts and gen == "config3":
        p = wl.rbf_kernel(npts=npts, sketch_dim=max(5, 250 * npts // 20000))
    else:
        p = getattr(wl, gen)()
    return p, precision or prec


# ----------------------------------------------------------------------------- clocks ---

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        with open(self.tmp.name) as f:
            lines = [l.strip() for l in f if l.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm --

def gpu_arm(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2604_05065_gb300 as pkg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if args.only_headline:
        args.no_plain = args.no_legs = args.no_spmv = args.no_batched = args.no_sketch = True
        args.no_cpu_baseline = True
    p, prec = make_workload(args.workload, args.npts, args.precision)
    precision = {"mixed": pkg.PREC_MIXED, "df32": pkg.PREC_DF32}.get(prec, pkg.PREC_FP64)
    if p.fmt == "dense":
        A_host = torch.from_numpy(p.dense).pin_memory()
        A = A_host.to(dev, non_blocking=True)
    else:
        crow = torch.from_numpy(p.indptr.astype(np.int64))
        col = torch.from_numpy(p.indices.astype(np.int64))
        val = torch.from_numpy(p.data)
        A_host = None
        A = torch.sparse_csr_tensor(crow, col, val, size=(p.m, p.n)).to(dev)
    b_host = torch.from_numpy(np.asarray(p.b, dtype=np.float64)).pin_memory()
    b = b_host.to(dev, non_blocking=True)
    torch.cuda.synchronize()
    opts = dict(precision=precision, profile=1, seed=1)
    if args.only_sketch:
        print(json.dumps({"workload": p.name, "sketch": sketch_measure(args, dev, A, b, p,
                                                                        precision)}))
        return None

    nfam = len(pkg.PROFILE_FAMILIES)
    prof_tot = {"ms": [0.0] * nfam, "launches": [0] * nfam, "work": [0.0] * nfam}
    sched = {}

    def one_solve(Adev, bdev, record=False):
        s = pkg.Solver(Adev, bdev, p.mu, p.sketch_dim, **opts)
        x = s.solve(TOL, args.maxit)
        st = s.stats()
        if record:
            pr = s.profile()
            for k in range(nfam):
                prof_tot["ms"][k] += pr["ms"][k]
                prof_tot["launches"][k] += pr["launches"][k]
                prof_tot["work"][k] += pr["work"][k]
            sched.update(steps=st["nsteps"], phases=st["nphases"], iters=st["iters"],
                         ell=st["ell"], builds=sum(1 for q in s.steps() if q["rebuild"]),
                         ne_res=st["ne_res"], converged=st["converged"],
                         ms_rank=round(st["time_rank_ms"], 1), ms_build=round(st["time_build_ms"], 1),
                         ms_lsqr=round(st["time_lsqr_ms"], 1), ms_setup=round(st["time_setup_ms"], 2),
                         phase_log=s.phases())
        s.close()
        return x, st

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        one_solve(A, b)
    torch.cuda.synchronize()
    launches0 = pkg.launch_count()
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        x, st = one_solve(A, b, record=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = pkg.launch_count() - launches0
    ms_max, value = aggregate(e0.elapsed_time(e1), args.steps, world, dev)

    # ---- end to end from pinned host buffers
    e2e = None
    if A_host is not None and not args.only_headline:
        Ae = torch.empty_like(A)
        be = torch.empty_like(b)
        for _ in range(1):
            Ae.copy_(A_host, non_blocking=True)
            be.copy_(b_host, non_blocking=True)
            xh = one_solve(Ae, be)[0].cpu()
        torch.cuda.synchronize()
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        # per step: the copies and the whole step (the region's own timing is f0 .. f1)
        marks = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
                  torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        f0.record(stream)
        for k in range(args.steps):
            marks[k][0].record(stream)
            Ae.copy_(A_host, non_blocking=True)
            be.copy_(b_host, non_blocking=True)
            marks[k][1].record(stream)
            xh = one_solve(Ae, be)[0].to("cpu")
            marks[k][2].record(stream)
        f1.record(stream)
        torch.cuda.synchronize()
        _, e2e_value = aggregate(f0.elapsed_time(f1), args.steps, world, dev)
        e2e = {"value": e2e_value, "unit": "solves/s",
               "h2d_bytes_per_step": int(A_host.numel() * A_host.element_size() + b_host.numel() * 8),
               "d2h_bytes_per_step": int(p.n * 8),
               "steps_ms": [round(a.elapsed_time(c), 1) for a, _, c in marks],
               "copy_ms": [round(a.elapsed_time(b_), 2) for a, b_, _ in marks]}
        del Ae, be

    # ---- plain (unpreconditioned) LSQR on the same GPU, same kernels
    plain = None
    if not args.no_plain:
        s = pkg.Solver(A, b, p.mu, p.sketch_dim, **opts)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        s.plain_lsqr(TOL, args.maxit)
        g1.record(stream)
        torch.cuda.synchronize()
        pst = s.stats()
        plain = {"ms": g0.elapsed_time(g1), "iters": pst["iters"], "ne_res": pst["ne_res"],
                 "converged": bool(pst["converged"])}
        s.close()

    # ---- roofline of the dominant kernel family of the step (largest device time)
    roof = roofline(prof_tot)
    hot = hot_loop_roofline(prof_tot)
    sketch = None if (args.no_sketch or p.fmt != "dense") else sketch_measure(
        args, dev, A, b, p, precision)
    legs = None if (args.no_legs or world > 1) else legs_measure(args, dev)
    spmv = None if args.no_spmv else spmv_measure(args, dev)
    batched = None if (args.no_batched or world > 1) else batched_measure(args, dev)
    return dict(value=value, ms=ms_max / args.steps, p=p, prec=prec, clocks=clk, e2e=e2e,
                batched=batched, hot=hot, legs=legs, sketch=sketch,
                plain=plain, roof=roof, launches=launches, sched=sched, ne=st["ne_res"],
                spmv=spmv)


def _timed(stream, fn):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0, out


def legs_measure(args, dev):
    """Time-to-1e-8 of the other configurations, APLICUR beside plain (unpreconditioned)
    GPU LSQR with the same kernels, one warm-up and one timed solve each:
      dense FP64 2000 x 200 (mu 1e-4, sketch 20): APLICUR and plain, FP64;
      sparse CSR 200000 x 20000 (mu 1e-6, sketch 100): APLICUR with the SVD-free
        preconditioner on a CUR of [A; sqrt(mu) I] (one solve), plain LSQR in FP64 and
        FP32 products;
      adjoint FP32 100000 x 2000 (mu 1e-4, sketch 100): forward and backward of
        0.5 ||x - x_target||^2, APLICUR and plain, compensated FP32 products."""
    import numpy as np
    import torch

    import paper_2604_05065_gb300 as pkg
    from paper_2604_05065_gb300 import workloads as wl
    stream = torch.cuda.current_stream(dev)
    legs = {}

    def solve_pair(A, b, mu, sd, precision, backward=None):
        out = {}
        for kind in ("aplicur", "plain"):
            for rep in range(2):
                s = pkg.Solver(A, b, mu, sd, precision=precision, seed=1)
                fn = (lambda s=s: s.solve(TOL, args.maxit)) if kind == "aplicur" else \
                    (lambda s=s: s.plain_lsqr(TOL, args.maxit))
                if backward is None:
                    secs, _ = _timed(stream, fn)
                else:
                    def fb(s=s, fn=fn):
                        x = fn()
                        return s.backward(x - backward, TOL, args.maxit, want_A=True)
                    secs, _ = _timed(stream, fb)
                st = s.stats()
                s.close()
            out[kind] = {"time_to_tol_s": round(secs, 5), "iters": st["iters"],
                         "ne_res": st["ne_res"], "converged": bool(st["converged"]),
                         "ell": st["ell"], "nphases": st["nphases"]}
        out["aplicur_over_plain_time"] = round(out["aplicur"]["time_to_tol_s"]
                                               / out["plain"]["time_to_tol_s"], 3)
        return out

    p = wl.config1()
    A = torch.from_numpy(p.dense).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    legs[p.name] = dict(precision="fp64", **solve_pair(A, b, p.mu, p.sketch_dim, pkg.PREC_FP64))
    del A, b
    p = wl.config2()
    A = torch.sparse_csr_tensor(torch.from_numpy(p.indptr.astype(np.int64)),
                                torch.from_numpy(p.indices.astype(np.int64)),
                                torch.from_numpy(p.data), size=(p.m, p.n)).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    leg = {}
    # APLICUR with the SVD-free preconditioner on a CUR of A_mu (one solve: the CUR rank
    # grows to about n, tens of seconds of dense factor products)
    s = pkg.Solver(A, b, p.mu, p.sketch_dim, precision=pkg.PREC_FP64, seed=1, variant=1)
    secs, _ = _timed(stream, lambda s=s: s.solve(TOL, args.maxit))
    st = s.stats()
    s.close()
    leg["aplicur_svdfree_fp64"] = {
        "time_to_tol_s": round(secs, 3), "iters": st["iters"], "ne_res": st["ne_res"],
        "converged": bool(st["converged"]), "ell": st["ell"], "nsteps": st["nsteps"],
        "ms_rank": round(st["time_rank_ms"]), "ms_build": round(st["time_build_ms"]),
        "ms_lsqr": round(st["time_lsqr_ms"]),
        "note": "variant 1 with mu > 0: CUR of [A; sqrt(mu) I]; one solve, no warm-up"}
    torch.cuda.empty_cache()
    for pname, prec in (("fp64", pkg.PREC_FP64), ("mixed", pkg.PREC_MIXED)):
        for rep in range(2):
            s = pkg.Solver(A, b, p.mu, p.sketch_dim, precision=prec, seed=1)
            secs, _ = _timed(stream, lambda s=s: s.plain_lsqr(TOL, args.maxit))
            st = s.stats()
            s.close()
        leg[f"plain_{pname}"] = {"time_to_tol_s": round(secs, 4), "iters": st["iters"],
                                 "ne_res": st["ne_res"], "converged": bool(st["converged"])}
    leg["aplicur_over_plain_time"] = round(leg["aplicur_svdfree_fp64"]["time_to_tol_s"]
                                           / leg["plain_fp64"]["time_to_tol_s"], 2)
    legs[p.name] = leg
    del A, b
    A, b, xt, mu, sd = wl.config5_device(dev)
    leg = solve_pair(A, b, mu, sd, pkg.PREC_DF32, backward=xt)
    leg.update(precision="df32", mode="forward + backward (gradients in b, mu and A)",
               note="inputs drawn on the GPU by the same recipe (workloads.config5_device)")
    legs["adjoint_fp32_100000x2000"] = leg
    del A, b
    torch.cuda.empty_cache()
    return legs


def sketch_measure(args, dev, A, b, p, precision):
    """The one-time sketch Y = S A of the headline workload (dense FP32 A, s = 1.1 sketch
    dim) with each operator: the sparse sign embedding (xi = 8, FP64 sums), the Gaussian
    embedding as a compensated-FP32 product, and the Gaussian embedding on the tensor
    cores with A in 1, 2 and 3 bfloat16 terms.  Device time of the product (the library's
    events around it in aplicur_create; the host draw of S is outside), median of three
    creations after one warm-up; the tensor-core forms also solve to the bench tolerance
    (APLICUR from that sketch, the same precision as the headline)."""
    import statistics

    import paper_2604_05065_gb300 as pkg
    m, n = p.m, p.n
    sd = p.sketch_dim
    srow = (11 * sd + 9) // 10
    va = A.element_size()
    out = {"s": srow}
    forms = [("sparse_sign", dict(sketch_kind=pkg.SKETCH_SPARSE_SIGN)),
             ("gaussian_compensated_fp32", dict(sketch_kind=pkg.SKETCH_GAUSSIAN)),
             ("gaussian_tc_1term", dict(sketch_kind=pkg.SKETCH_GAUSSIAN, sketch_tc=1)),
             ("gaussian_tc_2terms", dict(sketch_kind=pkg.SKETCH_GAUSSIAN, sketch_tc=2)),
             ("gaussian_tc_3terms", dict(sketch_kind=pkg.SKETCH_GAUSSIAN, sketch_tc=3))]
    for name, kw in forms:
        times = []
        for rep in range(4):
            s = pkg.Solver(A, b, p.mu, sd, precision=precision, seed=1, **kw)
            if rep:
                times.append(s.stats()["time_setup_ms"])
            if rep < 3:
                s.close()
        ms = statistics.median(times)
        rec = {"ms": round(ms, 3)}
        if kw.get("sketch_tc"):
            k = kw["sketch_tc"]
            # algorithmic bytes: A once, S~ once (bfloat16; re-read from L2 per column
            # tile), Y written in FP64
            byts = va * m * n + 2.0 * srow * m + 8.0 * srow * n
            rec["achieved_gbs"] = round(byts / (ms * 1e-3) / 1e9, 1)
            hbm, src = peaks()
            rec[f"hbm_frac_of_{src}"] = round(byts / (ms * 1e-3) / 1e9 / hbm, 3)
            rec["tensor_tflops"] = round(2.0 * k * srow * m * n / (ms * 1e-3) / 1e12, 1)
            secs, _ = _timed(torch_stream(dev), lambda s=s: s.solve(TOL, args.maxit))
            st = s.stats()
            rec.update(solve_s=round(secs, 4), ell=st["ell"], iters=st["iters"],
                       converged=bool(st["converged"]), rank_breakdown=st["rank_breakdown"])
        s.close()
        out[name] = rec
    return out


def torch_stream(dev):
    import torch
    return torch.cuda.current_stream(dev)


def spmv_measure(args, dev):
    """CSR A z (rows) and CSC A^T u (columns) device throughput on the sparse
    200000 x 20000 workload, timed live over a plain LSQR solve to the same tolerance."""
    import numpy as np
    import torch

    import paper_2604_05065_gb300 as pkg
    from paper_2604_05065_gb300 import workloads as wl
    p = wl.config2()
    A = torch.sparse_csr_tensor(torch.from_numpy(p.indptr.astype(np.int64)),
                                torch.from_numpy(p.indices.astype(np.int64)),
                                torch.from_numpy(p.data), size=(p.m, p.n)).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    s = pkg.Solver(A, b, p.mu, p.sketch_dim, profile=1, seed=1)
    s.plain_lsqr(TOL, args.maxit)          # warm-up
    s.reset_profile()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.plain_lsqr(TOL, args.maxit)
    e1.record(stream)
    torch.cuda.synchronize()
    st = s.stats()
    pr = s.profile()
    peak, _ = peaks()
    out = {"workload": p.name, "nnz": p.nnz, "dtype": "f64",
           "plain_lsqr_time_to_tol_s": e0.elapsed_time(e1) / 1000.0, "iters": st["iters"],
           "ne_res": st["ne_res"]}
    for k, nm in ((0, "spmv_csr_Az"), (1, "spmvT_csc_ATu")):
        if pr["launches"][k]:
            gbs = pr["work"][k] / (pr["ms"][k] * 1e-3) / 1e9
            out[nm] = {"GBps": round(gbs, 1), "frac_of_hbm_peak": round(gbs / peak, 4),
                       "avg_launch_us": round(1000 * pr["ms"][k] / pr["launches"][k], 2),
                       "bytes_per_launch": int(pr["work"][k] / pr["launches"][k]),
                       "note": "working set (CSR+CSC 6.4 MB, vectors ~5 MB) is L2-resident"}
    s.close()
    return out


FP64_PEAK_TFLOPS = 1.25  # GB300 nominal FP64: 152 SMs x 2.07 GHz x 4 FLOP/clk/SM
FP32_PEAK_TFLOPS = 80.5  # GB300 nominal FP32 SIMT: 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz
# Compensated FP32 (the default dense arithmetic): FP64-equivalent flops issued as about 6
# FP32 instructions each (a product needs a rounding-error FMA, two cross terms and a
# TwoSum), so its ceiling is the FP32 instruction rate / 6.
DF32_PEAK_TFLOPS = round(152 * 128 * 2.07e9 / 6 / 1e12, 2)
NAMES = ["A pass (fused_apass_kernel; k1_dense in the two-pass form)",
         "A^T u column sums (k2b_dense; k2a_dense + k2b_dense in the two-pass form)",
         "preconditioner passes (pre_qt, pre_qsum, pre_vt, pre_v, pre_expand)",
         "dense GEMM (df32gemm_kernel, compensated FP32)",
         "Jacobi stage 2 (jacobi_df_block_kernel, compensated FP32)",
         "LUPP selection (lupp_coop_kernel; lupp_step_kernel in batched builds)",
         "Jacobi stage 1 (jacobi32_block_kernel, FP32)"]
ALU = {3: (DF32_PEAK_TFLOPS, "derived compensated-FP32 ceiling: 152 SMs x 128 lanes x 2.07 GHz "
                             "FP32 instructions / 6 per FP64-equivalent flop"),
       4: (DF32_PEAK_TFLOPS, "derived compensated-FP32 ceiling: 152 SMs x 128 lanes x 2.07 GHz "
                             "FP32 instructions / 6 per FP64-equivalent flop"),
       6: (FP32_PEAK_TFLOPS, "nominal GB300 FP32 (152 SMs x 128 lanes x 2 FLOP x 2.07 GHz)")}


def batched_measure(args, dev):
    """The batched workload (uneven dense and CSR FP32 problems, 16 right-hand sides each,
    mu 1e-5, sketch dimension 50): one warm-up and one timed APLICUR batch solve to the
    time-to-tol target, one timed solve followed by its adjoint (gradients in b, mu and A
    of every pair), then the same batch by plain LSQR with the same grouped kernels.
    Throughput counts solved (problem, right-hand side) pairs per second."""
    import torch

    import paper_2604_05065_gb300 as pkg
    from paper_2604_05065_gb300 import workloads as wl

    nprob, R = args.batched_nprob, 16
    t0 = time.perf_counter()
    mats, rhs, sizes = wl.batched_device(dev, nprob=nprob, nrhs=R)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    abytes = sum(4 * m * n for (m, n, f) in sizes if f == "dense")
    abytes += sum(8 * a.values().numel() for a, (m, n, f) in zip(mats, sizes) if f == "csr")
    t0 = time.perf_counter()
    s = pkg.BatchSolver(mats, rhs, 1e-5, 50, seed=1)
    create_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    out = {"workload": f"batched_{nprob}x{R}", "problems": nprob, "nrhs": R,
           "note": ("the full 512-problem configuration" if nprob == 512 else
                    f"{nprob} problems drawn by the 512-problem recipe (--batched-nprob 512 "
                    "runs the full configuration)"),
           "pairs": nprob * R, "a_bytes": int(abytes), "generate_s": round(gen_s, 2),
           "create_s": round(create_s, 2)}

    def timed(fn, warm=True):
        if warm:
            fn(TOL, args.maxit)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn(TOL, args.maxit)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0

    secs = timed(s.solve)
    st = s.stats()
    out["breakdowns"] = sum(1 for q in range(nprob) if s.problem(q)["breakdown"])
    out.update(solve_s=round(secs, 3), solves_per_s=round(nprob * R / secs, 2),
               converged=st["converged"], ne_max=st["ne_max"], iters_max=st["iters_max"],
               iters_sum=st["iters_sum"], ms_rank=round(st["time_rank_ms"], 1),
               ms_build=round(st["time_build_ms"], 1), ms_lsqr=round(st["time_lsqr_ms"], 1),
               tuned={"rows_per_warp": st["rows_per_warp"], "cols_per_lane": st["cols_per_lane"]},
               launches_per_iter=st["launches_per_iter"])
    # with adjoint: the solve and the backward of 0.5 sum ||x - t||^2 (t = 0: dL/dx = x),
    # dL/db, dL/dmu and dL/dA for every pair
    xs = s.solve(TOL, args.maxit)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    xs = s.solve(TOL, args.maxit)
    s.backward(xs, TOL, args.maxit, want_A=True)
    e1.record(stream)
    torch.cuda.synchronize()
    asecs = e0.elapsed_time(e1) / 1000.0
    ast = s.stats()
    out["with_adjoint"] = {"solve_and_backward_s": round(asecs, 3),
                           "solves_per_s": round(nprob * R / asecs, 2),
                           "backward_converged": ast["converged"], "backward_ne_max": ast["ne_max"],
                           "backward_iters_max": ast["iters_max"]}
    del xs
    if not args.no_plain:
        psecs = timed(s.plain_lsqr, warm=False)  # kernels already warm from the solves
        pst = s.stats()
        out["plain_lsqr"] = {"solve_s": round(psecs, 3), "solves_per_s": round(nprob * R / psecs, 2),
                             "converged": pst["converged"], "ne_max": pst["ne_max"],
                             "iters_max": pst["iters_max"]}
        out["speedup_vs_plain"] = round(psecs / secs, 3)
    s.close()
    return out


def roofline(prof):
    nf = len(prof["ms"])
    k = max(range(nf), key=lambda q: prof["ms"][q])
    if not prof["launches"][k]:
        return None
    peak_bw, src = peaks()
    fams = {}
    for q in range(nf):
        if not prof["launches"][q]:
            continue
        rate = prof["work"][q] / max(prof["ms"][q], 1e-12) * 1e3  # work per second
        if q in ALU:
            fams[NAMES[q]] = {"ms_total": round(prof["ms"][q], 2), "timed": prof["launches"][q],
                              "TFLOPs": round(rate * 1e-12, 4),
                              "frac": round(rate * 1e-12 / ALU[q][0], 4)}
        else:
            fams[NAMES[q]] = {"ms_total": round(prof["ms"][q], 2), "timed": prof["launches"][q],
                              "GBps": round(rate * 1e-9, 1), "frac": round(rate * 1e-9 / peak_bw, 4)}
    avg_ms = prof["ms"][k] / prof["launches"][k]
    per = prof["work"][k] / prof["launches"][k]
    if k in ALU:
        achieved = per / (avg_ms * 1e-3) / 1e12
        out = {"bound": "alu", "achieved": round(achieved, 4), "peak": ALU[k][0],
               "unit": "TFLOP/s", "frac": round(achieved / ALU[k][0], 4),
               "traffic": traffic_for(k, per), "peak_source": ALU[k][1],
               "flops_per_launch": int(per)}
    else:
        achieved = per / (avg_ms * 1e-3) / 1e9
        out = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak_bw, "unit": "GB/s",
               "frac": round(achieved / peak_bw, 4), "traffic": traffic_for(k, per),
               "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured"
               else "fallback 6800 GB/s", "bytes_per_launch": int(per)}
    out.update(kernel=NAMES[k], avg_launch_ms=round(avg_ms, 5), launches_timed=prof["launches"][k],
               families=fams)
    return out


def hot_loop_roofline(prof):
    """The dense A pass of the LSQR iterations (family 0: the fused single-read pass with
    FP32 products, or A z of the two-pass form) against the measured HBM copy bandwidth."""
    if not prof["launches"][0]:
        return None
    peak_bw, src = peaks()
    avg_ms = prof["ms"][0] / prof["launches"][0]
    per = prof["work"][0] / prof["launches"][0]
    achieved = per / (avg_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "A pass of the LSQR iteration (fused_apass_kernel)",
            "achieved": round(achieved, 1), "peak": peak_bw, "unit": "GB/s",
            "frac": round(achieved / peak_bw, 4), "bytes_per_launch": int(per),
            "avg_launch_ms": round(avg_ms, 5), "launches_timed": prof["launches"][0],
            "traffic": traffic_for(0, per),
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured"
            else "fallback 6800 GB/s"}


def traffic_for(k, bpl):
    """DRAM bytes per launch from the committed ncu summary table (profiles/ncu_traffic.md),
    scaled to this launch size, or None when no capture of the current kernel source exists."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.md")
    try:
        for line in open(path):
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) < 4 or cells[0] != str(k):
                continue
            src = open(os.path.join(ROOT, cells[1]), "rb").read()
            if hashlib.sha256(src).hexdigest() != cells[2]:
                return None
            return int(float(cells[3]) * bpl)
    except (OSError, ValueError):
        return None
    return None


# ----------------------------------------------------------------------------- CPU arm --

class OracleReplay:
    """The oracle's solve of a workload cut into strata in the order the driver of
    Algorithm "APLICUR: detailed implementation" runs them: the sketch, every rank step
    (Parts 1 and 2), every preconditioner build and, per LSQR phase, a sample of
    SAMPLE_ITERS iterations plus the residual check.  The schedule (rebuild flags, phase
    lengths) is the oracle's own full run (tests/golden, written by make_schedules.py); the
    strata call the oracle's functions as they stand, on the full workload.  A phase is
    scaled by its length: the phase start and the residual check each cost about one
    iteration (one product with A and one with A^T), so a phase of k iterations costs
    (k + 2) / (SAMPLE_ITERS + 2) of its sample."""

    SAMPLE_ITERS = 3

    def __init__(self, p, gold):
        import numpy as np
        self.np = np
        self.p = p
        self.A = p.to_scipy() if p.fmt == "csr" else np.asarray(p.dense, dtype=np.float64)
        self.b = np.asarray(p.b, dtype=np.float64)
        self.mu = p.mu
        self.delta = math.sqrt(p.mu)
        self.rebuild = [bool(st["rebuild"]) for st in gold["rank_steps"]]
        self.phase_iters = list(gold["bench_tol"]["phases"])
        self.strata = []            # (name, fn, scale)
        ph = 0
        self.strata.append(("sketch", self._sketch, 1.0))
        for k, rb in enumerate(self.rebuild):
            self.strata.append((f"rank step {k + 1}", self._rank_step, 1.0))
            if rb:
                self.strata.append((f"build {ph + 1}", self._build, 1.0))
                it = self.phase_iters[ph] if ph < len(self.phase_iters) else 0
                self.strata.append((f"phase {ph + 1} ({it} iterations)", self._phase,
                                    (it + 2) / (self.SAMPLE_ITERS + 2)))
                ph += 1
        self.times = {}
        self.pos = 0

    # ---- the driver's pieces, on the oracle's functions
    def _sketch(self):
        from oracle import aplicur_oracle as O
        from oracle import rng as orng
        s = O.sketch_rows(self.p.sketch_dim)
        rows, signs = orng.sparse_sign(1, s, self.p.m, O.sketch_xi(s))
        self.W = orng.gaussian_w(1, self.p.n, 10)
        self.Y = O.apply_sketch(self.A, rows, signs, s)
        e = self.np.zeros(0, self.np.int64)
        self.I, self.J, self.core, self.E = e, e, None, self.Y.copy()
        self.Q = self.T = None
        self.x = self.np.zeros(self.p.n)
        self.norm_Atb = float(self.np.linalg.norm(O.rmatvec(self.A, self.b)))

    def _rank_step(self):
        from oracle import aplicur_oracle as O
        np = self.np
        kb = min(self.p.sketch_dim, min(self.p.m, self.p.n) - len(self.J))
        Ip, Jp, _ = O.augment_cur(self.A, self.I, self.J, self.E, self.core, kb)
        self.I = np.concatenate([self.I, Ip])
        self.J = np.concatenate([self.J, Jp])
        self.core = O.Core(self.A, self.I, self.J)
        self.E = O.sketched_residual(self.A, self.Y, self.I, self.J, self.core)
        O.norm_estimate(self.E, self.W)
        if Ip.size:
            self.Q, self.T = O.augment_qr(self.Q, self.T, O.rows(self.A, Ip).T)

    def _build(self):
        from oracle import aplicur_oracle as O
        self.P = O.build_preconditioner(O.cols(self.A, self.J), self.core, self.Q, self.T,
                                        self.delta)

    def _phase(self):
        from oracle import aplicur_oracle as O
        r = O.plsqr_phase(self.A, self.b, self.delta, self.x, self.P, eps_lsqr=0.0,
                          fixed_len=self.SAMPLE_ITERS)
        self.x = r.x
        O.ne_residual(self.A, self.b, self.mu, self.x, self.norm_Atb)

    def run_next(self):
        """Run the next stratum (after the last one, a new solve starts with the sketch);
        returns its wall time in seconds."""
        name, fn, _ = self.strata[self.pos]
        t0 = time.perf_counter()
        fn()
        dt = time.perf_counter() - t0
        self.times.setdefault(name, []).append(dt)
        self.pos = (self.pos + 1) % len(self.strata)
        return dt

    def covered(self):
        return all(name in self.times for name, _, _ in self.strata)

    def solve_seconds(self):
        """One full solve, from the strata measured (their means)."""
        return sum(statistics.mean(self.times[name]) * sc for name, _, sc in self.strata)

    def describe(self):
        parts = ", ".join(f"{name} {statistics.mean(self.times[name]) * sc:.2f} s"
                          for name, _, sc in self.strata)
        return (f"oracle solve of the full workload cut into {len(self.strata)} strata in "
                f"driver order on the oracle's own schedule (rank steps and builds at every "
                f"rank of the schedule, phases from {self.SAMPLE_ITERS}-iteration samples "
                f"scaled by their lengths): {parts}")


def cpu_info():
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith("model name") or low.startswith("cpu part"):
                model = line.split(":", 1)[1].strip()
                if low.startswith("model name"):
                    break
    except OSError:
        pass
    try:
        import platform
        model = model or platform.processor()
        arch = platform.machine()
    except Exception:
        arch = ""
    threads = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS")
    return {"cpu": model, "arch": arch, "cores": os.cpu_count(),
            "blas_threads": int(threads) if threads else os.cpu_count()}


def oracle_baseline(p, gold):
    """The oracle timed once through every stratum of a solve (CPU baseline of the GPU
    arm's line)."""
    rep = OracleReplay(p, gold)
    t0 = time.perf_counter()
    while not rep.covered():
        rep.run_next()
    wall = time.perf_counter() - t0
    secs = rep.solve_seconds()
    return 1.0 / secs, rep.describe(), wall


def make_config(p, prec, world):
    return {"workload": p.name, "m": p.m, "n": p.n, "mu": p.mu, "sketch_dim": p.sketch_dim,
            "tol": TOL,
            "precision": {"mixed": "fp32 products and sums, fp64 scalars/core/refinement",
                          "df32": "fp32 storage, compensated fp32 products and sums (hi/lo "
                                  "split), fp64 scalars/core/preconditioner"}.get(prec, "fp64"),
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2" if p.nnz * p.dtype.itemsize > 129e6
            else "L2-resident inputs (no flush)"}


def load_schedule(name):
    path = os.path.join(ROOT, "tests", "golden", f"schedule_{name}.json")
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return None


def reference_arm(args, rank, world):
    """The oracle as the reference arm: the K timed steps run the strata of OracleReplay
    in driver order (spread over the steps when K is smaller than the number of strata,
    one per step and cycling otherwise); the value is one full solve assembled from the
    strata.  Warm-up steps do no oracle work (nothing in it warms up)."""
    if rank != 0:
        return
    p, prec = make_workload(args.workload)
    gold = load_schedule(args.workload)
    if gold is None or "bench_tol" not in gold:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"no oracle schedule for {args.workload} under tests/golden"}))
        return
    rep = OracleReplay(p, gold)
    nstr = len(rep.strata)
    if args.steps >= nstr:
        per_step = [1] * args.steps
    else:
        per_step = [nstr // args.steps + (1 if k < nstr % args.steps else 0)
                    for k in range(args.steps)]
    step_s = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step[k]):
            rep.run_next()
        step_s.append(time.perf_counter() - t0)
    value = 1.0 / rep.solve_seconds()
    info = cpu_info()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(step_s), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": make_config(p, prec, world),
            "time_to_tol_s": 1.0 / value,
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": info["blas_threads"],
                             "kind": "oracle", "cpu": info["cpu"], "arch": info["arch"],
                             "sample": rep.describe()
                             + f"; each timed step ran {per_step[0]} stratum(s)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- main -----

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    r = gpu_arm(args, rank, world, local_rank)
    if r is None:
        return
    if rank == 0:
        p = r["p"]
        cpu = None
        gold = load_schedule(args.workload)
        if world == 1 and not args.no_cpu_baseline and gold and "bench_tol" in gold:
            v, sample, secs = oracle_baseline(p, gold)
            info = cpu_info()
            cpu = {"value": v, "unit": "solves/s", "cores": info["blas_threads"],
                   "kind": "oracle", "cpu": info["cpu"], "arch": info["arch"],
                   "sample": sample, "sample_seconds": round(secs, 2),
                   "oracle_full_run_seconds_on_build_host": gold["bench_tol"]["oracle_seconds"]}
        line = {"metric": METRIC, "value": r["value"], "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if r["prec"] in ("mixed", "df32") else "f64", "data": "synthetic",
                "config": make_config(p, r["prec"], world),
                "time_to_tol_s": r["ms"] / 1000.0, "schedule": r["sched"],
                "ne_res": r["ne"], "plain_lsqr": r["plain"], "clocks": r["clocks"],
                "e2e": r["e2e"], "gpu_launches": r["launches"], "roofline": r["roof"],
                "roofline_hot_loop": r["hot"], "legs": r["legs"], "sketch": r["sketch"],
                "spmv": r["spmv"], "batched": r["batched"],
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
