"""Run APLICUR solves of one synthetic workload for profiling (ncu launch lists and
single-kernel captures).  Prints one JSON line with the solve statistics.

  python -m paper_2604_05065_gb300.profile_run --workload rbf --npts 20000 --solves 1
  python -m paper_2604_05065_gb300.profile_run --workload rbf --npts 8000 --plain
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    import numpy as np
    import torch

    import paper_2604_05065_gb300 as pkg
    from paper_2604_05065_gb300 import workloads as wl

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="rbf", choices=["rbf", "dense", "sparse"])
    ap.add_argument("--npts", type=int, default=20000, help="RBF points (rbf workload)")
    ap.add_argument("--scale", type=int, default=1, help="shrink factor (dense, sparse)")
    ap.add_argument("--solves", type=int, default=1)
    ap.add_argument("--plain", action="store_true", help="unpreconditioned LSQR only")
    ap.add_argument("--precision", default="df32", choices=["fp64", "mixed", "df32"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=20000)
    args = ap.parse_args()

    if args.workload == "rbf":
        p = wl.rbf_kernel(npts=args.npts, sketch_dim=250 if args.npts >= 20000 else
                          max(5, 250 * args.npts // 20000))
    elif args.workload == "dense":
        p = wl.config1(args.scale)
    else:
        p = wl.config2(args.scale)
    dev = torch.device("cuda:0")
    if p.fmt == "dense":
        A = torch.from_numpy(p.dense).to(dev)
    else:
        A = torch.sparse_csr_tensor(torch.from_numpy(p.indptr.astype(np.int64)),
                                    torch.from_numpy(p.indices.astype(np.int64)),
                                    torch.from_numpy(p.data), size=(p.m, p.n)).to(dev)
    b = torch.from_numpy(np.asarray(p.b, dtype=np.float64)).to(dev)
    prec = {"fp64": pkg.PREC_FP64, "mixed": pkg.PREC_MIXED, "df32": pkg.PREC_DF32}[args.precision]
    out = []
    for _ in range(args.solves):
        t0 = time.perf_counter()
        s = pkg.Solver(A, b, p.mu, p.sketch_dim, precision=prec, seed=1)
        x = s.plain_lsqr(args.tol, args.maxit) if args.plain else s.solve(args.tol, args.maxit)
        torch.cuda.synchronize()
        st = s.stats()
        st["wall_ms"] = (time.perf_counter() - t0) * 1e3
        st["phases_log"] = s.phases()
        out.append(st)
        s.close()
    print(json.dumps({"workload": p.name, "solves": out}))


if __name__ == "__main__":
    main()
