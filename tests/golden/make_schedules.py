"""Write the oracle's full run of a bench workload to tests/golden/schedule_<workload>.json:
the schedule (rank steps with their rebuild flags and rho, phases with their lengths), the
CUR indices in selection order, and the solution at 256 seeded sample indices with its
norm.

Calls only the oracle.  The full-size replay parity test runs the GPU on this schedule
and compares indices and the sampled solution; the CPU baseline reads the oracle's time.

  python tests/golden/make_schedules.py rbf_fp32_20000x20000
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import aplicur_oracle as O  # noqa: E402
from paper_2604_05065_gb300 import workloads as wl  # noqa: E402

GENERATORS = {"rbf_fp32_20000x20000": wl.config3, "dense_fp64_2000x200": wl.config1}
SAMPLE_SEED = 20260404
# converged well past the bench's 1e-8, so that the replayed GPU solution can be compared
# with the oracle's at the FP32-storage gate (the solution error scales with the residual)
TOL = 1e-12


def main(name):
    p = GENERATORS[name]()
    A = p.to_scipy() if p.fmt == "csr" else np.asarray(p.dense, dtype=np.float64)
    t0 = time.time()
    res = O.aplicur(A, p.b, p.mu, p.sketch_dim, O.Options(seed=1), tol=TOL, maxit=20000)
    out = {"workload": p.name, "tol": TOL, "seed": 1, "steps": len(res.rank_steps),
           "builds": int(sum(1 for s in res.rank_steps if s["rebuild"])), "iters": int(res.iters),
           "ell": int(len(res.I)), "converged": bool(res.converged), "ne_res": res.ne_res,
           "phases": [{k: (float(v) if isinstance(v, (float, np.floating)) else v)
                       for k, v in ph.items()} for ph in res.phases],
           "rank_steps": [{"ell": int(st["ell"]), "rho": float(st["rho"]),
                           "rebuild": bool(st["rebuild"]), "margin": float(st["margin"])}
                          for st in res.rank_steps],
           "I": [int(i) for i in res.I], "J": [int(j) for j in res.J],
           "oracle_seconds": round(time.time() - t0, 1)}
    # the same solve to the bench's tolerance: its schedule and the oracle's time, which
    # the CPU baseline's stratified sample should reproduce
    t0 = time.time()
    r8 = O.aplicur(A, p.b, p.mu, p.sketch_dim, O.Options(seed=1), tol=1e-8, maxit=20000)
    out["bench_tol"] = {"tol": 1e-8, "iters": int(r8.iters), "ne_res": float(r8.ne_res),
                        "phases": [int(ph["iters"]) for ph in r8.phases],
                        "oracle_seconds": round(time.time() - t0, 1)}
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(p.n, size=min(256, p.n),
                                                            replace=False))
    out["x_sample_index"] = [int(i) for i in idx]
    out["x_sample"] = [float(v) for v in res.x[idx]]
    out["x_norm"] = float(np.linalg.norm(res.x))
    with open(os.path.join(HERE, f"schedule_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k not in ("I", "J", "x_sample",
                                                                "x_sample_index")}))


if __name__ == "__main__":
    main(sys.argv[1])
