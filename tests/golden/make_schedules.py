"""Write the oracle's full-run schedule of a bench workload (rank steps, preconditioner
builds, LSQR iterations) to tests/golden/schedule_<workload>.json.

Calls only the oracle.  The schedule scales the CPU baseline's bounded sample (sketch,
one rank step, one build, a few LSQR iterations) to one full solve.

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


def main(name):
    p = GENERATORS[name]()
    A = p.to_scipy() if p.fmt == "csr" else np.asarray(p.dense, dtype=np.float64)
    t0 = time.time()
    res = O.aplicur(A, p.b, p.mu, p.sketch_dim, O.Options(seed=1), tol=1e-8, maxit=20000)
    out = {"workload": p.name, "tol": 1e-8, "seed": 1, "steps": len(res.rank_steps),
           "builds": int(sum(1 for s in res.rank_steps if s["rebuild"])), "iters": int(res.iters),
           "ell": int(len(res.I)), "converged": bool(res.converged), "ne_res": res.ne_res,
           "phases": [{k: (float(v) if isinstance(v, (float, np.floating)) else v)
                       for k, v in ph.items()} for ph in res.phases],
           "oracle_seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, f"schedule_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main(sys.argv[1])
