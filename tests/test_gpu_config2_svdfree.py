"""The sparse 200000 x 20000 workload (10 nonzeros per column, column j scaled by
10^(-6 j / 19999), mu = 1e-6, sketch dimension 100) end to end with the SVD-free
preconditioner on a CUR of A_mu = [A; 1e-3 I]: FP64 values with FP64 products, and FP32
values with the mixed form.  Reference: the oracle's ridge solution of the same (rounded)
matrix by conjugate gradients on the normal equations to a residual of 1e-15.  The CUR
rank grows to about n here (the residual estimate on A_mu carries the unselected delta
rows), so the final preconditioner is nearly exact and the solve ends far below its
tolerance; the gate is 1e-6 relative (FP64) and 1e-5 (FP32 storage)."""
import numpy as np
import pytest

from oracle import aplicur_oracle as O
from paper_2604_05065_gb300 import workloads as wl

from gpu_helpers import rel, to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_config2_svdfree_end_to_end(form):
    import torch

    import paper_2604_05065_gb300 as pkg
    p = wl.config2(dtype=np.float64 if form == "fp64" else np.float32)
    xo, res = O.ridge_sparse(p.to_scipy(), p.b, p.mu)
    assert res <= 1e-14
    A, b = to_device(p)
    prec = pkg.PREC_FP64 if form == "fp64" else pkg.PREC_MIXED
    s = pkg.Solver(A, b, p.mu, p.sketch_dim, seed=1, variant=1, precision=prec)
    x = s.solve(1e-10, 200000).cpu().numpy()
    st = s.stats()
    assert st["converged"] == 1 and st["ne_res"] <= 1e-10
    err = rel(x, xo)
    print(f"config 2 SVD-free {form}: rank {st['ell']}, {st['nsteps']} rank steps, "
          f"{st['iters']} iterations, ne_res {st['ne_res']:.1e}, error vs oracle {err:.1e}, "
          f"rank steps {st['time_rank_ms'] / 1e3:.1f} s, builds {st['time_build_ms'] / 1e3:.1f} s",
          flush=True)
    assert err <= (1e-6 if form == "fp64" else 1e-5)
    s.close()
    del A, b
    torch.cuda.empty_cache()
