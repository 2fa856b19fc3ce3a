"""The single-shot schedules (options.schedule = 1) against the oracle: the rank grows as
in the oracle's single-shot run, the preconditioner is built once at the last rank step,
and the solve reaches the ridge solution; with max_rank = sketch_dim the one rank step is
the fixed-rank single-shot variant."""
import numpy as np
import pytest

from oracle import aplicur_oracle as O
from paper_2604_05065_gb300 import workloads as wl

from gpu_helpers import draws, oracle_matrix, rel, to_device

pytestmark = pytest.mark.gpu


def _solve(p, seed_draws=5, **kw):
    import paper_2604_05065_gb300 as pkg
    rows, signs, W = draws(p, seed=seed_draws)
    A, b = to_device(p)
    s = pkg.Solver(A, b, p.mu, p.sketch_dim, sketch_rows=rows, sketch_signs=signs,
                   normest_w=W, schedule=1, **kw)
    x = s.solve(1e-10).cpu().numpy()
    return s, x, (rows, signs, W)


@pytest.mark.parametrize("fixed", [False, True])
def test_single_shot_schedules_match_oracle(fixed):
    p = wl.config1(scale=4)
    kw = {"max_rank": p.sketch_dim} if fixed else {}
    s, x, (rows, signs, W) = _solve(p, **kw)
    A = oracle_matrix(p)
    ref = O.aplicur(A, p.b, p.mu, p.sketch_dim,
                    O.Options(single_shot=True, max_rank=kw.get("max_rank", 0)), tol=1e-10,
                    srows=rows, signs=signs, W=W)
    I, J = s.indices()
    assert np.array_equal(I, ref.I) and np.array_equal(J, ref.J)
    flags = [st["rebuild"] for st in s.steps()]
    assert flags == [st["rebuild"] for st in ref.rank_steps]
    assert flags[-1] and not any(flags[:-1])
    st = s.stats()
    assert st["converged"] and st["ne_res"] <= 1e-10
    # the same bound as the adaptive free-run test: ne_res <= 1e-10 with kappa ~ 1/delta
    assert rel(x, O.ridge_direct(A, p.b, p.mu)) <= max(1e-10, 10 * 1e-10 / np.sqrt(p.mu))
    s.close()
