"""The SVD-free preconditioner (options.variant = 1, mu = 0) against the oracle.

A small dense full-rank least-squares problem with the CUR rank capped below n: the solve
reaches the least-squares solution within the rigorous bound, the target level is the
smallest CUR singular value (the oracle's power iteration and the SVD agree on it), and the
preconditioner applies like the oracle's SVD-free operator built from the same indices,
factors and target level."""
import numpy as np
import pytest

from oracle import aplicur_oracle as O
from paper_2604_05065_gb300 import workloads as wl

from gpu_helpers import draws, oracle_matrix, rel, to_device

pytestmark = pytest.mark.gpu


def _problem():
    return wl.small_dense(300, 40, 905, decay=3.0, mu=0.0, sketch_dim=4)


def _solver(p, **kw):
    import paper_2604_05065_gb300 as pkg
    rows, signs, W = draws(p)
    A, b = to_device(p)
    return pkg.Solver(A, b, 0.0, p.sketch_dim, sketch_rows=rows, sketch_signs=signs,
                      normest_w=W, variant=1, fp64_dense=1, **kw)


def test_svdfree_solve_reaches_least_squares_solution():
    p = _problem()
    s = _solver(p, max_rank=24)
    x = s.solve(1e-10).cpu().numpy()
    st = s.stats()
    assert st["converged"] and st["ne_res"] <= 1e-10 and st["ell"] == 24
    A = oracle_matrix(p)
    xd = np.linalg.lstsq(A, p.b, rcond=None)[0]
    # ||x - x*|| <= ||A^T (b - A x)|| / sigma_min^2
    smin = np.linalg.svd(A, compute_uv=False)[-1]
    bound = st["ne_res"] * np.linalg.norm(A.T @ p.b) / smin ** 2
    assert np.linalg.norm(x - xd) <= 1.01 * bound + 1e-12
    s.close()


def test_svdfree_target_level_and_apply_match_oracle():
    import torch
    p = _problem()
    s = _solver(p, max_rank=24)
    s.solve(1e-10)
    I, J = s.indices()
    _, sighat = s.preconditioner()
    A = oracle_matrix(p)
    bsz = p.sketch_dim
    Q, T = None, None
    for k in range(0, len(I), bsz):
        Q, T = O.augment_qr(Q, T, A[I[k:k + bsz], :].T)
    Pt = O.build_svdfree_preconditioner(A[:, J], A[np.ix_(I, J)], Q, T, sighat)
    assert sighat == pytest.approx(O.svdfree_smallest_sigma(Pt, iters=200), rel=1e-6)
    w = np.random.default_rng(6).standard_normal(p.n)
    out = s.apply_preconditioner(torch.from_numpy(w).cuda()).cpu().numpy()
    assert rel(out, Pt.apply_inv(w)) <= 1e-9
    s.close()


def test_svdfree_needs_mu_zero():
    import paper_2604_05065_gb300 as pkg
    p = wl.small_dense(120, 20, 906, decay=2.0, mu=1e-4, sketch_dim=4)
    A, b = to_device(p)
    with pytest.raises(pkg.AplicurError):
        pkg.Solver(A, b, p.mu, p.sketch_dim, variant=1)
