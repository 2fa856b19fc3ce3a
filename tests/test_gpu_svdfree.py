"""The SVD-free preconditioner (options.variant = 1) against the oracle: mu = 0 (a CUR of A)
and mu > 0 (a CUR of A_mu = [A; sqrt(mu) I]).

A small dense full-rank least-squares problem with the CUR rank capped below n: the solve
reaches the least-squares solution within the rigorous bound, the target level is the
smallest CUR singular value (the oracle's power iteration and the SVD agree on it), and the
preconditioner applies like the oracle's SVD-free operator built from the same indices,
factors and target level."""
import math

import numpy as np
import pytest

from oracle import aplicur_oracle as O
from paper_2604_05065_gb300 import workloads as wl

from gpu_helpers import draws, oracle_matrix, rel, schedule, to_device

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


# ---- mu > 0: the CUR is of A_mu = [A; sqrt(mu) I] ------------------------------------

SEED = 31
MU_PROBS = {
    "dense64": lambda: wl.small_dense(400, 60, 904, decay=6.0, mu=1e-4, sketch_dim=4),
    "sparse64": lambda: wl.small_sparse(3000, 300, wl.BASE_SEED + 50, nnz_per_col=6, mu=1e-5,
                                        sketch_dim=10),
    "dense32": lambda: wl.dense_lowrank(m=600, n=120, mu=1e-4, sketch_dim=8, index=60,
                                        dtype=np.float32, name="dense32"),
    "sparse32": lambda: wl.small_sparse(2500, 250, wl.BASE_SEED + 51, nnz_per_col=5, mu=1e-5,
                                        sketch_dim=10, dtype=np.float32),
}


def _stored_delta(p):
    """sqrt(mu) as the library stores it in A_mu's appended rows (A's value type)."""
    d = math.sqrt(p.mu)
    return float(np.float32(d)) if p.dtype == np.float32 else d


def _mu_solver(p, **kw):
    import paper_2604_05065_gb300 as pkg
    A, b = to_device(p)
    return pkg.Solver(A, b, p.mu, p.sketch_dim, seed=SEED, variant=1, **kw)


def _ridge_ok(p, x):
    A = oracle_matrix(p)
    xd = O.ridge_direct(A.toarray() if hasattr(A, "toarray") else A, p.b, p.mu)
    kappa = 1.0 / math.sqrt(p.mu)
    return rel(x, xd), max(1e-10, 10 * kappa * 1e-10)


@pytest.mark.parametrize("name", list(MU_PROBS))
def test_svdfree_mu_replay_matches_oracle(name):
    """Replaying the oracle's schedule, the CUR of A_mu selects the oracle's indices (some
    of them rows of the delta I block) and the solve reaches the ridge solution."""
    p = MU_PROBS[name]()
    A = oracle_matrix(p)
    ref = O.aplicur(A, p.b, p.mu, p.sketch_dim,
                    O.Options(seed=SEED, variant="svdfree", cur_delta=_stored_delta(p)), tol=1e-10)
    assert ref.converged and np.any(ref.I >= p.m)
    s = _mu_solver(p, replay=schedule(ref))
    x = s.solve(1e-10).cpu().numpy()
    I, J = s.indices()
    assert np.array_equal(I, ref.I) and np.array_equal(J, ref.J)
    assert [q["iters"] for q in s.phases()] == [q["iters"] for q in ref.phases]
    err, bound = _ridge_ok(p, x)
    assert err <= bound, (err, bound)
    s.close()


@pytest.mark.parametrize("name", list(MU_PROBS))
def test_svdfree_mu_free_run_converges(name):
    p = MU_PROBS[name]()
    s = _mu_solver(p)
    x = s.solve(1e-10).cpu().numpy()
    st = s.stats()
    assert st["converged"] == 1 and st["ne_res"] <= 1e-10
    err, bound = _ridge_ok(p, x)
    assert err <= bound, (err, bound)
    print(f"{name}: rank {st['ell']}, {st['iters']} iterations, error {err:.1e}", flush=True)
    s.close()


@pytest.mark.parametrize("name", ["dense64", "sparse64"])
def test_svdfree_mu_apply_matches_oracle(name):
    """P~^{-1} w and the target level against the oracle's SVD-free operator built on A_mu
    from the solver's indices (block by block, as the rank steps grew them)."""
    import torch
    p = MU_PROBS[name]()
    s = _mu_solver(p)
    s.solve(1e-10)
    I, J = s.indices()
    _, sighat = s.preconditioner()
    Am = O.regularized_matrix(oracle_matrix(p), _stored_delta(p))
    ells = [0] + [q["ell"] for q in s.steps()]
    Q, T = None, None
    for a, b_ in zip(ells[:-1], ells[1:]):
        if b_ > a:
            Q, T = O.augment_qr(Q, T, O.rows(Am, I[a:b_]).T)
    Pt = O.build_svdfree_preconditioner(O.cols(Am, J), O.cross(Am, I, J), Q, T, sighat)
    # the power iteration converges to sigma_min(M) from above; with mu > 0 the smallest
    # singular values of A_mu cluster near sqrt(mu) and 50 steps stop within 1e-3 of it
    Minv = np.column_stack([Pt.minv(e) for e in np.eye(Pt.ell)])
    smin = 1.0 / np.linalg.svd(Minv, compute_uv=False)[0]
    assert smin * (1 - 1e-12) <= sighat <= smin * (1 + 1e-3), (sighat, smin)
    # the same 50 steps from the same start vector in the oracle
    assert sighat == pytest.approx(O.svdfree_smallest_sigma(Pt, iters=50), rel=1e-10)
    w = np.random.default_rng(6).standard_normal(p.n)
    out = s.apply_preconditioner(torch.from_numpy(w).cuda()).cpu().numpy()
    assert rel(out, Pt.apply_inv(w)) <= 1e-9
    s.close()
