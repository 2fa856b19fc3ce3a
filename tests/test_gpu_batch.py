"""Batched multi-right-hand-side solves (aplicur_batch_*) against the oracle.

A small batch of uneven dense and CSR FP32 problems (the batched workload's recipe at
reduced sizes), three right-hand sides each.  For every (problem, right-hand side) pair:
the CUR indices agree with the oracle's APLICUR run seeded with seed + p (bit-exact on
their common prefix: the batched run continues rank steps until all right-hand sides of
the problem converged), the reported normal-equation residual is at most tol, and the
solution is within the FP32-variant bound 1e-5 of the oracle's direct ridge solution and
within the rigorous bound ||x - x*|| <= ||A^T(b - Ax) - mu x|| / mu."""
import numpy as np
import pytest

from oracle import aplicur_oracle as O
from paper_2604_05065_gb300 import workloads as wl

from gpu_helpers import oracle_matrix, rel, to_device

pytestmark = pytest.mark.gpu

SEED = 11
MU = 1e-5


def _batch(nrhs=3, nprob=6, seed=7):
    return wl.batched(nprob=nprob, m_range=(300, 800), n_range=(30, 80), density=0.03,
                      nrhs=nrhs, mu=MU, sketch_dim=8, seed=seed)


def _solver(probs, **kw):
    import torch

    import paper_2604_05065_gb300 as pkg
    mats, rhs = [], []
    for p in probs:
        A, _ = to_device(p)
        mats.append(A)
        rhs.append(torch.from_numpy(np.asarray(p.b, dtype=np.float64)).cuda())
    return pkg.BatchSolver(mats, rhs, MU, probs[0].sketch_dim, seed=SEED, **kw)


def _dense64(p):
    A = oracle_matrix(p)
    return A.toarray() if hasattr(A, "toarray") else A


def _check_solution(x, A64, b, mu, ne, target=1e-5):
    xd = O.ridge_direct(A64, b, mu)
    err = np.linalg.norm(x - xd)
    atb = np.linalg.norm(A64.T @ b)
    assert err <= 1.01 * ne * atb / mu + 1e-13
    if target is not None:
        assert rel(x, xd) <= target


def test_batch_matches_oracle():
    probs = _batch()
    sol = _solver(probs)
    xs = sol.solve(1e-10)
    st = sol.stats()
    assert st["pairs"] == len(probs) * 3 and st["converged"] == st["pairs"]
    for p, prob in enumerate(probs):
        A64 = _dense64(prob)
        info = sol.problem(p)
        ref = O.aplicur(oracle_matrix(prob), prob.b[:, 0], MU, prob.sketch_dim,
                        O.Options(seed=SEED + p), tol=1e-10)
        k = min(len(ref.I), info["ell"])
        assert k > 0
        assert np.array_equal(info["I"][:k], ref.I[:k])
        assert np.array_equal(info["J"][:k], ref.J[:k])
        x = xs[p].cpu().numpy()
        for r in range(3):
            pr = sol.pair(p, r)
            assert pr["converged"] and pr["ne_res"] <= 1e-10
            _check_solution(x[:, r], A64, prob.b[:, r], MU, pr["ne_res"])
    sol.close()


def test_batch_plain_lsqr_reaches_the_same_solutions():
    """Unpreconditioned: the Paige-Saunders test 2 (relative to ||A|| ||r||, eps 1e-10)
    ends its phases near 1e-9 on the ill-conditioned dense problems, so the target is
    the benchmark's 1e-8 and the check the rigorous error bound."""
    probs = _batch()
    sol = _solver(probs)
    xs = sol.plain_lsqr(1e-8, 200000)
    for p, prob in enumerate(probs):
        A64 = _dense64(prob)
        x = xs[p].cpu().numpy()
        for r in range(3):
            pr = sol.pair(p, r)
            assert pr["converged"] and pr["ne_res"] <= 1e-8
            _check_solution(x[:, r], A64, prob.b[:, r], MU, pr["ne_res"], target=None)
    sol.close()


def test_batch_single_rhs_zero_rhs_and_rerun_is_bitwise():
    probs = _batch(nrhs=1, nprob=4, seed=9)
    probs[1].b[:] = 0.0
    sol = _solver(probs)
    x1 = [x.cpu().numpy() for x in sol.solve(1e-10)]
    x2 = [x.cpu().numpy() for x in sol.solve(1e-10)]
    assert np.all(x1[1] == 0.0) and sol.pair(1, 0)["converged"]
    for a, b in zip(x1, x2):
        assert np.array_equal(a, b)
    for p, prob in enumerate(probs):
        if p == 1:
            continue
        _check_solution(x1[p][:, 0], _dense64(prob), prob.b[:, 0], MU, sol.pair(p, 0)["ne_res"])
    sol.close()


def test_batch_rejects_bad_arguments():
    import torch

    import paper_2604_05065_gb300 as pkg
    probs = _batch(nrhs=1, nprob=2)
    A, _ = to_device(probs[0])
    b = torch.zeros(probs[0].m, 17, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.AplicurError):
        pkg.BatchSolver([A], [b], MU, 8)  # 17 right-hand sides
    A64 = A.double() if A.layout == torch.strided else A.to_dense().double()
    with pytest.raises(pkg.AplicurError):
        pkg.BatchSolver([A64], [b[:, :1]], MU, 8)  # FP64 values


def test_batch_sixteen_rhs_matches_the_direct_solution():
    """16 right-hand sides (the 16-wide kernel instances of the batched workload) on a
    small uneven batch; every pair against the oracle's direct ridge solution."""
    probs = wl.batched(nprob=4, m_range=(300, 700), n_range=(30, 70), density=0.03, nrhs=16,
                       mu=MU, sketch_dim=8, seed=21)
    sol = _solver(probs)
    xs = sol.solve(1e-10)
    assert sol.stats()["converged"] == 4 * 16
    for p, prob in enumerate(probs):
        A64 = _dense64(prob)
        x = xs[p].cpu().numpy()
        assert x.shape == (prob.n, 16)
        for r in range(16):
            _check_solution(x[:, r], A64, prob.b[:, r], MU, sol.pair(p, r)["ne_res"])
    sol.close()


def test_batch_backward_matches_oracle_gradients():
    """aplicur_batch_backward: for the loss 0.5 sum_r ||x_r - t_r||^2 of every problem,
    dL/db, dL/dmu per pair and dL/dA (dense problems, summed over the right-hand sides)
    against the oracle's ridge gradients at the oracle's direct solution (FP32-storage
    gate 1e-5); CSR problems get no dL/dA."""
    import torch
    probs = _batch(nrhs=3, nprob=6, seed=9)
    sol = _solver(probs)
    xs = sol.solve(1e-10)
    g = np.random.default_rng(12)
    targets = [g.standard_normal((q.n, 3)) for q in probs]
    grads = [xs[p] - torch.from_numpy(targets[p]).cuda() for p in range(len(probs))]
    gb, gmu, gA = sol.backward(grads, tol=1e-10)
    assert sol.stats()["converged"] == sol.stats()["pairs"]
    gmu = gmu.cpu().numpy()
    for p, prob in enumerate(probs):
        A64 = _dense64(prob)
        gA_o = np.zeros_like(A64)
        for r in range(3):
            xd = O.ridge_direct(A64, prob.b[:, r], MU)
            lam, gb_o, gmu_o, gA_r = O.ridge_gradients(A64, prob.b[:, r], MU, xd,
                                                       xd - targets[p][:, r])
            assert rel(gb[p][:, r].cpu().numpy(), gb_o) <= 1e-5
            assert abs(gmu[p, r] - gmu_o) <= 1e-5 * abs(gmu_o)
            gA_o += gA_r
        if prob.fmt == "dense":
            assert rel(gA[p].double().cpu().numpy(), gA_o) <= 1e-5
        else:
            assert gA[p] is None
    sol.close()


def test_batch_backward_needs_a_solve():
    import torch

    import paper_2604_05065_gb300 as pkg
    probs = _batch(nrhs=1, nprob=2, seed=5)
    sol = _solver(probs)
    with pytest.raises(pkg.AplicurError) as e:
        sol.backward([torch.zeros(q.n, 1, dtype=torch.float64, device="cuda") for q in probs])
    assert e.value.status == 1
    sol.close()
