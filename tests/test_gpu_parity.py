"""CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Tolerances: CUR indices and the sketch are compared exactly; FP64 solutions to a
relative error of 1e-10 (in replay mode the GPU runs the oracle's phase schedule);
FP32-storage mixed runs to 1e-5 against the oracle on the same rounded matrix."""
import math

import numpy as np
import pytest

from oracle import aplicur_oracle as O
from paper_2604_05065_gb300 import workloads as wl

from gpu_helpers import draws, oracle_matrix, rel, schedule, to_device

pytestmark = pytest.mark.gpu


def _solver(p, rows, signs, W, **kw):
    import paper_2604_05065_gb300 as pkg
    A, b = to_device(p)
    return pkg.Solver(A, b, p.mu, p.sketch_dim, sketch_rows=rows, sketch_signs=signs,
                      normest_w=W, **kw)


def _problems():
    return {
        "dense64": wl.config1(scale=4),
        "dense64_full": wl.config1(),
        "sparse64": wl.small_sparse(3000, 300, wl.BASE_SEED + 50, nnz_per_col=6, mu=1e-5,
                                    sketch_dim=10),
        "dense32": wl.dense_lowrank(m=600, n=120, mu=1e-4, sketch_dim=8, index=60,
                                    dtype=np.float32, name="dense32"),
        "sparse32": wl.small_sparse(2500, 250, wl.BASE_SEED + 51, nnz_per_col=5, mu=1e-5,
                                    sketch_dim=10, dtype=np.float32),
    }


PROBS = _problems()


@pytest.mark.parametrize("name", list(PROBS))
def test_sketch_is_bit_exact(name):
    p = PROBS[name]
    rows, signs, W = draws(p)
    s = _solver(p, rows, signs, W)
    Y = s.sketch().cpu().numpy()
    Yo = O.apply_sketch(oracle_matrix(p), rows, signs, O.sketch_rows(p.sketch_dim))
    assert Y.shape == Yo.shape
    assert np.array_equal(Y, Yo)


@pytest.mark.parametrize("name", ["dense64", "sparse64"])
def test_seeded_draws_match_oracle_generator(name):
    """Library and oracle implement the same counter-based generator independently."""
    import paper_2604_05065_gb300 as pkg
    p = PROBS[name]
    A, b = to_device(p)
    s = pkg.Solver(A, b, p.mu, p.sketch_dim, seed=12345)
    Y = s.sketch().cpu().numpy()
    srow = O.sketch_rows(p.sketch_dim)
    from oracle import rng as orng
    rows, signs = orng.sparse_sign(12345, srow, p.m, O.sketch_xi(srow))
    assert np.array_equal(Y, O.apply_sketch(oracle_matrix(p), rows, signs, srow))
    ref = O.aplicur(oracle_matrix(p), p.b, p.mu, p.sketch_dim, O.Options(seed=12345), tol=1e-10)
    s.set_replay(schedule(ref))
    s.solve(1e-10)
    I, J = s.indices()
    assert np.array_equal(I, ref.I) and np.array_equal(J, ref.J)


@pytest.mark.parametrize("name", ["dense64", "sparse64", "dense32"])
def test_matvec(name):
    import torch
    p = PROBS[name]
    rows, signs, W = draws(p)
    s = _solver(p, rows, signs, W)
    A = oracle_matrix(p)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(p.n)
    y = rng.standard_normal(p.m)
    Ax = s.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    Aty = s.matvec(torch.from_numpy(y).cuda(), trans=True).cpu().numpy()
    assert rel(Ax, A @ x) < 1e-13
    assert rel(Aty, A.T @ y) < 1e-13


@pytest.mark.parametrize("name", ["dense64", "dense64_full", "sparse64"])
def test_replay_solve_matches_oracle(name):
    p = PROBS[name]
    rows, signs, W = draws(p)
    A = oracle_matrix(p)
    ref = O.aplicur(A, p.b, p.mu, p.sketch_dim, tol=1e-10, srows=rows, signs=signs, W=W)
    s = _solver(p, rows, signs, W, replay=schedule(ref))
    x = s.solve(1e-10).cpu().numpy()
    I, J = s.indices()
    assert np.array_equal(I, ref.I)
    assert np.array_equal(J, ref.J)
    assert rel(x, ref.x) <= 1e-10
    ph = s.phases()
    assert [q["iters"] for q in ph] == [q["iters"] for q in ref.phases]
    st = s.steps()
    for a, b_ in zip(st, ref.rank_steps):
        assert a["ell"] == b_["ell"]
        assert a["rho"] == pytest.approx(b_["rho"], rel=1e-9)


@pytest.mark.parametrize("name", ["dense64_full", "sparse64"])
def test_free_run_matches_oracle(name):
    p = PROBS[name]
    rows, signs, W = draws(p)
    A = oracle_matrix(p)
    ref = O.aplicur(A, p.b, p.mu, p.sketch_dim, tol=1e-10, srows=rows, signs=signs, W=W)
    s = _solver(p, rows, signs, W)
    x = s.solve(1e-10).cpu().numpy()
    st = s.stats()
    assert st["converged"] == 1 and st["ne_res"] <= 1e-10
    I, J = s.indices()
    assert np.array_equal(I, ref.I) and np.array_equal(J, ref.J)
    # both converged to the same minimiser: error bounded by the residual tolerance
    xd = O.ridge_direct(A, p.b, p.mu) if p.n <= 400 else ref.x
    kappa = 1.0 / math.sqrt(p.mu)
    assert rel(x, xd) <= max(1e-10, 10 * kappa * 1e-10)


@pytest.mark.parametrize("fp64_dense", [0, 1])
def test_preconditioner_matches_oracle(fp64_dense):
    """Both arithmetic forms of the dense factor products (compensated FP32, the default,
    and FP64) reproduce the oracle's singular values and P^-1 to 1e-10."""
    import torch
    p = PROBS["dense64"]
    rows, signs, W = draws(p)
    A = oracle_matrix(p)
    ref = O.aplicur(A, p.b, p.mu, p.sketch_dim, tol=1e-10, srows=rows, signs=signs, W=W)
    s = _solver(p, rows, signs, W, replay=schedule(ref), fp64_dense=fp64_dense)
    s.solve(1e-10)
    sig, sighat = s.preconditioner()
    P = ref.last_P
    assert sig.numel() == P.ell
    sg = sig.cpu().numpy()
    assert rel(sg, P.sig) <= 1e-10
    # sighat = sqrt(sig_ell^2 + delta^2) inherits the absolute error of the smallest singular
    # value, which Weyl's inequality bounds by ||dM||_2 ~ eps * sig_1 (eps ~ 2^-46 for the
    # compensated FP32 products, 2^-53 * dimension for FP64)
    assert abs(sighat - P.sighat) <= 1e-11 * P.sig[0] + 1e-14 * P.sighat
    w = np.random.default_rng(4).standard_normal(p.n)
    out = s.apply_preconditioner(torch.from_numpy(w).cuda()).cpu().numpy()
    assert rel(out, P.apply_inv(w)) <= 1e-10


WELLCOND = {
    "dense": lambda: wl.small_dense(400, 60, 904, decay=1.0, mu=1e-3, sketch_dim=4),
    "sparse": lambda: wl.small_sparse(3000, 300, wl.BASE_SEED + 52, nnz_per_col=6, mu=1e-3,
                                      sketch_dim=10, col_decay=0.5),
}


@pytest.mark.parametrize("name", ["dense", "sparse"])
@pytest.mark.parametrize("k", [1, 5, 12])
def test_plain_lsqr_iterates(name, k):
    """Early iterates on well-conditioned problems, before the Golub-Kahan basis loses
    orthogonality (later iterates of any two LSQR implementations differ by rounding
    amplification, then reconverge; see test_plain_lsqr_converged)."""
    p = WELLCOND[name]()
    rows, signs, W = draws(p)
    A = oracle_matrix(p)
    ref = O.plsqr_phase(A, p.b, math.sqrt(p.mu), np.zeros(p.n), O.identity_preconditioner(p.n),
                        eps_lsqr=0.0, maxit=k)
    s = _solver(p, rows, signs, W)
    x = s.plain_lsqr(0.0, k).cpu().numpy()
    assert s.phases()[0]["iters"] == k
    assert rel(x, ref.x) <= 1e-10


@pytest.mark.parametrize("name", ["dense64", "sparse64"])
def test_plain_lsqr_converged(name):
    p = PROBS[name]
    rows, signs, W = draws(p)
    A = oracle_matrix(p)
    s = _solver(p, rows, signs, W)
    x = s.plain_lsqr(1e-12, 200000).cpu().numpy()
    assert s.stats()["ne_res"] <= 1e-12
    xd = O.ridge_direct(A, p.b, p.mu) if p.fmt == "dense" else O.plain_lsqr(
        A, p.b, p.mu, tol=1e-13).x
    assert rel(x, xd) <= 1e-8


def test_adjoint_gradients_match_oracle():
    import torch
    p = wl.small_dense(300, 40, 901, decay=3.0, mu=1e-3, sketch_dim=5)
    rows, signs, W = draws(p)
    A = p.dense
    s = _solver(p, rows, signs, W)
    x = s.solve(1e-12).cpu().numpy()
    xt = np.random.default_rng(6).standard_normal(p.n)
    g = x - xt
    gb, gmu, gA = s.backward(torch.from_numpy(g).cuda(), tol=1e-12)
    xd = O.ridge_direct(A, p.b, p.mu)
    lam, gb_o, gmu_o, gA_o = O.ridge_gradients(A, p.b, p.mu, xd, xd - xt)
    assert rel(gb.cpu().numpy(), gb_o) <= 1e-8
    assert gmu == pytest.approx(gmu_o, rel=1e-8)
    assert rel(gA.cpu().numpy(), gA_o) <= 1e-8


@pytest.mark.parametrize("name", ["dense32", "sparse32"])
def test_df32_matches_oracle_on_same_rounded_problem(name):
    """Compensated FP32 products reach FP64-level accuracy: same indices and 1e-10."""
    import paper_2604_05065_gb300 as pkg
    p = PROBS[name]
    rows, signs, W = draws(p)
    A = oracle_matrix(p)  # the FP32 values promoted exactly
    ref = O.aplicur(A, p.b, p.mu, p.sketch_dim, tol=1e-10, srows=rows, signs=signs, W=W)
    s = _solver(p, rows, signs, W, precision=pkg.PREC_DF32, replay=schedule(ref))
    x = s.solve(1e-10).cpu().numpy()
    I, J = s.indices()
    assert np.array_equal(I, ref.I) and np.array_equal(J, ref.J)
    assert rel(x, ref.x) <= 1e-10
    s2 = _solver(p, rows, signs, W, precision=pkg.PREC_DF32)
    x2 = s2.solve(1e-10).cpu().numpy()
    assert s2.stats()["ne_res"] <= 1e-10
    assert rel(x2, O.ridge_direct(A, p.b, p.mu)) <= 1e-8


@pytest.mark.parametrize("name", ["dense32", "sparse32"])
def test_mixed_fp32_refinement_against_same_rounded_problem(name):
    """Plain FP32 products: error against the FP64 oracle of the same rounded matrix
    within 1e-5, and the FP64 normal-equation residual at 1e-10.  Each phase solves for a
    correction with right-hand side [0; g / delta], g the FP64 normal-equation residual,
    so FP32 products resolve it to their relative accuracy at every refinement step."""
    import paper_2604_05065_gb300 as pkg
    p = PROBS[name]
    rows, signs, W = draws(p)
    A = oracle_matrix(p)
    xd = O.ridge_direct(A, p.b, p.mu)
    s = _solver(p, rows, signs, W, precision=pkg.PREC_MIXED)
    x = s.solve(1e-10, 200000).cpu().numpy()
    err = rel(x, xd)
    print(f"{name}: mixed FP32 error vs FP64 oracle {err:.3e}, phases {s.phases()}")
    assert err <= 1e-5
    assert s.stats()["ne_res"] <= 1e-10


def test_invalid_arguments_are_rejected():
    import torch
    import paper_2604_05065_gb300 as pkg
    A = torch.zeros(10, 20, dtype=torch.float64, device="cuda")  # m < n
    b = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.AplicurError) as e:
        pkg.Solver(A, b, 1e-4, 2)
    assert e.value.status == 1
    A = torch.randn(30, 10, dtype=torch.float64, device="cuda")
    b = torch.randn(30, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.AplicurError):
        pkg.Solver(A, b, -1.0, 2)
    with pytest.raises(pkg.AplicurError):
        pkg.Solver(A, b, 1e-4, 0)
    with pytest.raises(pkg.AplicurError):
        pkg.Solver(A, b, 1e-4, 11)


def test_zero_rhs_and_exact_low_rank():
    import torch
    import paper_2604_05065_gb300 as pkg
    p = wl.small_dense(200, 30, 902, rank=12, decay=2.0, mu=1e-6, sketch_dim=4)
    A, b = to_device(p)
    s = pkg.Solver(A, torch.zeros_like(b), p.mu, 4, seed=2)
    x = s.solve(1e-10)
    assert float(x.abs().max()) == 0.0
    rows, signs, W = draws(p)
    ref = O.aplicur(p.dense, p.b, p.mu, 4, tol=1e-9, srows=rows, signs=signs, W=W)
    s2 = _solver(p, rows, signs, W)
    x2 = s2.solve(1e-9).cpu().numpy()
    I, J = s2.indices()
    assert len(I) == len(ref.I) == 12
    assert np.array_equal(I, ref.I) and np.array_equal(J, ref.J)
    assert rel(x2, O.ridge_direct(p.dense, p.b, p.mu)) <= 1e-6


def test_rank_beyond_exact_rank_ends_rank_growth_like_the_oracle():
    """Exact rank 9 with blocks of 4: the third block adds columns from rounding noise and
    C^T C is numerically singular.  On both sides rank growth ends at rank 8 (the step is
    dropped) and the solve finishes with the last preconditioner built."""
    p = wl.small_dense(200, 30, 902, rank=9, decay=2.0, mu=1e-6, sketch_dim=4)
    rows, signs, W = draws(p)
    ref = O.aplicur(p.dense, p.b, p.mu, 4, tol=1e-9, srows=rows, signs=signs, W=W)
    assert ref.rank_breakdown and len(ref.I) == 8
    s = _solver(p, rows, signs, W)
    x = s.solve(1e-9).cpu().numpy()
    st = s.stats()
    assert st["rank_breakdown"] == 1 and st["ell"] == 8
    I, J = s.indices()
    assert np.array_equal(I, ref.I) and np.array_equal(J, ref.J)
    assert st["converged"] == int(ref.converged)
    if ref.converged:
        xd = O.ridge_direct(p.dense, p.b, p.mu)
        assert rel(x, xd) <= 10 * 1e-9 / math.sqrt(p.mu)


def test_square_and_full_block():
    """m == n and a block that spans all columns (rank reaches min(m, n))."""
    p = wl.small_dense(48, 48, 903, decay=3.0, mu=1e-4, sketch_dim=16)
    rows, signs, W = draws(p)
    ref = O.aplicur(p.dense, p.b, p.mu, 16, tol=1e-10, srows=rows, signs=signs, W=W)
    s = _solver(p, rows, signs, W, replay=schedule(ref))
    x = s.solve(1e-10).cpu().numpy()
    I, J = s.indices()
    assert np.array_equal(I, ref.I) and np.array_equal(J, ref.J)
    assert rel(x, ref.x) <= 1e-10


def test_deterministic_bitwise_rerun():
    p = PROBS["sparse64"]
    rows, signs, W = draws(p)
    s = _solver(p, rows, signs, W)
    x1 = s.solve(1e-10).cpu().numpy()
    x2 = s.solve(1e-10).cpu().numpy()
    assert np.array_equal(x1, x2)


def test_autograd_function_gradients():
    """torch.autograd.Function wrapper: loss = 0.5 ||x(A, b, mu) - x_target||^2 on a
    scaled-down gradient workload (FP32 A, singular values exp(-i/200)); gradients with
    respect to A, b and mu against the oracle's closed forms at the direct solution."""
    import torch

    import paper_2604_05065_gb300 as pkg
    p = wl.config5(scale=50)  # 2000 x 40
    A64 = p.dense.astype(np.float64)
    xt = p.extra["x_target"]
    fn = pkg.aplicur_solve_fn()
    for mu in (1e-6, 1e-3, 1e-1):
        A = torch.from_numpy(p.dense).cuda().requires_grad_(True)
        b = torch.from_numpy(p.b).cuda().requires_grad_(True)
        m = torch.tensor(mu, dtype=torch.float64, device="cuda", requires_grad=True)
        x = fn.apply(A, b, m, p.sketch_dim, 1e-12, 100000, {"precision": pkg.PREC_DF32})
        loss = 0.5 * ((x - torch.from_numpy(xt).cuda()) ** 2).sum()
        loss.backward()
        xd = O.ridge_direct(A64, p.b, mu)
        _, gb, gmu, gA = O.ridge_gradients(A64, p.b, mu, xd, xd - xt)
        assert rel(x.detach().cpu().numpy(), xd) <= 1e-8
        assert rel(b.grad.cpu().numpy(), gb) <= 1e-7
        assert float(m.grad) == pytest.approx(gmu, rel=1e-6)
        assert rel(A.grad.double().cpu().numpy(), gA) <= 1e-6
