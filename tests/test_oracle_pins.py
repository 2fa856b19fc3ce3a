"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these checks re-derives the oracle's formulas; each compares the oracle
with a library routine, a closed form, an invariant or brute force.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import aplicur_oracle as O
from oracle import rng as orng
from paper_2604_05065_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(m, n, seed):
    return np.random.default_rng(seed).standard_normal((m, n))


# ---------------------------------------------------------------- generator -----------

def test_splitmix64_published_vectors():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            seed, *outs = map(int, line.split())
            assert orng.splitmix64_sequence(seed, 3) == outs


def test_vectorised_mix_matches_scalar():
    idx = np.arange(50, dtype=np.uint64)
    vec = orng._stream_state_np(99, 2, idx)
    assert [int(v) for v in vec] == [orng.stream_state(99, 2, int(i)) for i in idx]


def test_gaussian_w_statistics():
    W = orng.gaussian_w(7, 4000, 10)
    assert W.shape == (4000, 10)
    assert abs(W.mean()) < 0.02 and abs(W.var() - 1.0) < 0.03
    # fourth moment of N(0,1) is 3
    assert abs(np.mean(W ** 4) - 3.0) < 0.15


# ---------------------------------------------------------------- sketch --------------

@pytest.mark.parametrize("s,xi", [(22, 8), (5, 5), (110, 8), (3, 1)])
def test_sparse_sign_structure(s, xi):
    rows, signs = orng.sparse_sign(11, s, 500, xi)
    assert rows.shape == (500, xi)
    assert rows.min() >= 0 and rows.max() < s
    for i in range(500):
        assert len(set(rows[i].tolist())) == xi
    assert set(np.unique(signs).tolist()) <= {-1, 1}
    S = O.dense_S(rows, signs, s)
    nnz = np.count_nonzero(S, axis=0)
    assert np.all(nnz == xi)
    assert np.allclose(np.abs(S[S != 0]), 1.0 / math.sqrt(xi), rtol=0, atol=0)


def test_sketch_equals_dense_S_product():
    A = _rand(300, 40, 1)
    rows, signs = orng.sparse_sign(3, 22, 300, 8)
    Y = O.apply_sketch(A, rows, signs, 22)
    S = O.dense_S(rows, signs, 22)
    assert np.allclose(Y, S @ A, rtol=1e-13, atol=1e-13)


def test_sketch_sparse_and_dense_bitwise_equal():
    p = wl.small_sparse(400, 60, wl.BASE_SEED + 40, nnz_per_col=4)
    rows, signs = orng.sparse_sign(5, 11, p.m, 8)
    Ys = O.apply_sketch(p.to_scipy(), rows, signs, 11)
    Yd = O.apply_sketch(p.to_dense64(), rows, signs, 11)
    assert np.array_equal(Ys, Yd)


def test_sketch_is_norm_preserving_in_expectation():
    x = np.random.default_rng(2).standard_normal((200, 1))
    vals = []
    for seed in range(300):
        rows, signs = orng.sparse_sign(seed, 11, 200, 8)
        vals.append(float(np.sum(O.apply_sketch(x, rows, signs, 11) ** 2)))
    assert abs(np.mean(vals) / float(np.sum(x * x)) - 1.0) < 0.05


def test_sketch_rows_is_exact_ceiling():
    for b in range(1, 400):
        assert O.sketch_rows(b) == math.ceil(11 * b / 10)
    assert O.sketch_rows(20) == 22 and O.sketch_rows(100) == 110 and O.sketch_rows(250) == 275


# ---------------------------------------------------------------- LUPP ----------------

def _lapack_perm(X):
    _, piv = sla.lu_factor(X, check_finite=False)
    perm = np.arange(X.shape[0])
    for i, p in enumerate(piv):
        perm[[i, p]] = perm[[p, i]]
    return perm


@pytest.mark.parametrize("shape,k", [((50, 10), 10), ((200, 30), 25), ((30, 30), 30),
                                     ((1000, 7), 7)])
def test_lupp_matches_lapack_getrf(shape, k):
    X = _rand(*shape, seed=shape[0] + k)
    res = O.lupp_pivots(X, k)
    assert res.nz == k
    assert np.array_equal(res.piv, _lapack_perm(X)[:k])


def test_lupp_ties_follow_lapack():
    X = np.array([[1.0, 2.0], [-1.0, 1.0], [1.0, 5.0], [0.5, -4.0]])
    res = O.lupp_pivots(X, 2)
    assert np.array_equal(res.piv, _lapack_perm(X)[:2])
    assert res.piv[0] == 0


def test_lupp_zero_pivot_stops():
    X = np.zeros((6, 3))
    X[2, 0] = 1.0
    res = O.lupp_pivots(X, 3)
    assert res.nz == 1 and res.piv.tolist() == [2]


# ---------------------------------------------------------------- CUR -----------------

def _cur_state(A, b, steps, seed=4):
    m, n = A.shape
    s = O.sketch_rows(b)
    rows, signs = orng.sparse_sign(seed, s, m, O.sketch_xi(s))
    Y = O.apply_sketch(A, rows, signs, s)
    I = np.zeros(0, np.int64)
    J = np.zeros(0, np.int64)
    core = None
    E = Y.copy()
    for _ in range(steps):
        Ip, Jp, _ = O.augment_cur(A, I, J, E, core, b)
        I = np.concatenate([I, Ip])
        J = np.concatenate([J, Jp])
        core = O.Core(A, I, J)
        E = O.sketched_residual(A, Y, I, J, core)
    return Y, I, J, core, E


def test_cur_cross_interpolation():
    p = wl.small_dense(120, 40, 777, decay=4.0)
    A = p.dense
    Y, I, J, core, E = _cur_state(A, 5, 3)
    assert len(I) == len(J) == 15 and len(set(I)) == 15 and len(set(J)) == 15
    CUR = A[:, J] @ core.solve(A[I, :])
    scale = np.abs(A).max()
    assert np.allclose(CUR[I, :], A[I, :], atol=1e-10 * scale)
    assert np.allclose(CUR[:, J], A[:, J], atol=1e-10 * scale)
    # the sketched residual vanishes on the selected columns and equals S (A - CUR)
    assert np.abs(E[:, J]).max() < 1e-10 * np.abs(Y).max()
    s = O.sketch_rows(5)
    rows, signs = orng.sparse_sign(4, s, A.shape[0], O.sketch_xi(s))
    S = O.dense_S(rows, signs, s)
    assert np.allclose(E, S @ (A - CUR), atol=1e-10 * np.abs(Y).max())


def test_cur_column_residual_vanishes_on_selected_rows():
    p = wl.small_dense(100, 30, 778, decay=3.0)
    A = p.dense
    Y, I, J, core, E = _cur_state(A, 4, 2)
    Er = E.copy()
    Er[:, J] = 0
    Jp = O.lupp_pivots(Er.T, 4).piv
    Ecol = A[:, Jp] - A[:, J] @ core.solve(A[np.ix_(I, Jp)])
    assert np.abs(Ecol[I, :]).max() < 1e-11 * np.abs(A).max()


def test_exact_low_rank_terminates_with_zero_residual():
    p = wl.small_dense(90, 30, 779, rank=12, decay=2.0, mu=1e-6, sketch_dim=4)
    res = O.aplicur(p.dense, p.b, p.mu, 4, O.Options(seed=3), tol=1e-9)
    assert len(res.I) == 12
    assert res.rank_steps[-1]["rho"] < 1e-9
    assert res.converged


def test_norm_estimate_bounds_two_norm():
    E = _rand(30, 200, 12) * np.logspace(0, -3, 200)
    W = orng.gaussian_w(1, 200, 10)
    rho = O.norm_estimate(E, W)
    assert rho >= np.linalg.norm(E, 2)
    # ||E w|| <= ||E||_2 ||w||: the estimate is at most 10 sqrt(2/pi) ||E||_2 max ||w_i||
    assert rho <= O.NORMEST_FACTOR * np.linalg.norm(E, 2) * np.linalg.norm(W, axis=0).max()


# ---------------------------------------------------------------- augmentQR -----------

def test_augment_qr_matches_householder():
    X = _rand(80, 24, 21)
    Q, T = O.augment_qr(None, None, X[:, :8])
    Q, T = O.augment_qr(Q, T, X[:, 8:16])
    Q, T = O.augment_qr(Q, T, X[:, 16:])
    assert np.allclose(Q.T @ Q, np.eye(24), atol=1e-13)
    assert np.allclose(np.triu(T), T)
    assert np.allclose(Q @ T, X, atol=1e-12)
    Qh, Rh = np.linalg.qr(X)
    sg = np.sign(np.diag(Rh))
    assert np.allclose(Q, Qh * sg, atol=1e-11)
    assert np.allclose(T, Rh * sg[:, None], atol=1e-11)


# ---------------------------------------------------------------- preconditioner ------

def _cur_preconditioner(A, b, steps, delta):
    Y, I, J, core, E = _cur_state(A, b, steps)
    Q, T = None, None
    for k in range(steps):
        Q, T = O.augment_qr(Q, T, A[I[k * b:(k + 1) * b], :].T)
    P = O.build_preconditioner(A[:, J], core, Q, T, delta)
    return P, I, J, core


def test_preconditioner_exact_spectrum_on_cur_approximation():
    """Theorem (condition number bound), proof: the regularised CUR approximation times
    P^{-1} has singular values sighat (ell times) and delta (n - ell times)."""
    p = wl.small_dense(150, 40, 780, decay=5.0)
    A = p.dense
    delta = 1e-2
    P, I, J, core = _cur_preconditioner(A, 5, 3, delta)
    CUR = A[:, J] @ core.solve(A[I, :])
    n = A.shape[1]
    Pinv = np.column_stack([P.apply_inv(e) for e in np.eye(n)])
    sv = np.linalg.svd(np.vstack([CUR, delta * np.eye(n)]) @ Pinv, compute_uv=False)
    ell = P.ell
    assert ell == 15
    assert np.allclose(sv[:ell], P.sighat, rtol=1e-9)
    assert np.allclose(sv[ell:], delta, rtol=1e-9)
    # ||P^{-1}|| <= 1 and P P^{-1} = I
    assert np.linalg.norm(Pinv, 2) <= 1 + 1e-12
    PP = np.column_stack([P.apply(P.apply_inv(e)) for e in np.eye(n)])
    assert np.allclose(PP, np.eye(n), atol=1e-12)
    # the CUR singular values are those of the CUR approximation itself
    assert np.allclose(P.sig, np.linalg.svd(CUR, compute_uv=False)[:ell], rtol=1e-8)


def test_optimal_preconditioner_condition_number():
    """Section 3.1: with Vhat = V_ell and target level sqrt(sigma_{ell+1}^2 + mu^2) the
    condition number drops to sqrt((sigma_{ell+1}^2+mu^2)/(sigma_n^2+mu^2))."""
    p = wl.small_dense(100, 30, 781, decay=6.0)
    A = p.dense
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    ell, delta = 8, 1e-3
    Lam = np.sqrt(s[:ell] ** 2 + delta ** 2)
    sighat = math.sqrt(s[ell] ** 2 + delta ** 2)
    P = O.Preconditioner(Vt[:ell].T, s[:ell], Lam, sighat, sighat / Lam - 1.0)
    n = A.shape[1]
    Pinv = np.column_stack([P.apply_inv(e) for e in np.eye(n)])
    sv = np.linalg.svd(np.vstack([A, delta * np.eye(n)]) @ Pinv, compute_uv=False)
    kappa = sv[0] / sv[-1]
    assert kappa == pytest.approx(math.sqrt((s[ell] ** 2 + delta ** 2) / (s[-1] ** 2 + delta ** 2)),
                                  rel=1e-9)


# ---------------------------------------------------------------- SVD-free variant ----

def _svdfree_pair(A, b, steps, sighat):
    """The SVD-free operator and the SVD-based one (mu = 0, same target level sighat)
    from the same CUR factors."""
    Y, I, J, core, E = _cur_state(A, b, steps)
    Q, T = None, None
    for k in range(steps):
        Q, T = O.augment_qr(Q, T, A[I[k * b:(k + 1) * b], :].T)
    Pt = O.build_svdfree_preconditioner(A[:, J], A[np.ix_(I, J)], Q, T, sighat)
    P0 = O.build_preconditioner(A[:, J], core, Q, T, 0.0)
    P = O.Preconditioner(P0.Vhat, P0.sig, P0.Lam, sighat, sighat / P0.Lam - 1.0)
    return Pt, P, I, J


def _dense_op(f, n):
    return np.column_stack([f(e) for e in np.eye(n)])


def test_svdfree_exact_low_rank_flattens_to_the_target_level():
    """For A = C U R exactly (rank ell), A Q_R = Q_C M, so A Ptilde^{-1} = sighat Q_C Q_R^T:
    ell singular values equal to sighat and the rest zero (a transposed factor or a missing
    T_C in M^{-1} breaks this)."""
    rng = np.random.default_rng(790)
    m, n, r = 90, 36, 12
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    sighat = 0.37
    Pt, _, I, J = _svdfree_pair(A, 4, 3, sighat)
    assert Pt.ell == r
    sv = np.linalg.svd(A @ _dense_op(Pt.apply_inv, n), compute_uv=False)
    assert np.allclose(sv[:r], sighat, rtol=1e-9)
    assert np.all(sv[r:] <= 1e-9 * sighat)


def test_svdfree_lemma_same_spectrum_as_svd_based():
    """Lemma (SVD-free preconditioner): Ptilde^{-1} = P^{-1} W with W orthogonal, so at
    mu = 0 the preconditioned matrices have the same singular values."""
    p = wl.small_dense(120, 40, 791, decay=4.0)
    A = p.dense
    Pt, P, I, J = _svdfree_pair(A, 5, 3, 2.5e-3)
    n = A.shape[1]
    Ptinv = _dense_op(Pt.apply_inv, n)
    Pinv = _dense_op(P.apply_inv, n)
    s1 = np.linalg.svd(A @ Ptinv, compute_uv=False)
    s2 = np.linalg.svd(A @ Pinv, compute_uv=False)
    assert np.allclose(s1, s2, rtol=1e-9, atol=1e-12 * s2[0])
    W = np.linalg.solve(Pinv, Ptinv)
    assert np.allclose(W.T @ W, np.eye(n), atol=1e-8)


def test_svdfree_transpose_inverse_and_complement():
    """apply_inv_T is the adjoint of apply_inv, apply inverts apply_inv, and both act as
    the identity on the orthogonal complement of range(Q_R)."""
    p = wl.small_dense(100, 30, 792, decay=3.0)
    A = p.dense
    Pt, _, I, J = _svdfree_pair(A, 4, 2, 0.9)
    n = A.shape[1]
    rng = np.random.default_rng(793)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    assert float(Pt.apply_inv(x) @ y) == pytest.approx(float(x @ Pt.apply_inv_T(y)), rel=1e-12)
    assert np.allclose(Pt.apply(Pt.apply_inv(x)), x, atol=1e-10 * np.linalg.norm(x))
    w = x - Pt.Q_R @ (Pt.Q_R.T @ x)
    assert np.allclose(Pt.apply_inv(w), w, atol=1e-13 * np.linalg.norm(x))
    assert np.allclose(Pt.apply_inv_T(w), w, atol=1e-13 * np.linalg.norm(x))


def test_svdfree_power_iteration_finds_the_smallest_cur_singular_value():
    """sigma_min(M) from M^{-1} alone equals the smallest singular value of the CUR
    approximation (the SVD-based form's sigma_ell), so the SVD-free operator with that
    target level conditions A like the SVD-based one (the Lemma)."""
    p = wl.small_dense(300, 40, 905, decay=3.0)
    A = p.dense
    Pt, P, I, J = _svdfree_pair(A, 4, 6, 1.0)
    est = O.svdfree_smallest_sigma(Pt, iters=80)
    assert est == pytest.approx(float(P.sig[-1]), rel=1e-6)
    Pt.sighat = est
    n = A.shape[1]
    P2 = O.Preconditioner(P.Vhat, P.sig, P.Lam, est, est / P.Lam - 1.0)
    s1 = np.linalg.svd(A @ _dense_op(Pt.apply_inv, n), compute_uv=False)
    s2 = np.linalg.svd(A @ _dense_op(P2.apply_inv, n), compute_uv=False)
    assert np.allclose(s1, s2, rtol=1e-9)
    assert s1[0] / s1[-1] < 0.1 * np.linalg.cond(A)


# ---------------------------------------------------------------- single-shot ---------

def test_fixed_rank_single_shot_selects_like_lupp_on_the_sketch():
    """Fixed-rank single-shot (bsize = max_rank = ell): the columns are LAPACK's first ell
    row pivots of (S A)^T and the rows its first ell row pivots of C = A(:, J)
    (Algorithm "Sketched CUR with cross approximation using LUPP"), on the same sketch."""
    p = wl.small_dense(160, 40, 794, decay=3.0, mu=1e-6, sketch_dim=12)
    A = p.dense
    ell = 12
    s = O.sketch_rows(ell)
    rows, signs = orng.sparse_sign(9, s, p.m, O.sketch_xi(s))
    W = orng.gaussian_w(9, p.n, 10)
    res = O.aplicur(A, p.b, p.mu, ell, O.Options(seed=9, single_shot=True, max_rank=ell),
                    tol=1e-10, srows=rows, signs=signs, W=W)
    Y = O.apply_sketch(A, rows, signs, s)
    J = _lapack_perm(Y.T)[:ell]
    I = _lapack_perm(A[:, J])[:ell]
    assert np.array_equal(res.J, J) and np.array_equal(res.I, I)
    assert len(res.rank_steps) == 1 and res.rank_steps[0]["rebuild"]


def test_rank_adaptive_single_shot_builds_once_and_solves():
    """Rank-adaptive single-shot: the rank grows as in the adaptive driver, the
    preconditioner is built once (at the last rank step), every phase runs with it, and the
    solve reaches the ridge solution."""
    p = wl.config1(scale=4)
    A = p.dense
    ada = O.aplicur(A, p.b, p.mu, p.sketch_dim, O.Options(seed=3), tol=1e-10)
    res = O.aplicur(A, p.b, p.mu, p.sketch_dim, O.Options(seed=3, single_shot=True), tol=1e-10)
    flags = [st["rebuild"] for st in res.rank_steps]
    assert flags[-1] and not any(flags[:-1])
    assert np.array_equal(res.I, ada.I) and np.array_equal(res.J, ada.J)
    assert {ph["ell"] for ph in res.phases} == {len(res.I)}
    assert res.converged
    xd = O.ridge_direct(A, p.b, p.mu)
    assert np.linalg.norm(res.x - xd) <= 1e-6 * np.linalg.norm(xd)


# ---------------------------------------------------------------- LSQR ----------------

@pytest.mark.parametrize("k", [1, 2, 5, 12])
def test_unpreconditioned_phase_equals_scipy_damped_lsqr(k):
    """LSQR on [A; delta I] and Paige-Saunders damped LSQR minimise the same residual over
    the same Krylov space, so their k-th iterates coincide."""
    p = wl.small_dense(200, 50, 782, decay=2.0)
    delta = 0.05
    P = O.identity_preconditioner(50)
    res = O.plsqr_phase(p.dense, p.b, delta, np.zeros(50), P, eps_lsqr=0.0, maxit=k)
    ref = spla.lsqr(p.dense, p.b, damp=delta, atol=0, btol=0, conlim=0, iter_lim=k)[0]
    assert res.iters == k
    assert np.linalg.norm(res.x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_phibar_tracks_explicit_residual():
    p = wl.small_dense(150, 40, 783, decay=3.0)
    delta = 1e-2
    P, *_ = _cur_preconditioner(p.dense, 5, 2, delta)
    x0 = np.random.default_rng(5).standard_normal(40) * 0.1
    for k in (1, 3, 6):
        res = O.plsqr_phase(p.dense, p.b, delta, x0, P, eps_lsqr=0.0, maxit=k)
        r = np.concatenate([p.b - p.dense @ res.x, -delta * res.x])
        assert res.phibar[-1] == pytest.approx(np.linalg.norm(r), rel=1e-10)


def test_preconditioned_phase_converges_to_ridge_solution():
    p = wl.small_dense(200, 50, 784, decay=4.0, mu=1e-4)
    delta = 1e-2
    P, *_ = _cur_preconditioner(p.dense, 5, 3, delta)
    res = O.plsqr_phase(p.dense, p.b, delta, np.zeros(50), P, eps_lsqr=1e-14, maxit=2000)
    xd = O.ridge_direct(p.dense, p.b, p.mu)
    assert np.linalg.norm(res.x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_ridge_direct_matches_normal_equations():
    A = _rand(60, 20, 8)
    b = np.random.default_rng(9).standard_normal(60)
    mu = 0.3
    x = O.ridge_direct(A, b, mu)
    assert np.allclose(x, np.linalg.solve(A.T @ A + mu * np.eye(20), A.T @ b), rtol=1e-12)
    assert np.allclose(O.ridge_direct(sp.csr_matrix(A), b, mu), x, rtol=1e-13)


def test_dynamic_stop_rule():
    # rate_1 = log 2; rate_j = log(1.001) -> ratio ~ 694 > 100
    assert O.dynamic_stop(1.001, 1.0, math.log(2.0), 100.0, 0.0)
    assert not O.dynamic_stop(2.0, 1.0, math.log(2.0), 100.0, 0.0)
    # absolute drop below sigma_ell
    assert O.dynamic_stop(2.0, 1.0, math.log(2.0), 100.0, 1.5)
    # no progress counts as an infinite ratio; disabled in the final phase
    assert O.dynamic_stop(1.0, 1.0, math.log(2.0), 100.0, 0.0)
    assert not O.dynamic_stop(1.0, 1.0, math.log(2.0), math.inf, 5.0)


# ---------------------------------------------------------------- driver --------------

def test_aplicur_reaches_ridge_solution_and_residual_is_monotone():
    p = wl.config1(scale=4)       # 500 x 50
    res = O.aplicur(p.dense, p.b, p.mu, p.sketch_dim, O.Options(seed=2), tol=1e-11)
    xd = O.ridge_direct(p.dense, p.b, p.mu)
    assert res.converged
    kappa = 1.0 / math.sqrt(p.mu)
    assert np.linalg.norm(res.x - xd) <= kappa * 1e-10 * np.linalg.norm(xd) * 10
    assert len(res.phases) >= 2
    ne = [ph["ne_res"] for ph in res.phases]
    assert ne[-1] <= 1e-11


def test_aplicur_warm_restart_residual_nonincreasing():
    p = wl.small_dense(300, 60, 785, decay=5.0, mu=1e-5, sketch_dim=5)
    A = p.dense
    delta = math.sqrt(p.mu)
    res_norms = []
    orig = O.plsqr_phase

    def spy(A_, b_, d_, x0, P, **kw):
        r = orig(A_, b_, d_, x0, P, **kw)
        for xv in (x0, r.x):
            res_norms.append(math.hypot(np.linalg.norm(b_ - A_ @ xv), d_ * np.linalg.norm(xv)))
        return r

    O.plsqr_phase = spy
    try:
        O.aplicur(A, p.b, p.mu, 5, O.Options(seed=4), tol=1e-10)
    finally:
        O.plsqr_phase = orig
    assert len(res_norms) >= 4
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res_norms, res_norms[1:]))


def test_replay_reproduces_free_run():
    p = wl.small_dense(200, 40, 786, decay=5.0, mu=1e-5, sketch_dim=4)
    free = O.aplicur(p.dense, p.b, p.mu, 4, O.Options(seed=5), tol=1e-10)
    sched = {"phases": [ph["iters"] for ph in free.phases],
             "rebuild": [st["rebuild"] for st in free.rank_steps]}
    rep = O.aplicur(p.dense, p.b, p.mu, 4, O.Options(seed=5, replay=sched), tol=1e-10)
    assert np.array_equal(rep.I, free.I) and np.array_equal(rep.J, free.J)
    assert np.array_equal(rep.x, free.x)


# ---------------------------------------------------------------- adjoint -------------

def test_ridge_gradients_match_central_differences():
    rng = np.random.default_rng(10)
    A = rng.standard_normal((40, 12))
    b = rng.standard_normal(40)
    xt = rng.standard_normal(12)
    mu = 0.05

    def loss(A_, b_, mu_):
        x = O.ridge_direct(A_, b_, mu_)
        return 0.5 * float(np.sum((x - xt) ** 2))

    x = O.ridge_direct(A, b, mu)
    lam, gb, gmu, gA = O.ridge_gradients(A, b, mu, x, x - xt)
    h = 1e-6
    db = rng.standard_normal(40)
    fd = (loss(A, b + h * db, mu) - loss(A, b - h * db, mu)) / (2 * h)
    assert fd == pytest.approx(float(gb @ db), rel=1e-6)
    hm = 1e-6 * mu
    fd = (loss(A, b, mu + hm) - loss(A, b, mu - hm)) / (2 * hm)
    assert fd == pytest.approx(gmu, rel=1e-6)
    for (i, j) in [(0, 0), (5, 3), (39, 11), (17, 6)]:
        E = np.zeros_like(A)
        E[i, j] = 1.0
        fd = (loss(A + h * E, b, mu) - loss(A - h * E, b, mu)) / (2 * h)
        assert fd == pytest.approx(gA[i, j], rel=1e-5, abs=1e-9)


# ---------------------------------------------------------------- pins of three steps --
# Row selection at ell > 0, the re-preconditioning decision, and the constant of rho.
# Each pin has a companion test that plants a plausible mistake in the oracle (on the
# CPU, through monkeypatch) and checks that the pin then fails.

def _independent_row_pivots(A, Y_S, I, J, Jp):
    """I_+ from first principles (Algorithm augmentCUR, row step): the residual
    A - A(:,J) pinv(A(I,J)) A(I,:) formed with the SVD-based pseudo-inverse, restricted
    to the new columns J_+, rows I zeroed, and LAPACK getrf's first |J_+| row pivots."""
    Res = A - A[:, J] @ np.linalg.pinv(A[np.ix_(I, J)]) @ A[I, :]
    Ecol = Res[:, Jp].copy()
    Ecol[I, :] = 0.0
    return _lapack_perm(Ecol)[:len(Jp)]


def _independent_col_pivots(A, S, I, J, b):
    """J_+ from first principles (column step): S (A - CUR) with a dense S and the
    pseudo-inverse core, columns J zeroed, LAPACK's first b pivots of its transpose."""
    Res = A - A[:, J] @ np.linalg.pinv(A[np.ix_(I, J)]) @ A[I, :]
    Er = S @ Res
    Er[:, J] = 0.0
    return _lapack_perm(Er.T)[:b]


def _row_selection_case():
    p = wl.small_dense(150, 45, 4242, decay=3.0)
    A = p.dense
    b = 5
    Y, I, J, core, E = _cur_state(A, b, 3, seed=6)       # ell = 15
    s = O.sketch_rows(b)
    rows_, signs = orng.sparse_sign(6, s, A.shape[0], O.sketch_xi(s))
    S = O.dense_S(rows_, signs, s)
    return A, S, I, J, core, E, b


def _row_selection_matches(A, S, I, J, core, E, b):
    Ip, Jp, margin = O.augment_cur(A, I, J, E, core, b)
    Jx = _independent_col_pivots(A, S, I, J, b)
    Ix = _independent_row_pivots(A, None, I, J, Jp)
    return np.array_equal(Jp, Jx) and np.array_equal(Ip, Ix), margin


def test_row_selection_at_positive_rank_matches_lapack_on_independent_residual():
    A, S, I, J, core, E, b = _row_selection_case()
    assert len(I) == 15
    ok, margin = _row_selection_matches(A, S, I, J, core, E, b)
    assert margin > 1e-6          # no near-tie: the pivots are well defined
    assert ok


@pytest.mark.parametrize("plant", ["drop_cur_term", "transposed_core_solve"])
def test_row_selection_pin_catches_planted_mistakes(monkeypatch, plant):
    A, S, I, J, core, E, b = _row_selection_case()
    if plant == "drop_cur_term":
        # E_col = A(:, J+) without the C U A(I, J+) correction
        monkeypatch.setattr(O.Core, "solve", lambda self, B: np.zeros((self.ell, B.shape[1])))
    else:
        # A(I,J)^{-T} B in place of A(I,J)^{-1} B
        monkeypatch.setattr(O.Core, "solve",
                            lambda self, B: sla.lu_solve(self.lu, B, trans=1, check_finite=False))
    ok, _ = _row_selection_matches(A, S, I, J, core, E, b)
    assert not ok


# hand-worked rho sequence: eps_cur = 0.5, nu_prec = 10; every quotient is exact in binary
#   rho     gap    d_cur before   d_cur / gap      rebuild   d_cur after
#   1000.5  1000   inf            inf              yes       1000
#   500.5   500    1000           2                no        1000
#   100.5   100    1000           10 (>= 10)       yes       100
#   20.5    20     100            5                no        100
#   12.5    12     100            8.33             no        100
#   10.5    10     100            10               yes       10
#   40.5    40     10             0.25             no        10
#   0.5     0      10             (rho <= eps)     yes       0
_RHO_SEQ = [1000.5, 500.5, 100.5, 20.5, 12.5, 10.5, 40.5, 0.5]
_REBUILD = [True, False, True, False, False, True, False, True]


def _run_rule(rule_cls):
    rule = rule_cls(0.5, 10.0)
    flags = []
    for rho in _RHO_SEQ:
        f = rule.wants_rebuild(rho)
        flags.append(f)
        if f:
            rule.rebuilt(rho)
    return flags


def test_rebuild_decision_on_hand_worked_rho_sequence():
    assert _run_rule(O.RebuildRule) == _REBUILD


@pytest.mark.parametrize("plant", ["strict_compare", "gap_every_step"])
def test_rebuild_decision_pin_catches_planted_mistakes(monkeypatch, plant):
    if plant == "strict_compare":
        def wants(self, rho):
            return rho <= self.eps_cur or self.d_cur / (rho - self.eps_cur) > self.nu_prec
        monkeypatch.setattr(O.RebuildRule, "wants_rebuild", wants)
    else:
        orig = O.RebuildRule.wants_rebuild

        def wants(self, rho):
            f = orig(self, rho)
            self.d_cur = rho - self.eps_cur      # gap recorded at every step
            return f
        monkeypatch.setattr(O.RebuildRule, "wants_rebuild", wants)
    assert _run_rule(O.RebuildRule) != _REBUILD


def test_driver_uses_the_rebuild_rule(monkeypatch):
    """The driver's rebuild flags follow RebuildRule (a planted always-rebuild rule
    changes them), so the hand-worked pin covers the free-running schedule."""
    p = wl.config1(scale=4)
    base = O.aplicur(p.dense, p.b, p.mu, p.sketch_dim, O.Options(seed=2), tol=1e-11)
    monkeypatch.setattr(O.RebuildRule, "wants_rebuild", lambda self, rho: True)
    planted = O.aplicur(p.dense, p.b, p.mu, p.sketch_dim, O.Options(seed=2), tol=1e-11)
    fb = [s["rebuild"] for s in base.rank_steps]
    fp = [s["rebuild"] for s in planted.rank_steps]
    assert not all(fb) and all(fp)


def test_norm_estimate_closed_form_on_rank_one():
    """E = u v^T: ||E w_i|| = ||u|| |v^T w_i|, so Eq. 2normestimate gives
    rho = 10 sqrt(2/pi) ||u|| max_i |v^T w_i| (the paper's constant, typed here)."""
    g = np.random.default_rng(77)
    u = g.standard_normal(40)
    v = g.standard_normal(300)
    W = orng.gaussian_w(5, 300, 10)
    closed = 10.0 * math.sqrt(2.0 / math.pi) * np.linalg.norm(u) * np.abs(v @ W).max()
    assert O.norm_estimate(np.outer(u, v), W) == pytest.approx(closed, rel=1e-13)


@pytest.mark.parametrize("factor", [10.0, 10.0 * math.sqrt(2.0), math.sqrt(2.0 / math.pi)])
def test_norm_estimate_pin_catches_a_wrong_constant(monkeypatch, factor):
    monkeypatch.setattr(O, "NORMEST_FACTOR", factor)
    g = np.random.default_rng(77)
    u = g.standard_normal(40)
    v = g.standard_normal(300)
    W = orng.gaussian_w(5, 300, 10)
    closed = 10.0 * math.sqrt(2.0 / math.pi) * np.linalg.norm(u) * np.abs(v @ W).max()
    assert O.norm_estimate(np.outer(u, v), W) != pytest.approx(closed, rel=1e-6)


# ---------------------------------------------------------------- reused QR -----------

def test_ridge_qr_reuse_matches_direct_solves_and_gradients():
    """RidgeQR gives ridge_direct's solution and ridge_gradients' lambda from one
    factorisation, and grad_A_entries the entries of the full gradient."""
    p = wl.small_dense(150, 25, 4343, decay=2.0, mu=1e-3)
    A, b, mu = p.dense, p.b, p.mu
    qr = O.RidgeQR(A, mu)
    x = qr.solve(b)
    assert np.allclose(x, O.ridge_direct(A, b, mu), rtol=1e-12, atol=0)
    g = np.random.default_rng(3).standard_normal(25)
    lam_o, gb_o, gmu_o, gA_o = O.ridge_gradients(A, b, mu, x, g)
    lam = qr.solve(np.zeros(150), g / math.sqrt(mu))
    assert np.allclose(lam, lam_o, rtol=1e-12, atol=0)
    rows = np.array([0, 7, 149, 33])
    cols = np.array([0, 24, 5, 5])
    assert np.allclose(O.grad_A_entries(A, b, x, lam, rows, cols), gA_o[rows, cols], rtol=1e-12)


def test_ridge_reduced_matches_direct_solves_and_rank_one_changes():
    """The QR-reduced ridge problem gives ridge_direct's solution for several mu, the
    solution of A + h u v^T (u with components inside and outside range(A)), and
    ridge_gradients' lambda."""
    p = wl.small_dense(200, 30, 4545, decay=3.0, mu=1e-4)
    A, b = p.dense, p.b
    red = O.RidgeReduced(A)
    g = np.random.default_rng(5)
    u = g.standard_normal(200)
    v = g.standard_normal(30)
    for mu in (1e-8, 1e-4, 1e-1):
        x = red.solve(b, mu)
        assert np.allclose(x, O.ridge_direct(A, b, mu), rtol=1e-10, atol=0)
        xp = red.solve(b, mu, u, v, 1e-3)
        assert np.allclose(xp, O.ridge_direct(A + 1e-3 * np.outer(u, v), b, mu), rtol=1e-9,
                           atol=0)
        gg = g.standard_normal(30)
        lam_o = O.ridge_gradients(A, b, mu, x, gg)[0]
        assert np.allclose(red.adjoint(mu, gg), lam_o, rtol=1e-9, atol=0)


# ---------------------------------------------------------------- dense sketches ------

def test_gaussian_sketch_moments_and_embedding():
    """Entries of G / sqrt(s) have mean 0 and variance 1/s, and E ||S x||^2 = ||x||^2."""
    s, m = 20, 5000
    S = orng.gaussian_sketch(11, s, m)
    assert S.shape == (s, m)
    v = S.ravel() * math.sqrt(s)
    assert abs(v.mean()) < 5.0 / math.sqrt(v.size)
    assert abs(v.var() - 1.0) < 5.0 * math.sqrt(2.0 / v.size)
    x = np.random.default_rng(2).standard_normal(300)
    # seeds far apart: the stream of entry i is keyed by seed ^ i, so nearby small seeds
    # would share entries
    vals = [np.linalg.norm(orng.gaussian_sketch(k << 40, 10, 300) @ x) ** 2 for k in range(200)]
    assert np.mean(vals) == pytest.approx(float(x @ x), rel=0.1)


def test_srht_rows_are_sylvester_hadamard_rows():
    """S sqrt(s) / d equals the sampled rows of scipy's Sylvester-Hadamard matrix (columns
    past m cut), S S^T = (m/s) I when m is a power of two, and E ||S x||^2 = ||x||^2 with
    padding."""
    s, m = 12, 64
    S = orng.srht_sketch(4, s, m)
    rows, d = orng.srht_rows_signs(4, s, m)
    assert len(set(rows.tolist())) == s
    H = sla.hadamard(64)
    assert np.array_equal(S * math.sqrt(s) / d[None, :], H[rows, :m])
    assert np.allclose(S @ S.T, (m / s) * np.eye(s), atol=1e-12)
    x = np.random.default_rng(3).standard_normal(50)   # padded to 64
    vals = [np.linalg.norm(orng.srht_sketch(k << 40, 16, 50) @ x) ** 2 for k in range(300)]
    assert np.mean(vals) == pytest.approx(float(x @ x), rel=0.1)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(9).standard_normal(10000) * 10.0 ** np.random.default_rng(10).integers(-20, 20, 10000)
    ours = orng.round_bf16(x)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)
    assert orng.round_bf16([1.0 + 2.0 ** -8])[0] == 1.0             # tie to even
    assert orng.round_bf16([1.0 + 3 * 2.0 ** -8])[0] == 1.0 + 2 ** -6  # tie to even, up


def test_bf16_expansion():
    """Three bfloat16 terms hold an FP32 value exactly; each term is a bfloat16 number at
    most 2^-8 of the one before (rounding to nearest leaves half an ulp of 8 bits); two
    terms leave at most 2^-16 relative."""
    g = np.random.default_rng(11)
    x = g.standard_normal(20000) * 10.0 ** g.integers(-30, 30, 20000)
    f = x.astype(np.float32).astype(np.float64)
    p = orng.bf16_pieces(x, 3)
    assert np.array_equal(p[0] + p[1] + p[2], f)
    for q in p:
        assert np.array_equal(orng.round_bf16(q), q)
    assert np.all(np.abs(p[1]) <= 2.0 ** -8 * np.abs(p[0]))
    assert np.all(np.abs(p[2]) <= 2.0 ** -8 * np.abs(p[1]))
    assert np.all(np.abs(f - p[0] - p[1]) <= 2.0 ** -16 * np.abs(f))
    assert np.array_equal(orng.bf16_pieces(x, 1)[0], orng.round_bf16(x))
    # a value that needs all three terms: 1 + 2^-9 + 2^-20
    v = orng.bf16_pieces([1.0 + 2.0 ** -9 + 2.0 ** -20], 3)
    assert [float(q[0]) for q in v] == [1.0, 2.0 ** -9, 2.0 ** -20]


@pytest.mark.parametrize("kind", ["gaussian", "srht"])
def test_aplicur_with_dense_sketch_reaches_ridge_solution(kind):
    p = wl.small_dense(400, 50, 4646, decay=3.0, mu=1e-4, sketch_dim=5)
    s = O.sketch_rows(5)
    S = (orng.gaussian_sketch if kind == "gaussian" else orng.srht_sketch)(2, s, p.m)
    res = O.aplicur(p.dense, p.b, p.mu, 5, O.Options(seed=2), tol=1e-11, S=S)
    assert res.converged
    assert np.allclose(res.Y, S @ p.dense, rtol=1e-13, atol=1e-13 * np.abs(res.Y).max())
    x = O.ridge_direct(p.dense, p.b, p.mu)
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) < 1e-7


# ------------------------------------------------------- SVD-free variant, mu > 0 ------

def test_regularized_matrix():
    """A_mu = [A; delta I]: A_mu^T A_mu = A^T A + delta^2 I, row m + j is delta e_j^T (dense
    and CSR alike)."""
    import scipy.sparse as sps
    g = np.random.default_rng(41)
    A = g.standard_normal((30, 12))
    for M in (A, sps.csr_matrix(A)):
        Am = O.regularized_matrix(M, 0.25)
        D = Am.toarray() if sps.issparse(Am) else Am
        assert D.shape == (42, 12)
        assert np.allclose(D.T @ D, A.T @ A + 0.0625 * np.eye(12), rtol=1e-13, atol=1e-13)
        assert np.array_equal(D[30 + 5], 0.25 * np.eye(12)[5])


def test_svdfree_mu_full_rank_cur_flattens_the_regularized_matrix():
    """At full rank the CUR of A_mu is exact (A_mu = C U R), so [A; delta I] Ptilde^{-1}
    = sighat Q_C Q_R^T: all n singular values equal sighat.  The same operator built from a
    CUR of A alone (also exact at full rank, for A) leaves [A; delta I] unflattened."""
    g = np.random.default_rng(42)
    m, n, delta = 60, 20, 0.3
    A = (g.standard_normal((m, n)) * 10.0 ** -np.linspace(0, 3, n)) @ np.linalg.qr(
        g.standard_normal((n, n)))[0]
    Am = O.regularized_matrix(A, delta)
    sighat = 0.7
    Pt, _, I, J = _svdfree_pair(Am, 5, 4, sighat)
    assert Pt.ell == n and np.any(I >= m)
    sv = np.linalg.svd(Am @ _dense_op(Pt.apply_inv, n), compute_uv=False)
    assert np.allclose(sv, sighat, rtol=1e-9)
    Pa, _, _, _ = _svdfree_pair(A, 5, 4, sighat)
    sva = np.linalg.svd(Am @ _dense_op(Pa.apply_inv, n), compute_uv=False)
    assert sva[0] / sva[-1] > 10.0


@pytest.mark.parametrize("kind", ["dense", "sparse"])
def test_svdfree_mu_driver_reaches_ridge_solution(kind):
    """The SVD-free variant with mu > 0 (CUR of A_mu, sketch over m + n columns, LSQR on
    [A; delta I] Ptilde^{-1} with the transposed operator on the A^T side) converges to
    the ridge solution and selects rows of the appended delta I block."""
    p = (wl.small_dense(400, 60, 904, decay=6.0, mu=1e-4, sketch_dim=4) if kind == "dense"
         else wl.small_sparse(3000, 300, wl.BASE_SEED + 50, nnz_per_col=6, mu=1e-5,
                              sketch_dim=10))
    A = p.dense if kind == "dense" else p.to_scipy()
    res = O.aplicur(A, p.b, p.mu, p.sketch_dim, O.Options(seed=3, variant="svdfree"), tol=1e-10)
    assert res.converged
    assert np.any(res.I >= p.m)
    xd = O.ridge_direct(A if kind == "dense" else A.toarray(), p.b, p.mu)
    kappa = 1.0 / math.sqrt(p.mu)
    assert np.linalg.norm(res.x - xd) / np.linalg.norm(xd) <= 10 * kappa * 1e-10


def test_svdfree_lsqr_needs_the_transposed_operator():
    """Ptilde is not symmetric: LSQR on A Ptilde^{-1} must apply Ptilde^{-T} on the A^T
    side.  With Ptilde^{-1} there instead (a planted mistake) the phase no longer solves
    the least-squares problem."""
    p = wl.small_dense(200, 30, 906, decay=4.0, mu=0.0, sketch_dim=4)
    A = p.dense
    Pt, _, I, J = _svdfree_pair(A, 4, 3, 0.5)
    xd = np.linalg.lstsq(A, p.b, rcond=None)[0]

    def run(P):
        r = O.plsqr_phase(A, p.b, 0.0, np.zeros(p.n), P, eps_lsqr=1e-14, maxit=400)
        return np.linalg.norm(r.x - xd) / np.linalg.norm(xd)

    assert run(Pt) <= 1e-8

    class Planted(O.SvdFreePreconditioner):
        def apply_inv_T(self, w):
            return self.apply_inv(w)

    bad = Planted(Pt.Q_R, Pt.T_R, Pt.T_C, Pt.A_IJ, Pt.sighat)
    assert run(bad) > 1e-3


def test_ridge_sparse_matches_the_dense_solution():
    """Conjugate gradients on the normal equations reach the dense QR ridge solution (a
    different method for the same closed form) and report a residual at its tolerance."""
    p = wl.small_sparse(2000, 150, wl.BASE_SEED + 53, nnz_per_col=4, mu=1e-4, sketch_dim=10)
    A = p.to_scipy()
    x, res = O.ridge_sparse(A, p.b, p.mu)
    xd = O.ridge_direct(A.toarray(), p.b, p.mu)
    assert res <= 1e-14
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-9


def test_rank_step_breakdown_ends_rank_growth():
    """Past the exact rank (rank 9, blocks of 4) the third block's columns make C^T C
    singular: the oracle drops that step, ends rank growth at rank 8 and still reaches the
    ridge solution with the last preconditioner."""
    p = wl.small_dense(200, 30, 902, rank=9, decay=2.0, mu=1e-6, sketch_dim=4)
    s = O.sketch_rows(4)
    rows, signs = orng.sparse_sign(5, s, p.m, O.sketch_xi(s))
    W = orng.gaussian_w(5, p.n, 10)
    res = O.aplicur(p.dense, p.b, p.mu, 4, tol=1e-9, srows=rows, signs=signs, W=W)
    assert res.rank_breakdown and len(res.I) == 8 and len(res.rank_steps) == 2
    assert res.converged
    xd = O.ridge_direct(p.dense, p.b, p.mu)
    assert np.linalg.norm(res.x - xd) / np.linalg.norm(xd) <= 1e-6
