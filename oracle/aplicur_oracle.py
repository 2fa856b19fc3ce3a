"""Plain FP64 CPU restatement of APLICUR (adaptive CUR-preconditioned LSQR).

TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and the benchmark's CPU
baseline leg may import this module.  It shares no code with the CUDA path.

Paper: Huh, Cartis, Nakatsukasa, "Adaptive LSQR Preconditioning from One Small
Sketch" (arXiv 2604.05065).  Section / equation / algorithm names below are the
paper's.  Conventions fixed for this project where the paper is loose:

* the user coefficient `mu` multiplies ||x||^2 (Eq. regularizedLLS); the damping
  used in every formula that the paper writes with mu (A_mu, Lambda-hat, the
  target level, eps_cur = 30 mu) is delta = sqrt(mu).
* sketch rows s = ceil(1.1 b), sparsity xi = min(8, s) (Algorithm "APLICUR:
  detailed implementation", Initialise).
* target level sigma-hat = sqrt(sigma_ell^2 + delta^2) (Algorithm
  CURPreconditioner).
* rho is the absolute randomized 2-norm bound of Eq. 2normestimate, r = 10.
* LUPP ties go to the first candidate in the current (swapped) row order,
  as in LAPACK getrf; a zero pivot ends the selection (rank exhausted).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import rng as orng

NORMEST_FACTOR = 10.0 * math.sqrt(2.0 / math.pi)


# --------------------------------------------------------------------------------------
# matrix access (A is a dense float64 ndarray or a scipy.sparse CSR matrix)
# --------------------------------------------------------------------------------------

def _is_sparse(A) -> bool:
    return sp.issparse(A)


def cols(A, J) -> np.ndarray:
    """A(:, J) as a dense m x |J| array."""
    J = np.asarray(J, dtype=np.int64)
    if _is_sparse(A):
        return np.asarray(A[:, J].toarray(), dtype=np.float64)
    return np.array(A[:, J], dtype=np.float64)


def rows(A, I) -> np.ndarray:
    """A(I, :) as a dense |I| x n array."""
    I = np.asarray(I, dtype=np.int64)
    if _is_sparse(A):
        return np.asarray(A[I, :].toarray(), dtype=np.float64)
    return np.array(A[I, :], dtype=np.float64)


def cross(A, I, J) -> np.ndarray:
    """A(I, J) as a dense array."""
    return cols(A, J)[np.asarray(I, dtype=np.int64), :] if len(I) else np.zeros((0, len(J)))


def matvec(A, x):
    return np.asarray(A @ x, dtype=np.float64)


def rmatvec(A, y):
    return np.asarray(A.T @ y, dtype=np.float64)


def regularized_matrix(A, delta: float):
    """A_mu = [A; delta I] ((m + n) x n): the matrix whose CUR the SVD-free variant takes
    for regularised problems (section "SVD-free variant", last paragraph).  Row m + j is
    delta e_j^T."""
    n = A.shape[1]
    if _is_sparse(A):
        return sp.vstack([A.tocsr().astype(np.float64), delta * sp.identity(n, format="csr")],
                         format="csr")
    return np.vstack([np.asarray(A, dtype=np.float64), delta * np.eye(n)])


# --------------------------------------------------------------------------------------
# Sketch (Definition "sparse sign embedding", Section 5.1; Algorithm APLICUR lines 3-4)
# --------------------------------------------------------------------------------------

def sketch_rows(b: int) -> int:
    """s = ceil(1.1 b) computed exactly in integers."""
    return (11 * b + 9) // 10


def sketch_xi(s: int, xi_max: int = 8) -> int:
    return min(xi_max, s)


def dense_S(srows: np.ndarray, signs: np.ndarray, s: int) -> np.ndarray:
    """The s x m sparse sign embedding as a dense matrix: column i holds signs[i,k] /
    sqrt(xi) at rows srows[i,k]."""
    m, xi = srows.shape
    S = np.zeros((s, m))
    scale = 1.0 / math.sqrt(xi)
    for i in range(m):
        for k in range(xi):
            S[srows[i, k], i] = signs[i, k] * scale
    return S


def apply_sketch(A, srows: np.ndarray, signs: np.ndarray, s: int) -> np.ndarray:
    """Y = S A.  Every Y(r, j) is accumulated over the rows i of A in ascending order
    (the canonical order), in FP64, then scaled by xi^(-1/2) once."""
    m, xi = srows.shape
    n = A.shape[1]
    Y = np.zeros((s, n))
    if _is_sparse(A):
        A = A.tocsr()
        for i in range(m):
            lo, hi = A.indptr[i], A.indptr[i + 1]
            if lo == hi:
                continue
            cj = A.indices[lo:hi]
            vals = np.asarray(A.data[lo:hi], dtype=np.float64)
            for k in range(xi):
                Y[srows[i, k], cj] += signs[i, k] * vals
    else:
        for i in range(m):
            ai = np.asarray(A[i], dtype=np.float64)
            for k in range(xi):
                if signs[i, k] > 0:
                    Y[srows[i, k]] += ai
                else:
                    Y[srows[i, k]] -= ai
    Y *= 1.0 / math.sqrt(xi)
    return Y


def dense_sketch(A, S: np.ndarray) -> np.ndarray:
    """Y = S A for a dense sketching operator S (s x m): the Gaussian embedding or the
    SRFT of the appendix "Sketch comparison", applied by its definition in FP64."""
    if _is_sparse(A):
        return np.asarray((A.T @ S.T).T, dtype=np.float64)
    return S @ np.asarray(A, dtype=np.float64)


# --------------------------------------------------------------------------------------
# LU with partial pivoting, first k pivots (used by augmentCUR)
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class LuppResult:
    piv: np.ndarray        # original row indices of the first `nz` pivots
    nz: int                # pivots taken before the first zero pivot
    margin: float          # min over steps of (|best| - |second best|) / |best|


def lupp_pivots(X: np.ndarray, k: int) -> LuppResult:
    """Row pivots of Gaussian elimination with partial pivoting on X (N x K), k steps.

    Step j: among the rows not yet pivoted, take the one with the largest |X(., j)|
    (first in the current swapped order on ties), swap it to position j and eliminate
    column j from the rows below.  Stops early at a zero pivot."""
    X = np.array(X, dtype=np.float64, copy=True)
    N, K = X.shape
    k = min(k, N, K)
    perm = np.arange(N)
    margin = math.inf
    nz = 0
    for j in range(k):
        col = np.abs(X[j:, j])
        p = j + int(np.argmax(col))
        best = col[p - j]
        if not best > 0.0:
            break
        if col.size > 1:
            rest = np.delete(col, p - j)
            margin = min(margin, (best - rest.max()) / best)
        if p != j:
            X[[j, p], :] = X[[p, j], :]
            perm[[j, p]] = perm[[p, j]]
        l = X[j + 1:, j] / X[j, j]
        X[j + 1:, j] = l
        X[j + 1:, j + 1:] -= np.outer(l, X[j, j + 1:])
        nz += 1
    return LuppResult(perm[:nz].copy(), nz, margin)


# --------------------------------------------------------------------------------------
# CUR pieces (Definition "cur"; Algorithms augmentCUR, IterativeCUR)
# --------------------------------------------------------------------------------------

class Core:
    """U = A(I, J)^dagger held as an LU factorisation of the square cross A(I, J);
    pseudo-inverse only when the LU has an exact zero pivot."""

    def __init__(self, A, I, J):
        self.ell = len(I)
        self.AIJ = cross(A, I, J)
        self.pinv = None
        self.lu = None
        if self.ell:
            lu, piv = sla.lu_factor(self.AIJ, check_finite=False)
            if np.any(np.diag(lu) == 0.0):
                self.pinv = np.linalg.pinv(self.AIJ)
            else:
                self.lu = (lu, piv)

    def solve(self, B):
        """U B = A(I,J)^{-1} B."""
        if self.pinv is not None:
            return self.pinv @ B
        return sla.lu_solve(self.lu, B, check_finite=False)

    def rsolve(self, B):
        """B U = B A(I,J)^{-1}."""
        if self.pinv is not None:
            return B @ self.pinv
        return sla.lu_solve(self.lu, B.T, trans=1, check_finite=False).T


def augment_cur(A, I, J, E_row, core: Core | None, bsize: int):
    """Algorithm augmentCUR: next column indices from LUPP of E_row^T, next row indices
    from LUPP of the column residual.  Returns (I_plus, J_plus, margin)."""
    m, n = A.shape
    ell = len(J)
    Er = np.array(E_row, copy=True)
    if ell:
        Er[:, np.asarray(J)] = 0.0
    kj = min(bsize, min(m, n) - ell)
    rc = lupp_pivots(Er.T, kj)
    Jp = rc.piv
    if rc.nz == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), rc.margin
    # E_col = A(:, J+) - C U R(:, J+)
    Ecol = cols(A, Jp)
    if ell:
        Ecol -= cols(A, J) @ core.solve(cross(A, I, Jp))
        Ecol[np.asarray(I), :] = 0.0
    rr = lupp_pivots(Ecol, len(Jp))
    k = min(rc.nz, rr.nz)
    return rr.piv[:k], Jp[:k], min(rc.margin, rr.margin)


def sketched_residual(A, Y, I, J, core: Core | None) -> np.ndarray:
    """E_row = S A - S C U R = Y - Y(:, J) A(I,J)^{-1} A(I, :)  (S C taken from Y)."""
    if not len(J):
        return np.array(Y, copy=True)
    return Y - core.rsolve(Y[:, np.asarray(J)]) @ rows(A, I)


def norm_estimate(E_row: np.ndarray, W: np.ndarray) -> float:
    """Eq. 2normestimate: rho = 10 sqrt(2/pi) max_i ||E_row w_i||."""
    return NORMEST_FACTOR * float(np.max(np.linalg.norm(E_row @ W, axis=0)))


def qr_pos(X: np.ndarray):
    """Householder thin QR with a nonnegative diagonal of R."""
    Q, R = np.linalg.qr(X, mode="reduced")
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * sgn, R * sgn[:, None]


def augment_qr(Q, T, C):
    """Algorithm augmentQR: append columns C to the thin QR (Q, T) with two classical
    Gram-Schmidt passes, then a thin QR of the remaining block."""
    if Q is None or Q.shape[1] == 0:
        return qr_pos(C)
    P1 = Q.T @ C
    E = C - Q @ P1
    P2 = Q.T @ E
    E = E - Q @ P2
    QE, RE = qr_pos(E)
    k, p = T.shape[0], C.shape[1]
    Tn = np.zeros((k + p, k + p))
    Tn[:k, :k] = T
    Tn[:k, k:] = P1 + P2
    Tn[k:, k:] = RE
    return np.hstack([Q, QE]), Tn


# --------------------------------------------------------------------------------------
# Preconditioner (Eq. preconditioner2, Algorithm CURPreconditioner)
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Preconditioner:
    Vhat: np.ndarray          # n x ell, orthonormal columns
    sig: np.ndarray           # singular values of M, descending (Sigma-hat)
    Lam: np.ndarray           # sqrt(sig^2 + delta^2)
    sighat: float             # target level sqrt(sig_ell^2 + delta^2)
    coef: np.ndarray          # sighat / Lam - 1

    @property
    def ell(self) -> int:
        return self.Vhat.shape[1]

    def apply_inv(self, w):
        """P^{-1} w = sighat Vhat Lam^{-1} Vhat^T w + (I - Vhat Vhat^T) w."""
        return w + self.Vhat @ (self.coef * (self.Vhat.T @ w))

    def apply_inv_T(self, w):
        """P^{-T} w = P^{-1} w (P is symmetric)."""
        return self.apply_inv(w)

    def apply(self, w):
        """P w = sighat^{-1} Vhat Lam Vhat^T w + (I - Vhat Vhat^T) w."""
        return w + self.Vhat @ ((self.Lam / self.sighat - 1.0) * (self.Vhat.T @ w))

    @property
    def norm(self) -> float:
        """||P||_2 = Lam_1 / sighat (>= 1)."""
        return float(self.Lam[0] / self.sighat) if self.ell else 1.0

    @property
    def sig_ell(self) -> float:
        return float(self.sig[-1]) if self.ell else 0.0


def chol_upper(G: np.ndarray) -> np.ndarray:
    """Upper-triangular T with T^T T = G (Cholesky)."""
    return sla.cholesky(G, lower=False, check_finite=False)


def build_preconditioner(C: np.ndarray, core: Core, Q_R: np.ndarray, T_R: np.ndarray,
                         delta: float, T_C: np.ndarray | None = None) -> Preconditioner:
    """Algorithm CURPreconditioner: T_C = chol(C^T C) (or the given factor); M = T_C U T_R^T;
    SVD of M; Vhat = Q_R V_M; Lam = sqrt(sig^2 + delta^2); sighat = sqrt(sig_ell^2 + delta^2)."""
    if T_C is None:
        T_C = chol_upper(C.T @ C)
    M = T_C @ core.solve(T_R.T)
    _, sig, VMt = np.linalg.svd(M)
    Vhat = Q_R @ VMt.T
    Lam = np.sqrt(sig * sig + delta * delta)
    sighat = math.sqrt(sig[-1] ** 2 + delta * delta)
    return Preconditioner(Vhat, sig, Lam, sighat, sighat / Lam - 1.0)


def identity_preconditioner(n: int) -> Preconditioner:
    e = np.zeros(0)
    return Preconditioner(np.zeros((n, 0)), e, e, 1.0, e)


# --------------------------------------------------------------------------------------
# SVD-free variant (Section "SVD-free variant", Eq. preconditioner_svdfree, Algorithm
# SVD-free CURPreconditioner; unregularised problems, mu = 0)
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class SvdFreePreconditioner:
    """Ptilde^{-1} = sighat Q_R M^{-1} Q_R^T + (I - Q_R Q_R^T) with the core
    M = T_C A(I,J)^{-1} T_R^T never formed or decomposed: M^{-1} = T_R^{-T} A(I,J) T_C^{-1}
    is applied as two triangular solves around a product with the cross A(I,J).
    Ptilde is not symmetric, so LSQR on A Ptilde^{-1} needs apply_inv_T as well."""
    Q_R: np.ndarray           # n x ell, orthonormal columns
    T_R: np.ndarray           # ell x ell upper triangular, R^T = Q_R T_R
    T_C: np.ndarray           # ell x ell upper triangular, C^T C = T_C^T T_C
    A_IJ: np.ndarray          # ell x ell cross A(I, J)
    sighat: float             # target level: the CUR error estimate

    @property
    def ell(self) -> int:
        return self.Q_R.shape[1]

    def minv(self, t):
        """M^{-1} t = T_R^{-T} (A(I,J) (T_C^{-1} t))."""
        y = sla.solve_triangular(self.T_C, t, lower=False, check_finite=False)
        return sla.solve_triangular(self.T_R, self.A_IJ @ y, trans="T", lower=False,
                                    check_finite=False)

    def minv_T(self, t):
        """M^{-T} t = T_C^{-T} (A(I,J)^T (T_R^{-1} t))."""
        y = sla.solve_triangular(self.T_R, t, lower=False, check_finite=False)
        return sla.solve_triangular(self.T_C, self.A_IJ.T @ y, trans="T", lower=False,
                                    check_finite=False)

    def apply_inv(self, w):
        t = self.Q_R.T @ w
        return w + self.Q_R @ (self.sighat * self.minv(t) - t)

    def apply_inv_T(self, w):
        t = self.Q_R.T @ w
        return w + self.Q_R @ (self.sighat * self.minv_T(t) - t)

    @property
    def norm(self) -> float:
        """Taken as 1 in the explicit-residual trigger (||Ptilde||_2 is not formed)."""
        return 1.0

    @property
    def sig_ell(self) -> float:
        """The dynamic stop's smallest CUR singular value: the target level."""
        return self.sighat

    def apply(self, w):
        """Ptilde w = sighat^{-1} Q_R M Q_R^T w + (I - Q_R Q_R^T) w, M = T_C A(I,J)^{-1} T_R^T."""
        t = self.Q_R.T @ w
        Mt = self.T_C @ np.linalg.solve(self.A_IJ, self.T_R.T @ t)
        return w + self.Q_R @ (Mt / self.sighat - t)


def build_svdfree_preconditioner(C: np.ndarray, A_IJ: np.ndarray, Q_R: np.ndarray,
                                 T_R: np.ndarray, sighat: float,
                                 T_C: np.ndarray | None = None) -> SvdFreePreconditioner:
    """Algorithm SVD-free CURPreconditioner: T_C = chol(C^T C) (or the given factor); the
    operator is kept as its factors (Q_R, T_R, T_C, A(I,J)) and the target level sighat
    (the estimate rho of Eq. 2normestimate)."""
    return SvdFreePreconditioner(Q_R, T_R, chol_upper(C.T @ C) if T_C is None else T_C,
                                 np.array(A_IJ, copy=True), float(sighat))


def svdfree_start_vector(ell: int) -> np.ndarray:
    """The power iteration's fixed start vector, entries 1 + ((7919 i) mod 101) / 101 for
    i = 0 .. ell - 1 (no special structure; the same start on every implementation)."""
    i = np.arange(ell, dtype=np.int64)
    return 1.0 + ((7919 * i) % 101).astype(np.float64) / 101.0


def svdfree_smallest_sigma(P: SvdFreePreconditioner, iters: int = 50) -> float:
    """sigma_min(M) = 1 / ||M^{-1}||_2 by `iters` steps of power iteration on M^{-T} M^{-1}
    from the fixed start vector, using only the variant's triangular solves and A(I,J)
    products.  (Not in the paper: a target level near sigma_ell without the SVD, see the
    measured sensitivity of sighat = rho.)  Converges from above; when the smallest
    singular values of M cluster, 50 steps stop measurably above sigma_min."""
    v = svdfree_start_vector(P.ell)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        y = P.minv_T(P.minv(v))
        lam = float(np.linalg.norm(y))
        v = y / lam
    return 1.0 / math.sqrt(lam)


# --------------------------------------------------------------------------------------
# Preconditioned LSQR phase (Section 2.2; warm start of Section 3.2; stopping rules of
# Section 5.3.2).  Golub-Kahan bidiagonalisation of Abar = [A; delta I] P^{-1} with an
# explicit (m+n)-vector u, right-hand side rbar = b_aug - A_delta x0.
# --------------------------------------------------------------------------------------

def dynamic_stop(phibar_prev: float, phibar: float, rate1: float, nu: float,
                 sig_ell: float) -> bool:
    """Section 5.3.2: stop when cvgrate_1/cvgrate_j > nu or cvgdiff_j < sigma_ell, with
    cvgrate_j = log(phibar_{j-1}/phibar_j), cvgdiff_j = phibar_{j-1} - phibar_j.
    A non-positive rate counts as an infinite ratio."""
    if not math.isfinite(nu):
        return False
    if phibar_prev - phibar < sig_ell:
        return True
    if phibar <= 0.0:
        return False
    rate = math.log(phibar_prev / phibar)
    if rate <= 0.0:
        return True
    return rate1 / rate > nu


@dataclasses.dataclass
class PhaseResult:
    x: np.ndarray
    iters: int
    reason: str
    phibar: list
    ne_checks: int = 0


def ne_residual(A, b, mu, x, norm_Atb) -> float:
    """||A^T (b - A x) - mu x|| / ||A^T b||."""
    r = b - matvec(A, x)
    return float(np.linalg.norm(rmatvec(A, r) - mu * x) / norm_Atb)


def plsqr_phase(A, b, delta, x0, P: Preconditioner, *, eps_lsqr=1e-10, nu=math.inf,
                maxit=10 ** 6, tol=0.0, norm_Atb=1.0, check_gap=10, fixed_len=None
                ) -> PhaseResult:
    """One warm-started LSQR phase.  Stops on (in this order): exact breakdown, the
    fixed length (replay), Paige-Saunders test 2 (alpha |c| <= eps ||Abar||_est),
    test 1 (phibar <= eps beta_1), the dynamic rule, an explicit normal-equation
    residual <= tol (tried when ||P|| phibar alpha |c| / ||A^T b|| <= tol), maxit."""
    mu = delta * delta
    x = np.array(x0, dtype=np.float64, copy=True)
    u_top = b - matvec(A, x)
    u_bot = -delta * x
    beta = math.sqrt(float(u_top @ u_top + u_bot @ u_bot))
    if beta == 0.0:
        return PhaseResult(x, 0, "exact", [0.0])
    u_top /= beta
    u_bot /= beta
    # Abar^T u = P^{-T} (A^T u_top + delta u_bot); Abar z = [A; delta I] P^{-1} z
    v = P.apply_inv_T(rmatvec(A, u_top) + delta * u_bot)
    alpha = math.sqrt(float(v @ v))
    if alpha == 0.0:
        return PhaseResult(x, 0, "exact", [beta])
    v /= alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    beta1 = beta
    anorm2 = 0.0
    hist = [phibar]
    rate1 = None
    next_check = 0
    checks = 0
    if fixed_len is not None and fixed_len <= 0:
        return PhaseResult(x, 0, "replay", hist)
    it = 0
    while True:
        it += 1
        z = P.apply_inv(v)
        u_top = matvec(A, z) - alpha * u_top
        u_bot = delta * z - alpha * u_bot
        beta = math.sqrt(float(u_top @ u_top + u_bot @ u_bot))
        if beta > 0.0:
            u_top /= beta
            u_bot /= beta
        anorm2 += alpha * alpha + beta * beta
        v = P.apply_inv_T(rmatvec(A, u_top) + delta * u_bot) - beta * v
        alpha = math.sqrt(float(v @ v))
        if alpha > 0.0:
            v /= alpha
        rho = math.sqrt(rhobar * rhobar + beta * beta)
        c = rhobar / rho
        s = beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar_prev = phibar
        phibar = s * phibar
        x += (phi / rho) * P.apply_inv(w)
        w = v - (theta / rho) * w
        hist.append(phibar)
        if it == 1:
            rate1 = math.log(phibar_prev / phibar) if phibar > 0 else math.inf
        if fixed_len is not None:
            if it >= fixed_len:
                return PhaseResult(x, it, "replay", hist)
            continue
        if beta == 0.0 or alpha == 0.0:
            return PhaseResult(x, it, "exact", hist, checks)
        if alpha * abs(c) <= eps_lsqr * math.sqrt(anorm2):
            return PhaseResult(x, it, "ps_test2", hist, checks)
        if phibar <= eps_lsqr * beta1:
            return PhaseResult(x, it, "ps_test1", hist, checks)
        if dynamic_stop(phibar_prev, phibar, rate1, nu, P.sig_ell):
            return PhaseResult(x, it, "dynamic", hist, checks)
        if tol > 0.0 and it >= next_check:
            est = P.norm * phibar * alpha * abs(c) / norm_Atb
            if est <= tol:
                checks += 1
                if ne_residual(A, b, mu, x, norm_Atb) <= tol:
                    return PhaseResult(x, it, "tol", hist, checks)
                next_check = it + check_gap
        if it >= maxit:
            return PhaseResult(x, it, "maxit", hist, checks)


# --------------------------------------------------------------------------------------
# Driver: Algorithm "APLICUR: detailed implementation"
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Options:
    seed: int = 1
    eps_cur_factor: float = 30.0
    nu_prec: float = 10.0
    nu_lsqr: float = 100.0
    eps_lsqr: float = 1e-10
    xi: int = 8
    normest_r: int = 10
    check_gap: int = 10
    max_extra_phases: int = 8
    replay: dict | None = None       # {"phases": [...], "rebuild": [...]}
    # Section "Levels of adaptivity": rank-adaptive single-shot preconditioning builds the
    # preconditioner once, when rank growth ends, and runs a single phase (plus its warm
    # restarts); the default is fully adaptive
    single_shot: bool = False
    # > 0 caps the CUR rank: reaching it ends rank growth like reaching min(m, n) (the last
    # block is truncated to fit); with bsize = max_rank and single_shot the one rank step
    # is the fixed-rank single-shot variant (Algorithm "Sketched CUR with cross
    # approximation using LUPP", on the driver's sketch)
    max_rank: int = 0
    # "svd": Algorithm CURPreconditioner; "svdfree": the SVD-free preconditioner (Eq.
    # preconditioner_svdfree) with the target level sigma_min(M); for mu > 0 of a CUR of
    # A_mu = [A; delta I] (section "SVD-free variant", last paragraph)
    variant: str = "svd"
    # the delta stored in A_mu's appended rows (default sqrt(mu); an implementation that
    # keeps A_mu in FP32 stores sqrt(mu) rounded to FP32)
    cur_delta: float | None = None


class RebuildRule:
    """Part 3 of Algorithm "APLICUR: detailed implementation" (re-preconditioning
    criterion of Section "Adaptivity criteria"): rebuild the preconditioner when
    d_cur / (rho - eps_cur) >= nu_prec or rho <= eps_cur, where d_cur is the gap
    rho - eps_cur recorded at the previous rebuild (infinite before the first one).
    The gap is only updated when a rebuild happens."""

    def __init__(self, eps_cur: float, nu_prec: float):
        self.eps_cur = eps_cur
        self.nu_prec = nu_prec
        self.d_cur = math.inf

    def wants_rebuild(self, rho: float) -> bool:
        if rho <= self.eps_cur:
            return True
        return self.d_cur / (rho - self.eps_cur) >= self.nu_prec

    def rebuilt(self, rho: float) -> None:
        self.d_cur = rho - self.eps_cur


@dataclasses.dataclass
class Result:
    x: np.ndarray
    I: np.ndarray
    J: np.ndarray
    converged: bool
    iters: int
    ne_res: float
    rank_steps: list          # per step: dict(ell, rho, rebuild, margin)
    phases: list              # per phase: dict(ell, iters, reason, ne_res)
    Y: np.ndarray
    last_P: Preconditioner | None
    rank_breakdown: bool = False  # a rank step's new columns made C^T C singular


def aplicur(A, b, mu: float, bsize: int, opts: Options | None = None, *, tol=1e-10,
            maxit=100000, srows=None, signs=None, W=None, S=None) -> Result:
    """Adaptive CUR-preconditioned LSQR for min ||A x - b||^2 + mu ||x||^2."""
    opts = opts or Options()
    if _is_sparse(A):
        A = A.tocsr().astype(np.float64)
    else:
        A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, n = A.shape
    delta = math.sqrt(mu)
    eps_cur = opts.eps_cur_factor * delta
    s = sketch_rows(bsize)
    xi = sketch_xi(s, opts.xi)
    # the matrix of the CUR: A, or A_mu for the SVD-free variant of a regularised problem
    svdfree = opts.variant == "svdfree"
    CA = A
    if svdfree and mu > 0.0:
        CA = regularized_matrix(A, delta if opts.cur_delta is None else opts.cur_delta)
    cm = CA.shape[0]
    if srows is None:
        srows, signs = orng.sparse_sign(opts.seed, s, cm, xi)
    if W is None:
        W = orng.gaussian_w(opts.seed, n, opts.normest_r)
    norm_Atb = float(np.linalg.norm(rmatvec(A, b)))
    if norm_Atb == 0.0:
        return Result(np.zeros(n), np.zeros(0, np.int64), np.zeros(0, np.int64), True, 0, 0.0,
                      [], [], np.zeros((s, n)), None)

    # S: a dense sketching operator (s x m) in place of the sparse sign embedding
    Y = apply_sketch(CA, srows, signs, s) if S is None else dense_sketch(CA, S)
    I = np.zeros(0, np.int64)
    J = np.zeros(0, np.int64)
    core = None
    E_row = Y.copy()
    Q_R = T_R = None
    rule = RebuildRule(eps_cur, opts.nu_prec)
    x = np.zeros(n)
    steps, phases = [], []
    total = 0
    P = None
    replay = opts.replay
    rb_list = list(replay["rebuild"]) if replay else None
    ph_list = list(replay["phases"]) if replay else None

    def run_phase(P, nu, final):
        nonlocal x, total
        fixed = None
        if ph_list is not None:
            fixed = ph_list.pop(0) if ph_list else 0
        res = plsqr_phase(A, b, delta, x, P, eps_lsqr=opts.eps_lsqr, nu=nu,
                          maxit=max(0, maxit - total), tol=0.0 if replay else tol,
                          norm_Atb=norm_Atb, check_gap=opts.check_gap, fixed_len=fixed)
        x = res.x
        total += res.iters
        ne = ne_residual(A, b, mu, x, norm_Atb)
        phases.append(dict(ell=P.ell, iters=res.iters, reason=res.reason, ne_res=ne,
                           final=final))
        return ne

    def done(ne):
        return Result(x, I, J, ne <= tol, total, ne, steps, phases, Y, P, rank_breakdown)

    kmax = min(cm, n) if opts.max_rank <= 0 else min(cm, n, opts.max_rank)
    rank_breakdown = False
    Cn, T_C = cols(CA, J), None  # C = A(:, J) and its Cholesky factor at the current rank
    while True:
        # Part 1: update CUR
        kb = min(bsize, kmax - len(J))
        Ip, Jp, margin = augment_cur(CA, I, J, E_row, core, kb)
        if Ip.size:
            # new columns numerically dependent on the chosen ones (C^T C not positive
            # definite): rank growth ends at the current rank and the solve goes on with
            # the last preconditioner built
            Cn = cols(CA, np.concatenate([J, Jp]))
            try:
                T_C = chol_upper(Cn.T @ Cn)
            except np.linalg.LinAlgError:
                rank_breakdown = True
                break
        exhausted = Ip.size < kb
        I = np.concatenate([I, Ip])
        J = np.concatenate([J, Jp])
        core = Core(CA, I, J)
        E_row = sketched_residual(CA, Y, I, J, core)
        rho = norm_estimate(E_row, W)
        rho_eff = 0.0 if exhausted else rho
        last = rho_eff <= eps_cur or len(I) >= kmax or exhausted
        # Part 2: update factorisations of R^T
        if Ip.size:
            Q_R, T_R = augment_qr(Q_R, T_R, rows(CA, Ip).T)
        # Part 3: re-precondition and run LSQR
        if rb_list is not None:
            rebuild = bool(rb_list.pop(0)) if rb_list else last
        else:
            rebuild = last or (not opts.single_shot and rule.wants_rebuild(rho_eff))
        steps.append(dict(ell=len(I), rho=rho, rebuild=rebuild, margin=margin))
        if rebuild:
            C = Cn  # A(:, J) of this step, T_C its Cholesky factor
            if svdfree:
                P = build_svdfree_preconditioner(C, cross(CA, I, J), Q_R, T_R, 1.0, T_C)
                P.sighat = svdfree_smallest_sigma(P)
            else:
                P = build_preconditioner(C, core, Q_R, T_R, delta, T_C)
            nu = math.inf if last else opts.nu_lsqr
            ne = run_phase(P, nu, last)
            if not replay and ne <= tol:
                return done(ne)
            rule.rebuilt(rho_eff)
        if last:
            break
        if total >= maxit:
            return done(ne_residual(A, b, mu, x, norm_Atb))
    # final phase ended without reaching tol: warm-restart it with the same P
    if P is None:
        P = identity_preconditioner(n)
    ne = phases[-1]["ne_res"] if phases else ne_residual(A, b, mu, x, norm_Atb)
    extra = 0
    while (replay and ph_list) or (not replay and ne > tol and total < maxit
                                   and extra < opts.max_extra_phases):
        prev = ne
        ne = run_phase(P, math.inf, True)
        extra += 1
        if not replay and (phases[-1]["iters"] == 0 or ne > 0.5 * prev):
            break
    return done(ne)


def plain_lsqr(A, b, mu, *, tol=1e-10, maxit=100000, eps_lsqr=0.0, check_gap=10) -> Result:
    """Unpreconditioned LSQR on [A; delta I] (the comparison baseline), one phase."""
    if _is_sparse(A):
        A = A.tocsr().astype(np.float64)
    else:
        A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    delta = math.sqrt(mu)
    norm_Atb = float(np.linalg.norm(rmatvec(A, b)))
    P = identity_preconditioner(n)
    res = plsqr_phase(A, b, delta, np.zeros(n), P, eps_lsqr=eps_lsqr, maxit=maxit, tol=tol,
                      norm_Atb=norm_Atb, check_gap=check_gap)
    ne = ne_residual(A, b, mu, res.x, norm_Atb)
    return Result(res.x, np.zeros(0, np.int64), np.zeros(0, np.int64), ne <= tol, res.iters, ne,
                  [], [dict(ell=0, iters=res.iters, reason=res.reason, ne_res=ne, final=True)],
                  None, P)


# --------------------------------------------------------------------------------------
# Direct solves and the adjoint (plain definitions)
# --------------------------------------------------------------------------------------

def ridge_direct(A, b, mu: float) -> np.ndarray:
    """argmin ||A x - b||^2 + mu ||x||^2 by Householder QR of [A; sqrt(mu) I]."""
    Ad = A.toarray() if _is_sparse(A) else np.asarray(A, dtype=np.float64)
    m, n = Ad.shape
    delta = math.sqrt(mu)
    Aug = np.vstack([Ad, delta * np.eye(n)])
    rhs = np.concatenate([np.asarray(b, dtype=np.float64), np.zeros(n)])
    Q, R = np.linalg.qr(Aug, mode="reduced")
    return sla.solve_triangular(R, Q.T @ rhs, lower=False)


def ridge_sparse(A, b, mu: float, rtol: float = 1e-15):
    """The ridge solution (A^T A + mu I) x = A^T b of a sparse A by conjugate gradients on
    the normal equations with the Jacobi preconditioner diag(A^T A) + mu (scipy's cg),
    run until the normal-equation residual is rtol of ||A^T b||.  Returns (x, relative
    normal-equation residual); the relative error of x is at most that residual times
    cond(A^T A + mu I)."""
    import scipy.sparse.linalg as spla
    A = sp.csr_matrix(A, dtype=np.float64)
    n = A.shape[1]
    b = np.asarray(b, dtype=np.float64)
    d = np.asarray(A.multiply(A).sum(axis=0)).ravel() + mu
    op = spla.LinearOperator((n, n), matvec=lambda v: A.T @ (A @ v) + mu * v, dtype=np.float64)
    M = spla.LinearOperator((n, n), matvec=lambda v: v / d, dtype=np.float64)
    rhs = A.T @ b
    x, _ = spla.cg(op, rhs, M=M, rtol=rtol, atol=0.0, maxiter=100000)
    res = float(np.linalg.norm(A.T @ (b - A @ x) - mu * x) / np.linalg.norm(rhs))
    return np.asarray(x, dtype=np.float64), res


def ridge_gradients(A, b, mu: float, x: np.ndarray, g: np.ndarray):
    """Gradients of L(x(b, mu, A)) given g = dL/dx, where x solves (A^T A + mu I) x = A^T b:
    lambda = (A^T A + mu I)^{-1} g;  dL/db = A lambda;  dL/dmu = -lambda^T x;
    dL/dA = r lambda^T - (A lambda) x^T with r = b - A x.
    lambda is computed as argmin ||[A; delta I] lambda - [0; g/delta]|| by QR."""
    Ad = A.toarray() if _is_sparse(A) else np.asarray(A, dtype=np.float64)
    m, n = Ad.shape
    delta = math.sqrt(mu)
    Aug = np.vstack([Ad, delta * np.eye(n)])
    rhs = np.concatenate([np.zeros(m), g / delta])
    Q, R = np.linalg.qr(Aug, mode="reduced")
    lam = sla.solve_triangular(R, Q.T @ rhs, lower=False)
    Al = Ad @ lam
    r = np.asarray(b, dtype=np.float64) - Ad @ x
    return lam, Al, -float(lam @ x), np.outer(r, lam) - np.outer(Al, x)


class RidgeQR:
    """Householder QR of [A; sqrt(mu) I] in FP64, kept for several right-hand sides:
    solve(top, bot) = argmin ||[A; sqrt(mu) I] x - [top; bot]|| by the same definition as
    ridge_direct, without refactoring for each right-hand side (finite differences in b
    and the adjoint solve of ridge_gradients reuse one factorisation)."""

    def __init__(self, A, mu: float):
        Ad = A.toarray() if _is_sparse(A) else np.asarray(A, dtype=np.float64)
        self.m, self.n = Ad.shape
        self.delta = math.sqrt(mu)
        Aug = np.vstack([Ad, self.delta * np.eye(self.n)])
        self.Q, self.R = np.linalg.qr(Aug, mode="reduced")

    def solve(self, top, bot=None):
        rhs = self.Q[:self.m].T @ np.asarray(top, dtype=np.float64)
        if bot is not None:
            rhs = rhs + self.Q[self.m:].T @ np.asarray(bot, dtype=np.float64)
        return sla.solve_triangular(self.R, rhs, lower=False)


def grad_A_entries(A, b, x, lam, rows, cols):
    """Entries (rows[k], cols[k]) of dL/dA = r lambda^T - (A lambda) x^T, r = b - A x,
    without forming the m x n matrix."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    r = np.asarray(b, dtype=np.float64) - matvec(A, x)
    Al = matvec(A, lam)
    return r[rows] * lam[cols] - Al[rows] * x[cols]


class RidgeReduced:
    """The ridge problem of a tall dense A reduced by one Householder QR A = Q_A R_A:
    ||A x - b||^2 + mu ||x||^2 = ||R_A x - Q_A^T b||^2 + mu ||x||^2 + ||(I - Q_A Q_A^T) b||^2,
    so x_mu = argmin ||[R_A; sqrt(mu) I] x - [Q_A^T b; 0]|| is a 2n x n least-squares
    problem per mu (Householder QR), for any number of mu values and right-hand sides.
    A rank-1 change A + h u v^T stays exactly reduced with one more orthonormal column:
    u = Q_A w + u_perp gives A + h u v^T = [Q_A, q] [R_A + h w v^T; h ||u_perp|| v^T] with
    q = u_perp / ||u_perp||, and b enters through [Q_A^T b; q^T b] (finite differences in A
    without refactoring A)."""

    def __init__(self, A):
        self.A = np.asarray(A, dtype=np.float64)
        self.Q, self.R = np.linalg.qr(self.A, mode="reduced")
        self.n = self.A.shape[1]
        self._fact = {}  # mu -> QR of [R_A; sqrt(mu) I] (the unchanged A)

    def _factor(self, M, mu, key):
        if key is not None and key in self._fact:
            return self._fact[key]
        f = np.linalg.qr(np.vstack([M, math.sqrt(mu) * np.eye(self.n)]), mode="reduced")
        if key is not None:
            self._fact = {key: f}
        return f

    def _reduced(self, b, du=None, dv=None, h=0.0):
        cb = self.Q.T @ np.asarray(b, dtype=np.float64)
        if du is None or h == 0.0:
            return self.R, cb
        w = self.Q.T @ du
        up = du - self.Q @ w
        nu = float(np.linalg.norm(up))
        M = self.R + h * np.outer(w, dv)
        if nu == 0.0:
            return M, cb
        M = np.vstack([M, h * nu * np.asarray(dv, dtype=np.float64)[None, :]])
        return M, np.concatenate([cb, [float(up @ b) / nu]])

    def solve(self, b, mu, du=None, dv=None, h=0.0):
        """argmin ||(A + h du dv^T) x - b||^2 + mu ||x||^2."""
        M, rhs = self._reduced(b, du, dv, h)
        Qa, Ra = self._factor(M, mu, mu if (du is None or h == 0.0) else None)
        return sla.solve_triangular(Ra, Qa.T @ np.concatenate([rhs, np.zeros(self.n)]),
                                    lower=False)

    def adjoint(self, mu, g):
        """lambda = (A^T A + mu I)^{-1} g as argmin ||[R_A; sqrt(mu) I] l - [0; g / sqrt(mu)]||
        (the Q_A^T part of the right-hand side [0; g / sqrt(mu)] is zero)."""
        delta = math.sqrt(mu)
        Qa, Ra = self._factor(self.R, mu, mu)
        rhs = np.concatenate([np.zeros(self.n), np.asarray(g, dtype=np.float64) / delta])
        return sla.solve_triangular(Ra, Qa.T @ rhs, lower=False)
