"""The fused dense A pass (one read of A per LSQR iteration: u' = A z - alpha u and the
column partial sums of A^T u' from the same row tiles, thread-block clusters over column
panels) against the two-pass form and against the oracle.

Shapes span several clusters, column panels and row tiles, with ragged last tiles and
panels and a padded leading dimension.  Tolerances: compensated FP32 products (DF32)
against the FP64 oracle on the same rounded matrix at 1e-10 (early iterates of a
well-conditioned problem) and the two forms against each other at 1e-12; FP32 products
(MIXED) against each other at 1e-5."""
import math

import numpy as np
import pytest

from oracle import aplicur_oracle as O
from paper_2604_05065_gb300 import workloads as wl

from gpu_helpers import draws, rel, schedule

pytestmark = pytest.mark.gpu

# (m, n, ld): one panel with many row tiles; two panels (n = 6500 needs more than six
# float4 columns per thread in one panel) with a ragged last panel; padded rows; a tall
# problem with many clusters
SHAPES = [(3001, 516, 516), (13001, 6500, 6500), (2777, 1000, 1004), (20000, 2000, 2000)]


def _problem(m, n, ld, seed):
    g = np.random.default_rng(seed)
    # well conditioned (m >= 2n): singular values of a Gaussian matrix / sqrt(m) lie near
    # [1 - sqrt(n/m), 1 + sqrt(n/m)]
    A = (g.standard_normal((m, n)) / math.sqrt(m)).astype(np.float32)
    Ap = np.zeros((m, ld), np.float32)
    Ap[:, :n] = A
    b = g.standard_normal(m)
    return Ap, A.astype(np.float64), b


def _solver(Ap, n, b, mu, **kw):
    import torch

    import paper_2604_05065_gb300 as pkg
    At = torch.from_numpy(Ap).cuda()[:, :n]
    return pkg.Solver(At, torch.from_numpy(b).cuda(), mu, 4, **kw)


@pytest.mark.parametrize("m,n,ld", SHAPES)
def test_fused_plain_iterates_match_oracle_and_two_pass(m, n, ld):
    import paper_2604_05065_gb300 as pkg
    Ap, A64, b = _problem(m, n, ld, 100 + m % 97)
    mu, k = 1e-2, 8
    ref = O.plsqr_phase(A64, b, math.sqrt(mu), np.zeros(n), O.identity_preconditioner(n),
                        eps_lsqr=0.0, maxit=k)
    s1 = _solver(Ap, n, b, mu, precision=pkg.PREC_DF32, dense_pass=2)
    s2 = _solver(Ap, n, b, mu, precision=pkg.PREC_DF32, dense_pass=1)
    assert s1.stats()["fused_pass"] == 1 and s2.stats()["fused_pass"] == 0
    x1 = s1.plain_lsqr(0.0, k).cpu().numpy()
    x2 = s2.plain_lsqr(0.0, k).cpu().numpy()
    assert s1.phases()[0]["iters"] == k
    assert rel(x1, ref.x) <= 1e-10
    assert rel(x1, x2) <= 1e-12


@pytest.mark.parametrize("m,n,ld", SHAPES[:2])
def test_fused_mixed_products_match_two_pass(m, n, ld):
    import paper_2604_05065_gb300 as pkg
    Ap, _, b = _problem(m, n, ld, 200 + m % 89)
    mu, k = 1e-2, 6
    s1 = _solver(Ap, n, b, mu, precision=pkg.PREC_MIXED)  # fused by default
    s2 = _solver(Ap, n, b, mu, precision=pkg.PREC_MIXED, dense_pass=1)
    x1 = s1.plain_lsqr(0.0, k).cpu().numpy()
    x2 = s2.plain_lsqr(0.0, k).cpu().numpy()
    assert s1.stats()["fused_pass"] == 1 and s2.stats()["fused_pass"] == 0
    assert rel(x1, x2) <= 1e-5


def test_fused_preconditioned_replay_matches_oracle():
    """A full APLICUR solve in replay mode through the fused pass: CUR indices bit-exact,
    solution within 1e-10 of the oracle on the same rounded matrix."""
    import torch

    import paper_2604_05065_gb300 as pkg
    p = wl.dense_lowrank(m=2400, n=360, mu=1e-4, sketch_dim=12, index=61, dtype=np.float32,
                         name="dense32_fused")
    rows, signs, W = draws(p)
    A64 = np.asarray(p.dense, dtype=np.float64)
    ref = O.aplicur(A64, p.b, p.mu, p.sketch_dim, tol=1e-10, srows=rows, signs=signs, W=W)
    A = torch.from_numpy(np.ascontiguousarray(p.dense)).cuda()
    s = pkg.Solver(A, torch.from_numpy(p.b).cuda(), p.mu, p.sketch_dim, sketch_rows=rows,
                   sketch_signs=signs, normest_w=W, precision=pkg.PREC_DF32, dense_pass=2,
                   replay=schedule(ref))
    assert s.stats()["fused_pass"] == 1
    x = s.solve(1e-10).cpu().numpy()
    I, J = s.indices()
    assert np.array_equal(I, ref.I) and np.array_equal(J, ref.J)
    assert rel(x, ref.x) <= 1e-10


def test_fused_pass_not_used_when_rows_are_unaligned():
    """n not a multiple of 4: the rows are not 16-byte aligned for bulk copies, so the
    two-pass form runs (and still matches the oracle)."""
    import paper_2604_05065_gb300 as pkg
    Ap, A64, b = _problem(1000, 203, 203, 7)
    s = _solver(Ap, 203, b, 1e-2, precision=pkg.PREC_DF32, dense_pass=2)
    assert s.stats()["fused_pass"] == 0
    ref = O.plsqr_phase(A64, b, 0.1, np.zeros(203), O.identity_preconditioner(203),
                        eps_lsqr=0.0, maxit=5)
    assert rel(s.plain_lsqr(0.0, 5).cpu().numpy(), ref.x) <= 1e-10
