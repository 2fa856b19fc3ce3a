"""The adjoint workload at full size: dense FP32 A of 100000 x 2000 with singular values
exp(-i/200), loss 0.5 ||x(b, mu, A) - x_target||^2, forward and backward through
APLICURSolve (torch.autograd.Function over aplicur_solve / aplicur_backward) for every mu
of the sweep 1e-8 ... 1e-1.

References, all FP64 on the CPU from the oracle's QR-reduced ridge problem (one
Householder QR of the rounded A, then a 2n x n QR per mu or per rank-1 change of A):
  - the solution and the closed-form gradients (db = A lambda, dmu = -lambda^T x,
    dA = r lambda^T - (A lambda) x^T at 64 sampled entries), at every mu;
  - central finite differences with step 1e-6 (relative in mu): in mu at every mu; along
    seeded unit directions of b and seeded rank-1 unit directions u v^T of A (one at every
    mu, three at mu = 1e-8 and 1e-4); at 8 sampled entries of A at mu = 1e-4.
Gate: 1e-5 relative (the FP32-storage gate) for the solution and the closed-form
gradients.  A finite difference carries its own error: the rounding of the two FP64 loss
values divided by the step, which at mu = 1e-8 (kappa of [A; sqrt(mu) I] near 1e4) reaches
about 1e-5 of the derivative along b and A.  Each difference along b or A is therefore
taken with steps h and 2h; their disagreement estimates that error, and the gradient must
agree with the difference within max(1e-5 |fd|, 3 |fd_h - fd_2h|)."""
import math

import numpy as np
import pytest

from oracle import aplicur_oracle as O
from paper_2604_05065_gb300 import workloads as wl

from gpu_helpers import rel

pytestmark = pytest.mark.gpu

MUS = [1e-8, 1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1]
H = 1e-6


def _loss(x, xt):
    return 0.5 * float(np.sum((x - xt) ** 2))


def test_adjoint_full_size_mu_sweep_against_oracle_and_finite_differences():
    import torch

    import paper_2604_05065_gb300 as pkg
    p = wl.config5()
    A32 = p.dense
    A64 = A32.astype(np.float64)
    b, xt = p.b, p.extra["x_target"]
    m, n = A64.shape
    red = O.RidgeReduced(A64)
    g = np.random.default_rng(20260405)
    dbs = [d / np.linalg.norm(d) for d in g.standard_normal((3, m))]
    dAs = []
    for _ in range(3):
        u, v = g.standard_normal(m), g.standard_normal(n)
        dAs.append((u / np.linalg.norm(u), v / np.linalg.norm(v)))  # ||u v^T||_F = 1
    ri = g.choice(m, 64, replace=False)
    cj = g.choice(n, 64, replace=False)
    fn = pkg.aplicur_solve_fn()
    Ad = torch.from_numpy(A32).cuda()
    bd = torch.from_numpy(b).cuda()
    xtd = torch.from_numpy(xt).cuda()
    for mu in MUS:
        A_ = Ad.clone().requires_grad_(True)
        b_ = bd.clone().requires_grad_(True)
        mu_ = torch.tensor(mu, dtype=torch.float64, device="cuda", requires_grad=True)
        x = fn.apply(A_, b_, mu_, p.sketch_dim, 1e-12, 200000, {"precision": pkg.PREC_DF32})
        loss = 0.5 * ((x - xtd) ** 2).sum()
        loss.backward()
        xg = x.detach().cpu().numpy()
        gb = b_.grad.cpu().numpy()
        gmu = float(mu_.grad)
        # oracle: solution and closed-form gradients
        xo = red.solve(b, mu)
        lam = red.adjoint(mu, xo - xt)
        gb_o = A64 @ lam
        gmu_o = -float(lam @ xo)
        gA_o = O.grad_A_entries(A64, b, xo, lam, ri, cj)
        gA = A_.grad[torch.from_numpy(ri).cuda(), torch.from_numpy(cj).cuda()].double().cpu().numpy()
        errs = {"x": rel(xg, xo), "db": rel(gb, gb_o), "dmu": abs(gmu - gmu_o) / abs(gmu_o),
                "dA64": rel(gA, gA_o)}
        # central differences of the FP64 loss
        fd_mu = (_loss(red.solve(b, mu * (1 + H)), xt) - _loss(red.solve(b, mu * (1 - H)), xt)) \
            / (2 * H * mu)
        errs["fd_mu"] = abs(gmu - fd_mu) / abs(fd_mu)
        for k, v in errs.items():
            assert v <= 1e-5, (mu, k, v)
        # directional differences with steps h and 2h: the ratio is the gradient's error
        # over the allowed one, max(1e-5 |fd|, 3 |fd_h - fd_2h|), and must be <= 1
        ratios = {}

        def check(name, grad, f):
            fd1 = (f(H) - f(-H)) / (2 * H)
            fd2 = (f(2 * H) - f(-2 * H)) / (4 * H)
            allowed = max(1e-5 * abs(fd1), 3.0 * abs(fd1 - fd2))
            ratios[name] = abs(grad - fd1) / allowed
            errs[name] = abs(grad - fd1) / max(abs(fd1), 1e-300)

        nd = 3 if mu in (1e-8, 1e-4) else 1
        for k, d in enumerate(dbs[:nd]):
            check(f"fd_b{k}", float(gb @ d), lambda h, d=d: _loss(red.solve(b + h * d, mu), xt))
        gAd = A_.grad.double()
        for k, (u, v) in enumerate(dAs[:nd]):
            dirv = float(torch.from_numpy(u).cuda() @ (gAd @ torch.from_numpy(v).cuda()))
            check(f"fd_A{k}", dirv, lambda h, u=u, v=v: _loss(red.solve(b, mu, u, v, h), xt))
        if mu == 1e-4:
            for k in range(8):
                e_i = np.zeros(m)
                e_i[ri[k]] = 1.0
                e_j = np.zeros(n)
                e_j[cj[k]] = 1.0
                check(f"fd_A[{ri[k]},{cj[k]}]", float(gA[k]),
                      lambda h, e_i=e_i, e_j=e_j: _loss(red.solve(b, mu, e_i, e_j, h), xt))
        print(f"mu={mu:.0e} " + " ".join(f"{k}={v:.1e}" for k, v in errs.items())
              + " | fd error/allowed max " + f"{max(ratios.values()):.2f}", flush=True)
        for k, v in ratios.items():
            assert v <= 1.0, (mu, k, errs[k])
        del A_, b_, x, loss, gAd
        torch.cuda.empty_cache()
