"""Dense sketching operators (appendix "Sketch comparison"): the Gaussian embedding and the
subsampled randomized Hadamard transform, in place of the sparse sign embedding.

  - The library draws S itself from the project generator (streams 4-6); its Y = S A must
    match the oracle's FP64 product with the oracle's own draw of S, entry by entry within
    the rounding of an FP64 (or compensated FP32) product of length m:
    |Y - Y_o| <= 1e-12 (|S| |A|).
  - With the oracle's phase schedule replayed, the CUR indices are the oracle's and the
    solution agrees to 1e-10.
  - The tensor-core path rounds S to bfloat16, represents A by 1 to 3 terms of its
    bfloat16 expansion (k terms: k products per entry of A) and accumulates in FP32.  Its
    Y is compared with the oracle's FP64 product of the same rounded operands; the gap is
    the FP32 accumulation alone, bounded entry by entry by (k m + 32) 2^-22 (|S~| sum_j
    |A_j|) (one relative error of at most 2^-22 per addition, for any order of the k m
    additions and for an accumulator that truncates).  The CUR built from it is a different, equally valid
    sketch: the solve must converge to the same minimiser; index agreement with the FP64
    sketch is reported, not gated."""
import math

import numpy as np
import pytest

from oracle import aplicur_oracle as O
from oracle import rng as orng
from paper_2604_05065_gb300 import workloads as wl

from gpu_helpers import oracle_matrix, rel, schedule, to_device

pytestmark = pytest.mark.gpu

SEED = 777
KINDS = {"gaussian": 1, "srht": 2}


def _operator(kind, s, m):
    return orng.gaussian_sketch(SEED, s, m) if kind == "gaussian" else orng.srht_sketch(SEED, s, m)


def _problems():
    return {
        "dense64": wl.config1(scale=4),
        "dense32": wl.dense_lowrank(m=600, n=120, mu=1e-4, sketch_dim=8, index=60,
                                    dtype=np.float32, name="dense32"),
        "sparse64": wl.small_sparse(3000, 300, wl.BASE_SEED + 50, nnz_per_col=6, mu=1e-5,
                                    sketch_dim=10),
        "sparse32": wl.small_sparse(2500, 250, wl.BASE_SEED + 51, nnz_per_col=5, mu=1e-5,
                                    sketch_dim=10, dtype=np.float32),
    }


PROBS = _problems()


def _solver(p, kind, tc=0, **kw):
    import paper_2604_05065_gb300 as pkg
    A, b = to_device(p)
    return pkg.Solver(A, b, p.mu, p.sketch_dim, seed=SEED, sketch_kind=KINDS[kind],
                      sketch_tc=int(tc), **kw)


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("name", list(PROBS))
def test_dense_operator_sketch_matches_oracle(kind, name):
    p = PROBS[name]
    A = oracle_matrix(p)
    s_rows = O.sketch_rows(p.sketch_dim)
    S = _operator(kind, s_rows, p.m)
    Yo = O.dense_sketch(A, S)
    bound = 1e-12 * O.dense_sketch(abs(A), np.abs(S))
    Y = _solver(p, kind).sketch().cpu().numpy()
    assert Y.shape == Yo.shape
    assert np.all(np.abs(Y - Yo) <= bound + 1e-300), float(np.max(np.abs(Y - Yo) / (bound + 1e-300)))


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("name", ["dense64", "sparse64"])
def test_dense_operator_replay_matches_oracle(kind, name):
    p = PROBS[name]
    A = oracle_matrix(p)
    S = _operator(kind, O.sketch_rows(p.sketch_dim), p.m)
    ref = O.aplicur(A, p.b, p.mu, p.sketch_dim, O.Options(seed=SEED), tol=1e-10, S=S)
    s = _solver(p, kind, replay=schedule(ref))
    x = s.solve(1e-10).cpu().numpy()
    I, J = s.indices()
    assert np.array_equal(I, ref.I) and np.array_equal(J, ref.J)
    assert rel(x, ref.x) <= 1e-10
    assert [q["iters"] for q in s.phases()] == [q["iters"] for q in ref.phases]


# shapes for the tensor-core product: ragged tiles in both dimensions, s across the one-MMA
# (s <= 256) and two-MMA ranges, the largest s (512) and both value types
TC_CASES = {
    "f32_600x120_s9": lambda: wl.dense_lowrank(m=600, n=120, mu=1e-4, sketch_dim=8, index=60,
                                               dtype=np.float32, name="a"),
    "f64_1000x300_s275": lambda: wl.small_dense(1000, 300, 910, decay=3.0, mu=1e-4,
                                                sketch_dim=250),
    "f32_1111x520_s512": lambda: wl.dense_lowrank(m=1111, n=520, mu=1e-4, sketch_dim=465,
                                                  index=61, dtype=np.float32, name="c"),
    "f32_70x70_s17": lambda: wl.dense_lowrank(m=70, n=70, mu=1e-4, sketch_dim=16, index=62,
                                              dtype=np.float32, name="d"),
}


def _tc_check(Y, A, S, terms, what):
    St = orng.round_bf16(S)
    pieces = orng.bf16_pieces(A, terms)
    At = sum(pieces)
    Yt = St @ At
    m = A.shape[0]
    scale = np.abs(St) @ sum(np.abs(q) for q in pieces)
    bound = (terms * m + 32) * 2.0 ** -22 * scale
    err = np.abs(Y - Yt)
    assert np.all(err <= bound), (what, float(np.max(err / bound)))
    typ = float(np.median(err / np.maximum(scale, 1e-300)))
    print(f"{what}: max err / bound {float(np.max(err / bound)):.2e}, median "
          f"err / (|S~||A~|) {typ:.1e}", flush=True)


@pytest.mark.parametrize("terms", [1, 2, 3])
@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("case", list(TC_CASES))
def test_tensor_core_sketch_within_fp32_accumulation_bound(kind, case, terms):
    p = TC_CASES[case]()
    A = np.asarray(p.dense, dtype=np.float64)
    S = _operator(kind, O.sketch_rows(p.sketch_dim), p.m)
    Y = _solver(p, kind, tc=terms).sketch().cpu().numpy()
    assert Y.shape == (S.shape[0], p.n)
    _tc_check(Y, A, S, terms, f"{case}/{kind}/{terms} terms")


@pytest.mark.parametrize("dtype,n,ld", [(np.float32, 130, 136), (np.float64, 77, 81),
                                         (np.float32, 200, 203)])
def test_tensor_core_sketch_strided_rows(dtype, n, ld):
    """A as a view with row stride ld > n: 16-byte row loads with a ragged last group of
    columns (FP32, ld % 4 == 0), and the element-wise load path for rows that are not
    16-byte aligned (FP64 with odd ld, FP32 with ld % 4 != 0)."""
    import torch

    import paper_2604_05065_gb300 as pkg
    m = 900
    g = np.random.default_rng(n)
    full = g.standard_normal((m, ld)).astype(dtype)
    A = full[:, :n]
    b = g.standard_normal(m)
    At = torch.from_numpy(full).cuda()[:, :n]
    assert At.stride(0) == ld
    S = _operator("gaussian", O.sketch_rows(20), m)
    for terms in (1, 3):
        sv = pkg.Solver(At, torch.from_numpy(b).cuda(), 1e-4, 20, seed=SEED,
                        sketch_kind=KINDS["gaussian"], sketch_tc=terms)
        Y = sv.sketch().cpu().numpy()
        _tc_check(Y, np.asarray(A, dtype=np.float64), S, terms,
                  f"{np.dtype(dtype).name} n={n} ld={ld}/{terms} terms")


@pytest.mark.parametrize("terms", [1, 2, 3])
@pytest.mark.parametrize("kind", list(KINDS))
def test_tensor_core_sketch_solve_converges(kind, terms):
    p = PROBS["dense32"]
    A = oracle_matrix(p)
    acc = _solver(p, kind)
    xa = acc.solve(1e-10).cpu().numpy()
    tc = _solver(p, kind, tc=terms)
    x = tc.solve(1e-10).cpu().numpy()
    st = tc.stats()
    assert st["converged"] == 1 and st["ne_res"] <= 1e-10
    xd = O.ridge_direct(A, p.b, p.mu)
    kappa = 1.0 / math.sqrt(p.mu)
    assert rel(x, xd) <= max(1e-10, 10 * kappa * 1e-10)
    assert rel(xa, xd) <= max(1e-10, 10 * kappa * 1e-10)
    Ia, _ = acc.indices()
    It, _ = tc.indices()
    common = len(set(Ia.tolist()) & set(It.tolist()))
    print(f"{kind}/{terms} terms: tensor-core CUR rank {len(It)}, FP64-sketch rank {len(Ia)}, "
          f"{common} row indices in common", flush=True)


def test_option_checks():
    import paper_2604_05065_gb300 as pkg
    d = PROBS["dense32"]
    sp = PROBS["sparse64"]
    with pytest.raises(pkg.AplicurError) as e:     # the sparse sign embedding has no TC form
        A, b = to_device(d)
        pkg.Solver(A, b, d.mu, d.sketch_dim, sketch_tc=1)
    assert e.value.status == 1
    with pytest.raises(pkg.AplicurError) as e:     # CSR A
        _solver(sp, "gaussian", tc=True)
    assert e.value.status == 1
    with pytest.raises(pkg.AplicurError) as e:
        A, b = to_device(d)
        pkg.Solver(A, b, d.mu, d.sketch_dim, sketch_kind=3)
    assert e.value.status == 1
    big = TC_CASES["f32_1111x520_s512"]()
    with pytest.raises(pkg.AplicurError) as e:     # s = 517 > 512
        A, b = to_device(big)
        pkg.Solver(A, b, big.mu, 470, sketch_kind=1, sketch_tc=1)
    assert e.value.status == 1


def test_tensor_core_sketch_full_size_rbf():
    """The 20000 x 20000 FP32 RBF kernel matrix with sketch dimension 250 (s = 275): the
    tensor-core Gaussian sketch with 1, 2 and 3 bfloat16 terms of A at 64 sampled columns
    against the oracle's product of the rounded operands; the solves from them against the
    solve from the compensated-FP32 sketch.  The sketch error is far above the FP64 one
    here, and the rank search may select columns that are numerically dependent on the
    chosen ones: rank growth then ends (stats rank_breakdown) and the solve finishes with
    the last preconditioner built; it must still reach the tolerance."""
    import torch
    p = wl.config3()
    S = orng.gaussian_sketch(SEED, O.sketch_rows(p.sketch_dim), p.m)
    cols = np.random.default_rng(20260406).choice(p.n, 64, replace=False)
    Ac = np.asarray(p.dense[:, cols], dtype=np.float64)
    acc = _solver(p, "gaussian", precision=1)
    xa = acc.solve(1e-12).cpu().numpy()
    sa = acc.stats()
    assert sa["converged"] == 1
    Ia, _ = acc.indices()
    line = [f"compensated FP32 {sa['time_setup_ms']:.2f} ms, CUR rank {len(Ia)}, "
            f"{sa['iters']} iterations"]
    for terms in (1, 2, 3):
        tc = _solver(p, "gaussian", tc=terms, precision=1)
        Y = tc.sketch().cpu().numpy()
        _tc_check(Y[:, cols], Ac, S, terms, f"rbf20000/gaussian/{terms} terms")
        setup = tc.stats()["time_setup_ms"]
        x = tc.solve(1e-12).cpu().numpy()
        st = tc.stats()
        assert st["converged"] == 1
        # the same problem to the same normal-equation tolerance (the FP32-product solves
        # of this workload reach about 1e-8 of the FP64 minimiser here)
        assert rel(x, xa) <= 1e-6
        It, _ = tc.indices()
        common = len(set(Ia.tolist()) & set(It.tolist()))
        line.append(f"{terms} terms {setup:.2f} ms, CUR rank {len(It)} (breakdown "
                    f"{st['rank_breakdown']}), {common} row indices in common, "
                    f"{st['iters']} iterations")
        del tc
    print("rbf20000 sketch: " + "; ".join(line), flush=True)
    del acc
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kind", list(KINDS))
def test_dense_operator_on_the_regularized_matrix(kind):
    """SVD-free variant with mu > 0: the dense operator has m + n columns (it sketches
    A_mu = [A; sqrt(mu) I]); replaying the oracle's schedule gives its indices."""
    p = PROBS["dense64"]
    A = oracle_matrix(p)
    cm = p.m + p.n
    S = _operator(kind, O.sketch_rows(p.sketch_dim), cm)
    ref = O.aplicur(A, p.b, p.mu, p.sketch_dim, O.Options(seed=SEED, variant="svdfree"),
                    tol=1e-10, S=S)
    s = _solver(p, kind, variant=1, replay=schedule(ref))
    Y = s.sketch().cpu().numpy()
    Am = O.regularized_matrix(A, math.sqrt(p.mu))
    Yo = O.dense_sketch(Am, S)
    assert np.all(np.abs(Y - Yo) <= 1e-12 * O.dense_sketch(abs(Am), np.abs(S)) + 1e-300)
    s.solve(1e-10)
    I, J = s.indices()
    assert np.array_equal(I, ref.I) and np.array_equal(J, ref.J)
