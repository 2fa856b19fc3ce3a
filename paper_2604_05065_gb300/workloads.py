"""Seeded synthetic inputs for the regularized least-squares workloads.

This module only draws problem data (A, b, targets).  It holds none of the
solver's arithmetic, so both the CPU oracle and the CUDA path can take their
inputs from it.  Every generator is driven by a numpy PCG64 stream seeded with
``20260403 + config_index``; ``scale`` shrinks m and n by the same factor for
test-sized variants with the same structure.

Workloads (dimensions at scale=1):
  1  dense FP64 2000x200, A = U diag(s) V^T with U, V from QR of N(0,1),
     s_i = 10^(-6 i/(n-1)); b = A x_true + 1e-3 N(0,1); mu = 1e-4; sketch dim 20.
     Test-matrix construction of Section 6.3 (dense synthetic dataset).
  2  sparse CSR 200000x20000, 10 nonzeros per column at uniform distinct rows,
     N(0,1) values, column j scaled by 10^(-6 j/(n-1)); b ~ N(0,1); mu = 1e-6;
     sketch dim 100.  Stands in for the sparse sets of Section 8.4.
  3  dense RBF kernel 20000x20000 over uniform points in [0,1]^8,
     A_ij = exp(-|p_i - p_j|^2 / 2) stored FP32; b = A w + 1e-2 N(0,1);
     mu = 1e-3; sketch dim 250.
  5  dense FP32 100000x2000 with singular values exp(-i/200); b ~ N(0,1);
     x_target ~ N(0,1); sketch dim 100 (gradient workload).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20260403


@dataclasses.dataclass
class Problem:
    name: str
    m: int
    n: int
    fmt: str                       # "dense" (row-major) or "csr"
    dtype: np.dtype                # storage dtype of A's values
    mu: float
    sketch_dim: int
    b: np.ndarray                  # float64, shape (m,) or (m, nrhs)
    dense: np.ndarray | None = None        # (m, n) row-major
    indptr: np.ndarray | None = None       # int32 (m+1,)
    indices: np.ndarray | None = None      # int32 (nnz,)
    data: np.ndarray | None = None         # values (nnz,)
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1]) if self.fmt == "csr" else self.m * self.n

    def to_dense64(self) -> np.ndarray:
        """A as a dense float64 array (values promoted exactly)."""
        if self.fmt == "dense":
            return np.asarray(self.dense, dtype=np.float64)
        out = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.indptr))
        out[rows, self.indices] = self.data.astype(np.float64)
        return out

    def to_scipy(self):
        """A as scipy.sparse.csr_matrix with float64 values (csr only)."""
        import scipy.sparse as sp
        return sp.csr_matrix((self.data.astype(np.float64), self.indices, self.indptr),
                             shape=(self.m, self.n))


def _rng(index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + index))


def _orth(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((rows, cols)))
    return q * np.sign(np.diag(r))


def dense_lowrank(m=2000, n=200, mu=1e-4, sketch_dim=20, noise=1e-3, index=1,
                  decay="log6", dtype=np.float64, name="dense_fp64") -> Problem:
    """A = U diag(s) V^T, b = A x_true + noise * N(0,1)."""
    rng = _rng(index)
    U = _orth(rng, m, n)
    V = _orth(rng, n, n)
    i = np.arange(n)
    if decay == "log6":
        s = 10.0 ** (-6.0 * i / max(n - 1, 1))
    elif decay == "exp200":
        s = np.exp(-i / 200.0)
    else:
        raise ValueError(decay)
    A = (U * s) @ V.T
    A = np.ascontiguousarray(A.astype(dtype))
    x_true = rng.standard_normal(n)
    b = A.astype(np.float64) @ x_true + noise * rng.standard_normal(m)
    return Problem(name, m, n, "dense", np.dtype(dtype), mu, sketch_dim, b, dense=A,
                   extra={"x_true": x_true, "sigma": s})


def config1(scale: int = 1) -> Problem:
    return dense_lowrank(m=2000 // scale, n=200 // scale, mu=1e-4, sketch_dim=max(20 // scale, 2),
                         index=1, name=f"dense_fp64_{2000 // scale}x{200 // scale}")


def sparse_colscaled(m=200000, n=20000, nnz_per_col=10, mu=1e-6, sketch_dim=100, index=2,
                     dtype=np.float64, name=None, col_decay=6.0) -> Problem:
    """Each column holds nnz_per_col N(0,1) values at distinct uniform rows; column j is
    scaled by 10^(-col_decay j/(n-1)); b ~ N(0,1)."""
    rng = _rng(index)
    k = nnz_per_col
    rows = rng.integers(0, m, size=(n, k))
    # redraw duplicate rows inside a column until all k rows are distinct
    while True:
        srt = np.sort(rows, axis=1)
        dup = np.any(srt[:, 1:] == srt[:, :-1], axis=1)
        if not dup.any():
            break
        bad = np.nonzero(dup)[0]
        rows[bad] = rng.integers(0, m, size=(bad.size, k))
    vals = rng.standard_normal((n, k))
    colscale = 10.0 ** (-col_decay * np.arange(n) / max(n - 1, 1))
    vals = vals * colscale[:, None]
    cols = np.repeat(np.arange(n), k)
    rows = rows.reshape(-1)
    vals = vals.reshape(-1)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=indptr[1:])
    b = rng.standard_normal(m)
    nm = name or f"sparse_csr_{m}x{n}"
    return Problem(nm, m, n, "csr", np.dtype(dtype), mu, sketch_dim, b,
                   indptr=indptr.astype(np.int32), indices=cols.astype(np.int32),
                   data=np.ascontiguousarray(vals.astype(dtype)))


def config2(scale: int = 1, dtype=np.float64) -> Problem:
    return sparse_colscaled(m=200000 // scale, n=20000 // scale, mu=1e-6,
                            sketch_dim=100 if scale == 1 else max(100 // scale, 5),
                            index=2, dtype=dtype)


def rbf_kernel(npts=20000, dim=8, mu=1e-3, sketch_dim=250, index=3, chunk=2048) -> Problem:
    """Gaussian RBF kernel matrix over uniform points, stored FP32."""
    rng = _rng(index)
    p = rng.random((npts, dim))
    A = np.empty((npts, npts), dtype=np.float32)
    sq = np.sum(p * p, axis=1)
    for r0 in range(0, npts, chunk):
        r1 = min(npts, r0 + chunk)
        d2 = sq[r0:r1, None] + sq[None, :] - 2.0 * (p[r0:r1] @ p.T)
        np.maximum(d2, 0.0, out=d2)
        A[r0:r1] = np.exp(-0.5 * d2).astype(np.float32)
    w = rng.standard_normal(npts)
    b = np.empty(npts)
    for r0 in range(0, npts, chunk):
        r1 = min(npts, r0 + chunk)
        b[r0:r1] = A[r0:r1].astype(np.float64) @ w
    b += 1e-2 * rng.standard_normal(npts)
    return Problem(f"rbf_fp32_{npts}x{npts}", npts, npts, "dense", np.dtype(np.float32), mu,
                   sketch_dim, b, dense=A, extra={"points": p})


def config3(scale: int = 1) -> Problem:
    return rbf_kernel(npts=20000 // scale, sketch_dim=250 if scale == 1 else max(250 // scale, 5))


def config5(scale: int = 1, mu: float = 1e-4) -> Problem:
    m, n = 100000 // scale, 2000 // scale
    rng = _rng(5)
    U = _orth(rng, m, n)
    V = _orth(rng, n, n)
    s = np.exp(-np.arange(n) / 200.0)
    A = np.ascontiguousarray(((U * s) @ V.T).astype(np.float32))
    b = rng.standard_normal(m)
    x_target = rng.standard_normal(n)
    return Problem(f"adjoint_fp32_{m}x{n}", m, n, "dense", np.dtype(np.float32), mu,
                   max(100 // scale, 5), b, dense=A, extra={"x_target": x_target, "sigma": s})


def small_dense(m, n, seed, decay=6.0, mu=1e-4, sketch_dim=4, noise=1e-3, rank=None) -> Problem:
    """Small dense test problem; ``rank`` makes A exactly low rank."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = n if rank is None else rank
    U = _orth(rng, m, r)
    V = _orth(rng, n, r)
    s = 10.0 ** (-decay * np.arange(r) / max(n - 1, 1))
    A = np.ascontiguousarray((U * s) @ V.T)
    b = A @ rng.standard_normal(n) + noise * rng.standard_normal(m)
    return Problem(f"small_dense_{m}x{n}", m, n, "dense", np.dtype(np.float64), mu, sketch_dim,
                   b, dense=A, extra={"sigma": s})


def small_sparse(m, n, seed, nnz_per_col=3, mu=1e-4, sketch_dim=4, dtype=np.float64,
                 col_decay=6.0) -> Problem:
    rng_seed = seed - BASE_SEED
    return sparse_colscaled(m=m, n=n, nnz_per_col=nnz_per_col, mu=mu, sketch_dim=sketch_dim,
                            index=rng_seed, dtype=dtype, name=f"small_sparse_{m}x{n}",
                            col_decay=col_decay)


def by_name(name: str, scale: int = 1) -> Problem:
    return {"config1": config1, "config2": config2, "config3": config3,
            "config5": config5}[name](scale)


def batched(nprob=512, m_range=(2000, 50000), n_range=(100, 2000), density=1e-3, nrhs=16,
            mu=1e-5, sketch_dim=50, decay_orders=6.0, index=4, seed=None) -> list:
    """Batch of independent problems of uneven sizes: m ~ U[m_range], n ~ U[n_range]
    (m >= n); the first half dense, A = U diag(s) V^T with U, V from QR of Gaussians and
    s_i = 10^(-decay_orders i/(n-1)); the second half CSR with each entry nonzero with
    probability `density` and N(0,1) values; FP32 storage; nrhs right-hand sides ~ N(0,1)
    per problem (b has shape m x nrhs).  Host numpy generation (tests and small batches)."""
    rng = _rng(index) if seed is None else np.random.Generator(np.random.PCG64(seed))
    out = []
    half = nprob // 2
    for p in range(nprob):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        m = int(rng.integers(max(m_range[0], n), m_range[1] + 1))
        b = rng.standard_normal((m, nrhs))
        if p < half:
            U = _orth(rng, m, n)
            V = _orth(rng, n, n)
            sv = 10.0 ** (-decay_orders * np.arange(n) / max(n - 1, 1))
            A = np.ascontiguousarray(((U * sv) @ V.T).astype(np.float32))
            out.append(Problem(f"batch_dense_{p}_{m}x{n}", m, n, "dense", np.dtype(np.float32), mu,
                               sketch_dim, b, dense=A, extra={"sigma": sv}))
        else:
            mask = rng.random((m, n)) < density
            rows, cols = np.nonzero(mask)
            vals = rng.standard_normal(rows.size).astype(np.float32)
            indptr = np.zeros(m + 1, np.int64)
            np.add.at(indptr, rows + 1, 1)
            indptr = np.cumsum(indptr)
            out.append(Problem(f"batch_csr_{p}_{m}x{n}", m, n, "csr", np.dtype(np.float32), mu,
                               sketch_dim, b, indptr=indptr, indices=cols.astype(np.int64),
                               data=vals))
    return out


def batched_device(device, nprob=512, m_range=(2000, 50000), n_range=(100, 2000), density=1e-3,
                   nrhs=16, mu=1e-5, decay_orders=6.0, index=4):
    """The batched workload generated on the GPU (torch, seeded): same recipe as
    ``batched`` (sizes from the same host generator, U and V from QR of Gaussians drawn on
    the device, FP32 storage).  Dense rows are padded to a multiple of 4 floats (16-byte
    rows; A is a view with row stride ld).  Returns (mats, rhs, sizes) with device tensors
    (CSR matrices as torch.sparse_csr_tensor, right-hand sides m x nrhs float64)."""
    import torch

    rng = _rng(index)
    gen = torch.Generator(device=device)
    gen.manual_seed(BASE_SEED + index)
    mats, rhs, sizes = [], [], []
    half = nprob // 2
    for p in range(nprob):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        m = int(rng.integers(max(m_range[0], n), m_range[1] + 1))
        b = torch.randn(m, nrhs, generator=gen, device=device, dtype=torch.float64)
        if p < half:
            U, _ = torch.linalg.qr(torch.randn(m, n, generator=gen, device=device))
            V, _ = torch.linalg.qr(torch.randn(n, n, generator=gen, device=device))
            sv = 10.0 ** (-decay_orders * torch.arange(n, device=device, dtype=torch.float32)
                          / max(n - 1, 1))
            ld = (n + 3) // 4 * 4
            buf = torch.zeros(m, ld, device=device, dtype=torch.float32)
            buf[:, :n] = (U * sv) @ V.T
            del U, V
            mats.append(buf[:, :n])
        else:
            mask = torch.rand(m, n, generator=gen, device=device) < density
            idx = mask.nonzero()
            vals = torch.randn(idx.shape[0], generator=gen, device=device, dtype=torch.float32)
            counts = torch.bincount(idx[:, 0], minlength=m)
            crow = torch.zeros(m + 1, dtype=torch.int64, device=device)
            crow[1:] = torch.cumsum(counts, 0)
            mats.append(torch.sparse_csr_tensor(crow, idx[:, 1].contiguous(), vals, size=(m, n)))
            del mask
        rhs.append(b)
        sizes.append((m, n, "dense" if p < half else "csr"))
    return mats, rhs, sizes



def config5_device(device, mu: float = 1e-4, index=5):
    """The adjoint workload generated on the GPU (torch, seeded): the recipe of ``config5``
    (A = U diag(exp(-i/200)) V^T of 100000 x 2000 stored in FP32, U and V from QR of
    Gaussians drawn on the device; b and x_target ~ N(0, 1)), for the benchmark, where
    host generation would take a QR of a 100000 x 2000 matrix on the CPU.  Returns
    (A, b, x_target, mu, sketch_dim) as device tensors."""
    import torch

    m, n = 100000, 2000
    gen = torch.Generator(device=device)
    gen.manual_seed(BASE_SEED + 50 + index)
    U, _ = torch.linalg.qr(torch.randn(m, n, generator=gen, device=device, dtype=torch.float64))
    V, _ = torch.linalg.qr(torch.randn(n, n, generator=gen, device=device, dtype=torch.float64))
    s = torch.exp(-torch.arange(n, device=device, dtype=torch.float64) / 200.0)
    A = ((U * s) @ V.T).to(torch.float32).contiguous()
    del U, V
    b = torch.randn(m, generator=gen, device=device, dtype=torch.float64)
    xt = torch.randn(n, generator=gen, device=device, dtype=torch.float64)
    return A, b, xt, mu, 100
