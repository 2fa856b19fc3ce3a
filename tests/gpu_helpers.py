"""Shared helpers for the GPU parity tests: move a workload to the device and run the
oracle with the same random draws."""
import numpy as np

from oracle import aplicur_oracle as O
from oracle import rng as orng


def device():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")


def to_device(p):
    import torch
    dev = device()
    if p.fmt == "dense":
        A = torch.from_numpy(np.ascontiguousarray(p.dense)).to(dev)
    else:
        A = torch.sparse_csr_tensor(torch.from_numpy(p.indptr.astype(np.int64)),
                                    torch.from_numpy(p.indices.astype(np.int64)),
                                    torch.from_numpy(p.data), size=(p.m, p.n)).to(dev)
    b = torch.from_numpy(np.asarray(p.b, dtype=np.float64)).to(dev)
    return A, b


def oracle_matrix(p):
    """A as the oracle sees it: float64 values of the stored (possibly FP32) matrix."""
    return p.to_scipy() if p.fmt == "csr" else np.asarray(p.dense, dtype=np.float64)


def draws(p, seed=5, r=10):
    s = O.sketch_rows(p.sketch_dim)
    xi = O.sketch_xi(s)
    rows, signs = orng.sparse_sign(seed, s, p.m, xi)
    W = orng.gaussian_w(seed, p.n, r)
    return rows, signs, W


def schedule(res):
    return {"phases": [ph["iters"] for ph in res.phases],
            "rebuild": [bool(st["rebuild"]) for st in res.rank_steps]}


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
