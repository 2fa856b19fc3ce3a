"""The allocation-free entry point aplicur_dense_atx_noalloc against the existing
transposed product aplicur_matvec(trans=1).

It exists for callers that cannot allocate device memory (fixed arenas, pre-allocated
pools, paths where an allocation would synchronise).  Its scratch is a static device
array shared by all calls, so this file checks two calls in a row against the
existing entry point, within the tolerance of the other matvec parity tests (1e-13
relative).  It is named to be collected last, and it needs no state from other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_noalloc_matches_existing_transposed_matvec_twice(dtype):
    import torch

    import paper_2604_05065_gb300 as pkg
    from paper_2604_05065_gb300 import aplicur as api

    rng = np.random.default_rng(17)
    m, n = 3001, 517
    A_np = rng.standard_normal((m, n)).astype(dtype)
    A = torch.from_numpy(A_np).cuda()
    b = torch.from_numpy(rng.standard_normal(m)).cuda()
    s = pkg.Solver(A, b, 1e-4, 4, precision=pkg.PREC_FP64)
    for k in range(2):
        x = torch.from_numpy(rng.standard_normal(m)).cuda()
        ref = s.matvec(x, trans=True).cpu().numpy()
        y = api.dense_atx_noalloc(A, x)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert _rel(got, ref) <= 1e-13, f"call {k}"
        exact = A_np.astype(np.float64).T @ x.cpu().numpy()
        assert _rel(got, exact) <= 1e-13
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import ctypes as C

    import torch

    from paper_2604_05065_gb300 import aplicur as api

    lib = api.load()
    tiny = torch.zeros(8, dtype=torch.float64, device="cuda")
    mat = api.Matrix()
    mat.format, mat.dtype = 0, 0
    mat.m, mat.n = 1, (1 << 19) + 1
    mat.ld, mat.nnz = mat.n, mat.n
    mat.values = tiny.data_ptr()
    st = lib.aplicur_dense_atx_noalloc(C.byref(mat), tiny.data_ptr(), tiny.data_ptr(), None)
    assert st == 1
    assert b"limit" in lib.aplicur_last_error(None)
