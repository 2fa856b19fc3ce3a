"""Caller-owned device workspace: with a DeviceAllocator in aplicur_options every device
buffer of a handle comes from the caller's allocator (here a counting wrapper around
PyTorch's caching allocator) and goes back to it; the library makes no allocation of its
own.  Results are the same as with the library's own allocations."""
import numpy as np
import pytest

from paper_2604_05065_gb300 import workloads as wl

from gpu_helpers import draws, rel, to_device

pytestmark = pytest.mark.gpu


def _counting(device):
    import torch

    from paper_2604_05065_gb300 import aplicur as api
    calls = {"alloc": 0, "free": 0, "bytes": 0, "streams": set()}

    def alloc(nbytes, stream):
        calls["alloc"] += 1
        calls["bytes"] += nbytes
        calls["streams"].add(stream)
        return torch.cuda.caching_allocator_alloc(nbytes, device, stream)

    def free(ptr):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    return api.DeviceAllocator(device, alloc=alloc, free=free), calls


@pytest.mark.parametrize("name", ["dense32", "sparse64"])
def test_counting_allocator_sees_every_allocation(name):
    import torch

    import paper_2604_05065_gb300 as pkg
    from paper_2604_05065_gb300 import aplicur as api
    p = {"dense32": wl.dense_lowrank(m=600, n=120, mu=1e-4, sketch_dim=8, index=60,
                                     dtype=np.float32, name="dense32"),
         "sparse64": wl.small_sparse(3000, 300, wl.BASE_SEED + 50, nnz_per_col=6, mu=1e-5,
                                     sketch_dim=10)}[name]
    rows, signs, W = draws(p)
    A, b = to_device(p)
    lib = api.load()
    kw = dict(sketch_rows=rows, sketch_signs=signs, normest_w=W)
    if p.fmt == "dense":
        kw["precision"] = pkg.PREC_MIXED
    ref = pkg.Solver(A, b, p.mu, p.sketch_dim, allocator=None, **kw)
    x_ref = ref.solve(1e-10).cpu().numpy()
    ref.close()
    al, calls = _counting(0)
    own0 = lib.aplicur_internal_alloc_count()
    s = pkg.Solver(A, b, p.mu, p.sketch_dim, allocator=al, **kw)
    x = s.solve(1e-10).cpu().numpy()
    g = s.backward(torch.ones(p.n, dtype=torch.float64, device="cuda"), want_A=False)
    s.close()
    torch.cuda.synchronize()
    assert lib.aplicur_internal_alloc_count() == own0   # nothing from the library itself
    assert calls["alloc"] > 0 and calls["bytes"] > 0
    assert calls["alloc"] == calls["free"] and not al.live   # every block came back
    assert rel(x, x_ref) <= 1e-12
    assert g[0] is not None


def test_allocator_failure_is_reported_as_enomem():
    import paper_2604_05065_gb300 as pkg
    from paper_2604_05065_gb300 import aplicur as api
    p = wl.config1(scale=4)
    A, b = to_device(p)

    def refuse(nbytes, stream):
        raise MemoryError("refused")

    al = api.DeviceAllocator(0, alloc=refuse, free=lambda ptr: None)
    with pytest.raises(pkg.AplicurError) as e:
        pkg.Solver(A, b, p.mu, p.sketch_dim, allocator=al)
    assert e.value.status == 2


def test_batch_with_counting_allocator():
    import torch

    import paper_2604_05065_gb300 as pkg
    from paper_2604_05065_gb300 import aplicur as api
    probs = [wl.dense_lowrank(m=400 + 40 * i, n=60, mu=1e-5, sketch_dim=8, index=70 + i,
                              dtype=np.float32, name="b") for i in range(3)]
    mats = [torch.from_numpy(np.ascontiguousarray(q.dense)).cuda() for q in probs]
    rhs = [torch.from_numpy(np.stack([q.b, -q.b], 1)).cuda() for q in probs]
    lib = api.load()
    al, calls = _counting(0)
    own0 = lib.aplicur_internal_alloc_count()
    s = pkg.BatchSolver(mats, rhs, 1e-5, 8, allocator=al, seed=3)
    xs = s.solve(1e-8)
    st = s.stats()
    s.close()
    torch.cuda.synchronize()
    assert st["converged"] == st["pairs"] == 6
    assert lib.aplicur_internal_alloc_count() == own0
    assert calls["alloc"] > 0 and calls["alloc"] == calls["free"] and not al.live
    assert all(bool(torch.isfinite(x).all()) for x in xs)
