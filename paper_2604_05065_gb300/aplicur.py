"""Python binding of the APLICUR C ABI (include/aplicur.h).

Argument marshalling only: every numerical step runs in libaplicur.so.  PyTorch
provides device memory and the current CUDA stream.  There is no CPU fallback:
if the library or a GPU is missing, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

REASONS = {0: "none", 1: "exact", 2: "replay", 3: "ps_test2", 4: "ps_test1", 5: "dynamic",
           6: "tol", 7: "maxit", 9: "drift", 10: "inner"}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "EBREAKDOWN",
          6: "ETIMEOUT"}
PREC_FP64, PREC_MIXED, PREC_DF32 = 0, 1, 2
SKETCH_SPARSE_SIGN, SKETCH_GAUSSIAN, SKETCH_SRHT = 0, 1, 2


class AplicurError(RuntimeError):
    def __init__(self, status: int, msg: str, allocator=None):
        if status == 2 and allocator is not None and allocator.last_error:
            msg = f"{msg} ({allocator.last_error})"
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Matrix(C.Structure):
    _fields_ = [("format", C.c_int32), ("dtype", C.c_int32), ("m", C.c_int64), ("n", C.c_int64),
                ("ld", C.c_int64), ("nnz", C.c_int64), ("values", C.c_void_p),
                ("rowptr", C.c_void_p), ("colidx", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("eps_cur_factor", C.c_double), ("nu_prec", C.c_double),
                ("nu_lsqr", C.c_double), ("eps_lsqr", C.c_double), ("xi", C.c_int32),
                ("normest_r", C.c_int32), ("check_gap", C.c_int32),
                ("max_extra_phases", C.c_int32), ("precision", C.c_int32),
                ("graph_iters", C.c_int32), ("sketch_rows", C.c_void_p),
                ("sketch_signs", C.c_void_p), ("normest_w", C.c_void_p),
                ("replay_nphases", C.c_int32), ("replay_phases", C.c_void_p),
                ("replay_nsteps", C.c_int32), ("replay_rebuild", C.c_void_p),
                ("profile", C.c_int32), ("max_rank", C.c_int32), ("fp64_dense", C.c_int32),
                ("variant", C.c_int32), ("schedule", C.c_int32), ("dense_pass", C.c_int32),
                ("alloc", C.c_void_p), ("free_", C.c_void_p), ("alloc_ctx", C.c_void_p),
                ("sketch_kind", C.c_int32), ("sketch_tc", C.c_int32)]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 7), ("launches", C.c_int64 * 7), ("work", C.c_double * 7),
                ("kernel_launches", C.c_int64)]


# kernel families of aplicur_profile: (name, unit of work)
PROFILE_FAMILIES = [("A z pass", "bytes"), ("A^T u pass", "bytes"),
                    ("preconditioner passes", "bytes"), ("dense products", "flops"),
                    ("second Jacobi stage", "flops"), ("LUPP selection", "bytes"),
                    ("FP32 Jacobi sweeps", "flops32")]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int64), ("ell", C.c_int32), ("nphases", C.c_int32),
                ("nsteps", C.c_int32), ("converged", C.c_int32), ("ne_res", C.c_double),
                ("rho", C.c_double), ("time_setup_ms", C.c_double),
                ("time_solve_ms", C.c_double), ("time_rank_ms", C.c_double),
                ("time_build_ms", C.c_double), ("time_lsqr_ms", C.c_double),
                ("fused_pass", C.c_int32), ("cluster_size", C.c_int32),
                ("rank_breakdown", C.c_int32)]


class BatchStats(C.Structure):
    _fields_ = [("pairs", C.c_int32), ("converged", C.c_int32), ("iters_max", C.c_int64),
                ("iters_sum", C.c_int64), ("ne_max", C.c_double), ("time_setup_ms", C.c_double),
                ("time_rank_ms", C.c_double), ("time_build_ms", C.c_double),
                ("time_lsqr_ms", C.c_double), ("time_check_ms", C.c_double),
                ("rows_per_warp", C.c_int32), ("cols_per_lane", C.c_int32),
                ("launches_per_iter", C.c_int64)]


# every entry point of include/aplicur.h: name -> (restype, argtypes)
_VP, _D, _I32, _I64 = C.c_void_p, C.c_double, C.c_int32, C.c_int64
_PI32 = C.POINTER(C.c_int32)
SIGNATURES = {
    "aplicur_options_default": (None, [C.POINTER(Options)]),
    "aplicur_create": (C.c_int, [C.POINTER(_VP), C.POINTER(Matrix), _VP, _D, _I32,
                                 C.POINTER(Options), _VP]),
    "aplicur_solve": (C.c_int, [_VP, _D, _I64, _VP]),
    "aplicur_set_replay": (C.c_int, [_VP, _I32, _VP, _I32, _VP]),
    "aplicur_plain_lsqr": (C.c_int, [_VP, _D, _I64, _VP]),
    "aplicur_backward": (C.c_int, [_VP, _VP, _D, _I64, _VP, C.POINTER(_D), _VP]),
    "aplicur_get_indices": (C.c_int, [_VP, _VP, _VP, _PI32]),
    "aplicur_get_sketch": (C.c_int, [_VP, _VP, _PI32]),
    "aplicur_get_stats": (C.c_int, [_VP, C.POINTER(Stats)]),
    "aplicur_get_phase": (C.c_int, [_VP, _I32, _PI32, C.POINTER(_I64), _PI32, C.POINTER(_D)]),
    "aplicur_get_step": (C.c_int, [_VP, _I32, _PI32, C.POINTER(_D), _PI32, C.POINTER(_D)]),
    "aplicur_get_preconditioner": (C.c_int, [_VP, _PI32, _VP, C.POINTER(_D)]),
    "aplicur_apply_preconditioner": (C.c_int, [_VP, _VP, _VP]),
    "aplicur_matvec": (C.c_int, [_VP, _I32, _VP, _VP]),
    "aplicur_get_profile": (C.c_int, [_VP, C.POINTER(Profile)]),
    "aplicur_reset_profile": (C.c_int, [_VP]),
    "aplicur_launch_count": (C.c_int64, []),
    "aplicur_internal_alloc_count": (C.c_int64, []),
    "aplicur_dense_atx_noalloc": (C.c_int, [C.POINTER(Matrix), _VP, _VP, _VP]),
    "aplicur_batch_create": (C.c_int, [C.POINTER(_VP), _I32, C.POINTER(Matrix), _VP, _I32, _D,
                                       _I32, C.POINTER(Options), _VP]),
    "aplicur_batch_solve": (C.c_int, [_VP, _D, _I64, _VP]),
    "aplicur_batch_plain_lsqr": (C.c_int, [_VP, _D, _I64, _VP]),
    "aplicur_batch_backward": (C.c_int, [_VP, _VP, _D, _I64, _VP, _VP, _VP]),
    "aplicur_batch_get_pair": (C.c_int, [_VP, _I32, _I32, C.POINTER(_I64), C.POINTER(_D), _PI32]),
    "aplicur_batch_get_problem": (C.c_int, [_VP, _I32, _PI32, _PI32, _PI32, _PI32, _VP, _VP]),
    "aplicur_batch_get_stats": (C.c_int, [_VP, C.POINTER(BatchStats)]),
    "aplicur_batch_last_error": (C.c_char_p, [_VP]),
    "aplicur_batch_destroy": (None, [_VP]),
    "aplicur_last_error": (C.c_char_p, [_VP]),
    "aplicur_status_string": (C.c_char_p, [C.c_int]),
    "aplicur_destroy": (None, [_VP]),
}

_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Load libaplicur.so (in-tree).  Raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run __graft_entry__.build() first")
        _build.build_library()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class DeviceAllocator:
    """The caller-side device allocator of aplicur_options (alloc / free_ / alloc_ctx):
    by default PyTorch's caching allocator on `device`, allocating on the stream the
    library names (stream-ordered reuse, as cudaMallocAsync).  It keeps a record of the
    live blocks and of the bytes handed out (`live`, `allocs`, `bytes`), and must outlive
    every handle it was given to."""

    def __init__(self, device, alloc=None, free=None):
        import torch
        self.index = torch.device(device).index if torch.device(device).index is not None \
            else torch.cuda.current_device()
        self.live = {}
        self.allocs = 0
        self.bytes = 0
        self.last_error = None   # the exception of the last refused allocation
        alloc = alloc or (lambda nbytes, stream: torch.cuda.caching_allocator_alloc(
            nbytes, self.index, stream))
        free = free or torch.cuda.caching_allocator_delete

        def _alloc(nbytes, stream, _ctx):
            try:
                ptr = int(alloc(int(nbytes), int(stream or 0)))
            except Exception as e:   # the library turns NULL into ENOMEM
                self.last_error = f"{type(e).__name__}: {e}"
                return None
            self.live[ptr] = int(nbytes)
            self.allocs += 1
            self.bytes += int(nbytes)
            return ptr

        def _free(ptr, _nbytes, _stream, _ctx):
            if ptr is None:
                return
            self.live.pop(int(ptr), None)
            free(int(ptr))

        self._alloc = _ALLOC_FN(_alloc)
        self._free = _FREE_FN(_free)

    def install(self, opts: "Options") -> None:
        opts.alloc = C.cast(self._alloc, C.c_void_p).value
        opts.free_ = C.cast(self._free, C.c_void_p).value
        opts.alloc_ctx = None


# live handles (weakly held) are destroyed at exit, before the interpreter tears down the
# Python objects their allocator's free callbacks call into
import weakref as _weakref  # noqa: E402
_LIVE_HANDLES = _weakref.WeakSet()


def _destroy_live_handles():
    for obj in list(_LIVE_HANDLES):
        try:
            obj.close()
        except Exception:
            pass


import atexit as _atexit  # noqa: E402
_atexit.register(_destroy_live_handles)


def default_options() -> Options:
    o = Options()
    load().aplicur_options_default(C.byref(o))
    return o


def _check(lib, st, h=None, allocator=None):
    if st != 0 and st != 4:
        msg = lib.aplicur_last_error(h).decode() if h is not None else ""
        raise AplicurError(st, msg, allocator)
    return st


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("APLICUR needs a CUDA GPU")
    return torch


def _marshal_matrix(torch, A):
    """aplicur_matrix for a dense CUDA tensor (row-major rows, any row stride) or a
    torch.sparse_csr_tensor; returns (struct, tensors to keep alive, value dtype)."""
    mat = Matrix()
    if A.layout == torch.sparse_csr:
        rowptr = A.crow_indices().to(torch.int32).contiguous()
        colidx = A.col_indices().to(torch.int32).contiguous()
        vals = A.values().contiguous()
        keep = [rowptr, colidx, vals]
        mat.format = 1
        mat.nnz = vals.numel()
        mat.values = vals.data_ptr()
        mat.rowptr = rowptr.data_ptr()
        mat.colidx = colidx.data_ptr()
        mat.ld = A.shape[1]
        dt = vals.dtype
    else:
        if A.stride(1) != 1:
            A = A.contiguous()
        keep = [A]
        mat.format = 0
        mat.ld = A.stride(0)
        mat.nnz = A.shape[0] * A.shape[1]
        mat.values = A.data_ptr()
        dt = A.dtype
    if dt == torch.float64:
        mat.dtype = 0
    elif dt == torch.float32:
        mat.dtype = 1
    else:
        raise TypeError("A must be float64 or float32")
    mat.m, mat.n = int(A.shape[0]), int(A.shape[1])
    return mat, keep, dt


class Solver:
    """One APLICUR problem min ||A x - b||^2 + mu ||x||^2 on the GPU.

    A: a dense CUDA tensor (m x n, float64 or float32, row-major) or a
    torch.sparse_csr_tensor on CUDA; b: CUDA tensor of m values (converted to
    float64).  Options are fields of the C options struct."""

    def __init__(self, A, b, mu: float, sketch_dim: int, *, sketch_rows=None, sketch_signs=None,
                 normest_w=None, replay=None, allocator="torch", **opts):
        torch = _torch()
        lib = load()
        self._lib = lib
        self._h = None
        mat, self._keep, dt = _marshal_matrix(torch, A)
        self.m, self.n = mat.m, mat.n
        self.dtype = dt
        self.device = b.device
        b = b.to(torch.float64).contiguous()
        self._keep.append(b)
        self.b = b
        o = default_options()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        import numpy as np
        host = []
        if sketch_rows is not None:
            r = np.ascontiguousarray(sketch_rows, dtype=np.int32)
            s = np.ascontiguousarray(sketch_signs, dtype=np.int8)
            host += [r, s]
            o.sketch_rows = r.ctypes.data
            o.sketch_signs = s.ctypes.data
            o.xi = r.shape[1]
        if normest_w is not None:
            w = np.asfortranarray(normest_w, dtype=np.float64)
            host.append(w)
            o.normest_w = w.ctypes.data
            o.normest_r = w.shape[1]
        self.mu = float(mu)
        self.sketch_dim = int(sketch_dim)
        # device workspace: PyTorch's caching allocator (default), a DeviceAllocator, or
        # None for the library's own stream-ordered allocations
        if allocator == "torch":
            allocator = DeviceAllocator(self.device)
        self.allocator = allocator
        if allocator is not None:
            allocator.install(o)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        h = C.c_void_p()
        st = lib.aplicur_create(C.byref(h), C.byref(mat), b.data_ptr(), self.mu, self.sketch_dim,
                                C.byref(o), C.c_void_p(stream))
        if st != 0:
            raise AplicurError(st, lib.aplicur_last_error(None).decode(), allocator)
        self._h = h
        _LIVE_HANDLES.add(self)
        if replay is not None:
            self.set_replay(replay)

    def __del__(self):
        if getattr(self, "_h", None) is not None:
            self._lib.aplicur_destroy(self._h)
            self._h = None
        _LIVE_HANDLES.discard(self)

    def close(self):
        self.__del__()

    # ------------------------------------------------------------------ solves ------
    def solve(self, tol: float = 1e-10, maxit: int = 100000):
        torch = _torch()
        x = torch.empty(self.n, dtype=torch.float64, device=self.device)
        st = self._lib.aplicur_solve(self._h, tol, maxit, x.data_ptr())
        _check(self._lib, st, self._h, self.allocator)
        self.last_status = st
        return x

    def plain_lsqr(self, tol: float = 1e-10, maxit: int = 100000):
        torch = _torch()
        x = torch.empty(self.n, dtype=torch.float64, device=self.device)
        st = self._lib.aplicur_plain_lsqr(self._h, tol, maxit, x.data_ptr())
        _check(self._lib, st, self._h, self.allocator)
        self.last_status = st
        return x

    def backward(self, grad_x, tol: float = 1e-10, maxit: int = 100000, want_A: bool = True):
        torch = _torch()
        g = grad_x.to(torch.float64).contiguous()
        gb = torch.empty(self.m, dtype=torch.float64, device=self.device)
        gmu = C.c_double(0.0)
        gA = None
        if want_A:
            gA = torch.empty(self.m, self.n, dtype=self.dtype, device=self.device)
        st = self._lib.aplicur_backward(self._h, g.data_ptr(), tol, maxit, gb.data_ptr(),
                                        C.byref(gmu), gA.data_ptr() if gA is not None else None)
        _check(self._lib, st, self._h, self.allocator)
        return gb, gmu.value, gA

    def set_replay(self, replay: dict):
        import numpy as np
        ph = np.ascontiguousarray(replay.get("phases", []), dtype=np.int32)
        rb = np.ascontiguousarray(replay.get("rebuild", []), dtype=np.int8)
        st = self._lib.aplicur_set_replay(self._h, ph.size, ph.ctypes.data if ph.size else None,
                                          rb.size, rb.ctypes.data if rb.size else None)
        _check(self._lib, st, self._h, self.allocator)

    # ------------------------------------------------------------------ queries -----
    def indices(self):
        import numpy as np
        k = min(self.m, self.n)
        I = np.zeros(k, dtype=np.int32)
        J = np.zeros(k, dtype=np.int32)
        ell = C.c_int32(0)
        _check(self._lib, self._lib.aplicur_get_indices(self._h, I.ctypes.data, J.ctypes.data,
                                                        C.byref(ell)), self._h)
        return I[:ell.value].copy(), J[:ell.value].copy()

    def sketch(self):
        torch = _torch()
        s = C.c_int32(0)
        _check(self._lib, self._lib.aplicur_get_sketch(self._h, None, C.byref(s)), self._h)
        Y = torch.empty(self.n, s.value, dtype=torch.float64, device=self.device)
        _check(self._lib, self._lib.aplicur_get_sketch(self._h, Y.data_ptr(), C.byref(s)),
               self._h)
        return Y.T  # s x n

    def stats(self) -> dict:
        st = Stats()
        _check(self._lib, self._lib.aplicur_get_stats(self._h, C.byref(st)), self._h)
        return {f: getattr(st, f) for f, _ in Stats._fields_}

    def phases(self) -> list:
        out = []
        for k in range(self.stats()["nphases"]):
            ell, it, rs, ne = C.c_int32(), C.c_int64(), C.c_int32(), C.c_double()
            _check(self._lib, self._lib.aplicur_get_phase(self._h, k, C.byref(ell), C.byref(it),
                                                          C.byref(rs), C.byref(ne)), self._h)
            out.append(dict(ell=ell.value, iters=it.value, reason=REASONS.get(rs.value),
                            ne_res=ne.value))
        return out

    def steps(self) -> list:
        out = []
        for k in range(self.stats()["nsteps"]):
            ell, rho, rb, mg = C.c_int32(), C.c_double(), C.c_int32(), C.c_double()
            _check(self._lib, self._lib.aplicur_get_step(self._h, k, C.byref(ell), C.byref(rho),
                                                         C.byref(rb), C.byref(mg)), self._h)
            out.append(dict(ell=ell.value, rho=rho.value, rebuild=bool(rb.value),
                            margin=mg.value))
        return out

    def preconditioner(self):
        torch = _torch()
        ell = C.c_int32(0)
        sh = C.c_double(0.0)
        _check(self._lib, self._lib.aplicur_get_preconditioner(self._h, C.byref(ell), None,
                                                               C.byref(sh)), self._h)
        sig = torch.empty(max(ell.value, 1), dtype=torch.float64, device=self.device)
        _check(self._lib, self._lib.aplicur_get_preconditioner(self._h, C.byref(ell),
                                                               sig.data_ptr(), C.byref(sh)),
               self._h)
        return sig[:ell.value], sh.value

    def apply_preconditioner(self, w):
        torch = _torch()
        w = w.to(torch.float64).contiguous()
        out = torch.empty_like(w)
        _check(self._lib, self._lib.aplicur_apply_preconditioner(self._h, w.data_ptr(),
                                                                 out.data_ptr()), self._h)
        return out

    def profile(self) -> dict:
        pr = Profile()
        _check(self._lib, self._lib.aplicur_get_profile(self._h, C.byref(pr)), self._h)
        return {"ms": list(pr.ms), "launches": list(pr.launches), "work": list(pr.work),
                "kernel_launches": pr.kernel_launches}

    def reset_profile(self):
        _check(self._lib, self._lib.aplicur_reset_profile(self._h), self._h)

    def matvec(self, x, trans: bool = False):
        torch = _torch()
        x = x.to(torch.float64).contiguous()
        y = torch.empty(self.n if trans else self.m, dtype=torch.float64, device=self.device)
        _check(self._lib, self._lib.aplicur_matvec(self._h, 1 if trans else 0, x.data_ptr(),
                                                   y.data_ptr()), self._h)
        return y


def _check_noalloc_args(torch, A, x, y):
    """Argument checks of dense_atx_noalloc, all taken before any launch: dtypes first,
    then sizes, then devices (so that a mistake is reported by its real cause)."""
    if A.dim() != 2 or A.layout != torch.strided:
        raise ValueError("A must be a dense 2-D tensor")
    if A.dtype not in (torch.float64, torch.float32):
        raise TypeError("A must be float64 or float32")
    if A.shape[0] < 1 or A.shape[1] < 1:
        raise ValueError("A must have at least one row and one column")
    if A.stride(1) != 1:
        raise ValueError("A must be row-major (unit column stride)")
    m, n = int(A.shape[0]), int(A.shape[1])
    if x.dim() != 1 or x.numel() != m:
        raise ValueError(f"x must be a vector of m = {m} values")
    if y is not None:
        if y.dtype != torch.float64:
            raise TypeError("y must be float64")
        if y.dim() != 1 or y.numel() < n or not y.is_contiguous():
            raise ValueError(f"y must be a contiguous vector of at least n = {n} values")
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    if x.device != A.device:
        raise ValueError("x must be on A's device")
    if y is not None and y.device != A.device:
        raise ValueError("y must be on A's device")


def dense_atx_noalloc(A, x, y=None):
    """y = A^T x for a dense CUDA tensor A through the allocation-free entry point (the
    library allocates nothing; y, if not given, is allocated here by PyTorch, and x is
    converted to a contiguous float64 copy when it is not one already).  The call runs on
    A's device and that device's current stream."""
    import torch
    _check_noalloc_args(torch, A, x, y)
    torch = _torch()
    lib = load()
    mat = Matrix()
    mat.format = 0
    mat.dtype = 0 if A.dtype == torch.float64 else 1
    mat.m, mat.n = int(A.shape[0]), int(A.shape[1])
    mat.ld = A.stride(0)
    mat.nnz = mat.m * mat.n
    mat.values = A.data_ptr()
    with torch.cuda.device(A.device):
        x = x.to(torch.float64).contiguous()
        if y is None:
            y = torch.empty(mat.n, dtype=torch.float64, device=A.device)
        stream = torch.cuda.current_stream(A.device).cuda_stream
        st = lib.aplicur_dense_atx_noalloc(C.byref(mat), x.data_ptr(), y.data_ptr(),
                                           C.c_void_p(stream))
    if st != 0:
        raise AplicurError(st, lib.aplicur_last_error(None).decode())
    return y


def launch_count() -> int:
    """Kernels launched through the library by this process so far."""
    return int(load().aplicur_launch_count())


def solve(A, b, mu, sketch_dim, tol=1e-10, maxit=100000, **opts):
    """x = argmin ||A x - b||^2 + mu ||x||^2 by APLICUR on the GPU."""
    s = Solver(A, b, mu, sketch_dim, **opts)
    try:
        return s.solve(tol, maxit)
    finally:
        s.close()


def _autograd_function():
    import torch

    class APLICURSolve(torch.autograd.Function):
        """x(A, b, mu) = argmin ||A x - b||^2 + mu ||x||^2 with gradients with respect to
        A (dense), b and mu from the adjoint solve (A^T A + mu I) lambda = dL/dx."""

        @staticmethod
        def forward(ctx, A, b, mu, sketch_dim=100, tol=1e-10, maxit=100000, opts=None):
            mu_v = float(mu.item()) if torch.is_tensor(mu) else float(mu)
            s = Solver(A.detach(), b.detach(), mu_v, int(sketch_dim), **(opts or {}))
            x = s.solve(tol, maxit)
            ctx.solver = s
            ctx.tol, ctx.maxit = tol, maxit
            ctx.mu_is_tensor = torch.is_tensor(mu)
            ctx.mu_dtype = mu.dtype if torch.is_tensor(mu) else None
            return x

        @staticmethod
        def backward(ctx, gx):
            s = ctx.solver
            gb, gmu, gA = s.backward(gx, ctx.tol, ctx.maxit, want_A=ctx.needs_input_grad[0])
            gmu_t = None
            if ctx.needs_input_grad[2] and ctx.mu_is_tensor:
                gmu_t = torch.tensor(gmu, dtype=ctx.mu_dtype, device=gx.device)
            s.close()
            return (gA if ctx.needs_input_grad[0] else None,
                    gb if ctx.needs_input_grad[1] else None, gmu_t, None, None, None, None)

    return APLICURSolve


class _Lazy:
    def __get__(self, obj, owner):
        return _autograd_function()


def aplicur_solve_fn():
    """The torch.autograd.Function class (created lazily so that importing this module
    does not import torch)."""
    return _autograd_function()


class BatchSolver:
    """A batch of independent problems min ||A_p x - b_{p,r}||^2 + mu ||x||^2 solved by
    the library's grouped multi-right-hand-side APLICUR (aplicur_batch_* entry points).

    mats: list of FP32 CUDA matrices (dense, any row stride, or sparse CSR);
    rhs: list of CUDA tensors of shape (m_p, R) or (m_p,) (converted to float64).
    Problem p is seeded with options.seed + p."""

    def __init__(self, mats, rhs, mu: float, sketch_dim: int, allocator="torch", **opts):
        torch = _torch()
        lib = load()
        self._lib = lib
        self._h = None
        if len(mats) != len(rhs) or not mats:
            raise ValueError("need one right-hand-side block per matrix")
        self._keep = []
        arr = (Matrix * len(mats))()
        self.shapes = []
        R = None
        bptr = (C.c_void_p * len(mats))()
        self._dense = []
        for p, (A, b) in enumerate(zip(mats, rhs)):
            mat, keep, _ = _marshal_matrix(torch, A)
            self._dense.append(mat.format == 0)
            self._keep += keep
            arr[p] = mat
            b2 = b.reshape(b.shape[0], -1).to(torch.float64)
            if R is None:
                R = b2.shape[1]
            if b2.shape[1] != R or b2.shape[0] != mat.m:
                raise ValueError("right-hand sides must be (m_p, R) with one R")
            bt = b2.t().contiguous()  # column-major m x R
            self._keep.append(bt)
            bptr[p] = bt.data_ptr()
            self.shapes.append((mat.m, mat.n))
        self.R = R
        self.device = rhs[0].device
        o = default_options()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        if allocator == "torch":
            allocator = DeviceAllocator(self.device)
        self.allocator = allocator
        if allocator is not None:
            allocator.install(o)
        h = C.c_void_p()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        st = lib.aplicur_batch_create(C.byref(h), len(mats), arr, bptr, R, float(mu),
                                      int(sketch_dim), C.byref(o), C.c_void_p(stream))
        if st != 0:
            raise AplicurError(st, lib.aplicur_batch_last_error(None).decode(), allocator)
        self._h = h
        _LIVE_HANDLES.add(self)

    def __del__(self):
        if getattr(self, "_h", None) is not None:
            self._lib.aplicur_batch_destroy(self._h)
            self._h = None
        _LIVE_HANDLES.discard(self)

    def close(self):
        self.__del__()

    def _run(self, fn, tol, maxit):
        torch = _torch()
        xs = [torch.empty(self.R, n, dtype=torch.float64, device=self.device)
              for (_, n) in self.shapes]
        ptr = (C.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        st = fn(self._h, float(tol), int(maxit), ptr)
        if st != 0 and st != 4:
            raise AplicurError(st, self._lib.aplicur_batch_last_error(self._h).decode(),
                               self.allocator)
        self.last_status = st
        return [x.t() for x in xs]

    def solve(self, tol: float = 1e-8, maxit: int = 100000):
        """List of (n_p, R) float64 solutions."""
        return self._run(self._lib.aplicur_batch_solve, tol, maxit)

    def plain_lsqr(self, tol: float = 1e-8, maxit: int = 100000):
        return self._run(self._lib.aplicur_batch_plain_lsqr, tol, maxit)

    def backward(self, grad_x, tol: float = 1e-8, maxit: int = 100000, want_A: bool = True):
        """Adjoint of the last solve.  grad_x: list of (n_p, R) CUDA tensors dL/dx.
        Returns (grad_b: list of (m_p, R) float64, grad_mu: (nprob, R) float64,
        grad_A: list of (m_p, n_p) float32 for dense problems, None for CSR ones, or
        None when want_A is False)."""
        torch = _torch()
        npb = len(self.shapes)
        if len(grad_x) != npb:
            raise ValueError("need one gradient block per problem")
        keep, gptr = [], (C.c_void_p * npb)()
        for p, (g, (m, n)) in enumerate(zip(grad_x, self.shapes)):
            g2 = g.reshape(n, -1).to(device=self.device, dtype=torch.float64)
            if g2.shape[1] != self.R:
                raise ValueError("gradients must be (n_p, R)")
            gt = g2.t().contiguous()  # column-major n x R
            keep.append(gt)
            gptr[p] = gt.data_ptr()
        gb = [torch.empty(self.R, m, dtype=torch.float64, device=self.device)
              for (m, _) in self.shapes]
        bptr = (C.c_void_p * npb)(*[x.data_ptr() for x in gb])
        gmu = torch.empty(npb * self.R, dtype=torch.float64, device=self.device)
        gA, aptr = None, None
        if want_A:
            gA = [torch.empty(m, n, dtype=torch.float32, device=self.device) if self._dense[p]
                  else None for p, (m, n) in enumerate(self.shapes)]
            aptr = (C.c_void_p * npb)(*[x.data_ptr() if x is not None else None for x in gA])
        st = self._lib.aplicur_batch_backward(self._h, gptr, float(tol), int(maxit), bptr,
                                              C.c_void_p(gmu.data_ptr()), aptr)
        if st != 0 and st != 4:
            raise AplicurError(st, self._lib.aplicur_batch_last_error(self._h).decode(),
                               self.allocator)
        self.last_status = st
        return [x.t() for x in gb], gmu.reshape(npb, self.R), gA

    def pair(self, p: int, r: int) -> dict:
        it, ne, cv = C.c_int64(), C.c_double(), C.c_int32()
        _check_b(self._lib, self._lib.aplicur_batch_get_pair(self._h, p, r, C.byref(it),
                                                               C.byref(ne), C.byref(cv)), self._h)
        return {"iters": it.value, "ne_res": ne.value, "converged": bool(cv.value)}

    def problem(self, p: int) -> dict:
        import numpy as np
        ell, ns, nph, br = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check_b(self._lib, self._lib.aplicur_batch_get_problem(
            self._h, p, C.byref(ell), C.byref(ns), C.byref(nph), C.byref(br), None, None), self._h)
        I = np.zeros(max(ell.value, 1), np.int32)
        J = np.zeros(max(ell.value, 1), np.int32)
        _check_b(self._lib, self._lib.aplicur_batch_get_problem(
            self._h, p, None, None, None, None, I.ctypes.data, J.ctypes.data), self._h)
        return {"ell": ell.value, "nsteps": ns.value, "nphases": nph.value,
                "breakdown": bool(br.value),
                "I": I[:ell.value].astype(np.int64), "J": J[:ell.value].astype(np.int64)}

    def stats(self) -> dict:
        s = BatchStats()
        _check_b(self._lib, self._lib.aplicur_batch_get_stats(self._h, C.byref(s)), self._h)
        return {k: getattr(s, k) for k, _ in BatchStats._fields_}


def _check_b(lib, st, h):
    if st != 0:
        raise AplicurError(st, lib.aplicur_batch_last_error(h).decode())
    return st
