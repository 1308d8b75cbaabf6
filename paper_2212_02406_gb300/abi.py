"""Thin Python binding of the libnn C ABI (``include/nn.h``).

Argument marshalling only: every function here checks tensor placement, dtype and
layout, turns tensors into pointers and calls the entry point of the same name in
``lib/libnn.so``. There is no fallback: if the library is missing, every call raises.
PyTorch provides device memory and streams; all arithmetic runs in the CUDA kernels.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_size_t, c_void_p

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libnn.so")

NN_OK = 0
NN_ERR_ARG = 1
NN_ERR_DIVERGED = 2
NN_ERR_NOT_CONVERGED = 3
NN_ERR_OOM_BUDGET = 4
NN_ERR_TIMEOUT = 5
NN_ERR_CUDA = 6
NN_ERR_UNSUPPORTED = 7
NN_ERR_TOO_LARGE = 8
STATUS_NAMES = {0: "ok", 1: "arg", 2: "diverged", 3: "not_converged", 4: "oom_budget", 5: "timeout",
                6: "cuda", 7: "unsupported", 8: "too_large"}
NN_RESIDUAL_NOALLOC_MAX_N = 1440
NN_BATCHED_KERNELS = 22

NN_F64, NN_F32, NN_MIXED_BF16, NN_F64_DF, NN_F64_EMU, NN_MIXED_EMU, NN_MIXED_F16 = 0, 1, 2, 3, 4, 5, 6
DTYPES = {"f64": NN_F64, "f32": NN_F32, "mixed_bf16": NN_MIXED_BF16, "f64_df": NN_F64_DF,
          "f64_emu": NN_F64_EMU, "mixed_emu": NN_MIXED_EMU, "mixed_f16": NN_MIXED_F16}
NN_PC_PAN_SCHREIBER, NN_PC_SCALAR, NN_PC_TRACE, NN_PC_JACOBI, NN_PC_THETA2 = 0, 1, 2, 3, 4
PRECONDS = {"pan_schreiber": 0, "scalar": 1, "trace": 2, "jacobi": 3, "theta2": 4}
NN_MAX_HISTORY = 65


class NNOpts(ctypes.Structure):
    _fields_ = [("depth", c_int), ("tol", c_double), ("max_nests", c_int), ("dtype", c_int),
                ("refine_below", c_double), ("bulk_pieces", c_int), ("flags", c_int),
                ("depth_schedule", POINTER(c_int32)), ("schedule_len", c_int), ("x0_scalar", c_double),
                ("fwd_tol", c_double)]


class NNResult(ctypes.Structure):
    _fields_ = [("status", c_int), ("nests", c_int), ("residual", c_double),
                ("history", c_double * NN_MAX_HISTORY), ("pieces", c_int * NN_MAX_HISTORY),
                ("gemms", c_int), ("flops", c_double), ("hw_flops", c_double), ("launches", c_int),
                ("tc_launches", c_int), ("tc_ms", c_double), ("tc_flops", c_double),
                ("residual_est", c_double)]

    def as_dict(self) -> dict:
        k = self.nests
        return {"status": self.status, "status_name": STATUS_NAMES.get(self.status, "?"), "nests": k,
                "residual": self.residual, "history": [self.history[i] for i in range(k + 1)],
                "pieces": [self.pieces[i] for i in range(k + 1)], "gemms": self.gemms,
                "flops": self.flops, "hw_flops": self.hw_flops, "launches": self.launches,
                "tc_launches": self.tc_launches, "tc_ms": self.tc_ms, "tc_flops": self.tc_flops,
                "residual_est": self.residual_est}


class NNServerOpts(ctypes.Structure):
    _fields_ = [("arena", c_void_p), ("arena_bytes", c_size_t), ("max_active", c_int), ("depth", c_int),
                ("tol", c_double), ("max_nests", c_int)]


class NNRequest(ctypes.Structure):
    _fields_ = [("id", c_int64), ("n", c_int64), ("A", c_void_p), ("nrhs", c_int64), ("B", c_void_p),
                ("Y", c_void_p), ("X", c_void_p), ("dtype", c_int), ("precond", c_int), ("pc_scalar", c_double)]


class NNCompletion(ctypes.Structure):
    _fields_ = [("id", c_int64), ("status", c_int), ("nests", c_int), ("residual", c_double),
                ("t_submit", c_double), ("t_start", c_double), ("t_done", c_double), ("launches", c_int)]


_LIB = None

# Every symbol include/nn.h declares, with its ctypes signature.
_SIGNATURES = {
    "nn_set_gemm_variant": (c_int, [c_int]),
    "nn_debug_withhold_signal": (c_int, [c_int]),
    "nn_workspace_bytes": (c_size_t, [c_int64, c_int]),
    "nn_workspace_bytes_host": (c_size_t, [c_int64, c_int]),
    "nn_init_precond": (c_int, [c_void_p, c_int64, c_int64, c_int, c_double, c_void_p, c_int64, c_void_p, c_size_t,
                                c_void_p]),
    "nn_invert": (c_int, [c_void_p, c_int64, c_int64, c_void_p, c_int64, POINTER(NNOpts), c_void_p, c_int64,
                          POINTER(NNResult), c_void_p, c_size_t, c_void_p]),
    "nn_invert_host": (c_int, [c_void_p, c_int64, c_void_p, POINTER(NNOpts), c_void_p, POINTER(NNResult), c_void_p,
                               c_size_t, c_void_p]),
    "nn_invert_host_pc": (c_int, [c_void_p, c_int64, c_int, c_double, POINTER(NNOpts), c_void_p, POINTER(NNResult),
                                  c_void_p, c_size_t, c_void_p]),
    "nn_residual": (c_int, [c_void_p, c_int64, c_void_p, c_int64, c_int64, c_int, POINTER(c_double), c_void_p,
                            c_size_t, c_void_p]),
    "nn_csr_workspace_bytes": (c_size_t, [c_int64, c_int64, c_int64, c_int]),
    "nn_set_spmv_variant": (c_int, [c_int]),
    "nn_solve_csr_sched": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int, c_void_p, c_int64, c_int64,
                                   POINTER(c_int32), c_int, c_double, c_void_p, c_int64, POINTER(NNResult), c_void_p,
                                   c_size_t, c_void_p]),
    "nn_normal_workspace_bytes": (c_size_t, [c_int64, c_int64, c_int, c_int]),
    "nn_solve_normal": (c_int, [c_void_p, c_int64, c_int64, c_int, c_void_p, c_int64, c_int64, POINTER(NNOpts),
                                c_void_p, c_int64, POINTER(NNResult), c_void_p, c_size_t, c_void_p]),
    "nn_residual_noalloc": (c_int, [c_void_p, c_int64, c_void_p, c_int64, c_int64, POINTER(c_double), c_void_p]),
    "nn_server_request_bytes": (c_size_t, [c_int64, c_int64, c_int]),
    "nn_server_create": (c_int, [POINTER(NNServerOpts), POINTER(c_void_p)]),
    "nn_server_submit": (c_int, [c_void_p, POINTER(NNRequest)]),
    "nn_server_poll": (c_int, [c_void_p, POINTER(NNCompletion), c_int, POINTER(c_int)]),
    "nn_server_wait_idle": (c_int, [c_void_p, c_double]),
    "nn_server_stats": (c_int, [c_void_p, POINTER(c_size_t), POINTER(c_size_t), POINTER(c_int), POINTER(c_int)]),
    "nn_server_destroy": (c_int, [c_void_p]),
    "nn_batched_plan_size": (c_int64, [c_int64]),
    "nn_batched_plan": (c_int, [c_void_p, c_int64, c_void_p, c_void_p]),
    "nn_batched_plan_classes": (ctypes.c_uint32, [c_void_p]),
    "nn_batched_workspace_bytes": (c_size_t, [c_int64]),
    "nn_invert_batched_c64": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, ctypes.c_uint32, c_int, c_int,
                                      c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "nn_invert_batched": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int, c_int, c_double, c_void_p,
                                  ctypes.c_uint32, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "nn_csr_strip_workspace_bytes": (c_size_t, [c_int64]),
    "nn_csr_strip_diag_inv": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int, c_void_p, c_void_p,
                                      c_size_t, c_void_p]),
    "nn_csr_strip_scale": (c_int, [c_void_p, c_void_p, c_int64, c_int, c_void_p, c_void_p, c_void_p]),
    "nn_csr_strip_product": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "nn_csr_strip_residual": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int, c_void_p, c_void_p,
                                      POINTER(c_double), c_void_p, c_size_t, c_void_p]),
    "nn_csr_strip_finish": (c_int, [c_void_p, c_void_p, c_int64, c_int, c_void_p, c_void_p]),
    "nn_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_int64, c_int64, c_int, c_double,
                         POINTER(NNOpts), c_void_p, c_int64, POINTER(NNResult), c_void_p, c_size_t, c_void_p]),
    "nn_solve_csr": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int, c_void_p, c_int64, c_int64, c_int,
                             c_int, c_double, c_void_p, c_int64, POINTER(NNResult), c_void_p, c_size_t, c_void_p]),
}


def lib():
    """Loads libnn.so (built by ``paper_2212_02406_gb300.build``); raises if it is absent."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libnn.so not built ({LIB_PATH}); run python -m paper_2212_02406_gb300.build")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = handle
    return _LIB


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


# ---- marshalling helpers ---------------------------------------------------------------

def _stream_ptr(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _mat(t, name, dtype=None):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dim() != 2 or (t.stride(1) != 1 and t.shape[1] > 1):
        raise ValueError(f"{name} must be 2-D row-major (stride(1) == 1)")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    return c_void_p(t.data_ptr()), (t.stride(0) if t.shape[0] > 1 else t.shape[1])


def _ws(workspace):
    if workspace is None:
        return c_void_p(0), 0
    return c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()


NN_FLAG_TIME_KERNELS = 1


def make_opts(depth=2, tol=1e-6, max_nests=64, dtype="f64", refine_below=0.0, bulk_pieces=1,
              flags=0, depth_schedule=None, x0_scalar=0.0, fwd_tol=0.0) -> NNOpts:
    """depth_schedule: optional per-nest depths (the last one repeats), e.g. [2, 2, 1].
    x0_scalar > 0: the caller asserts X_0 = x0_scalar * I (the mixed dtypes then run the first
    nest's residual and update element-wise). fwd_tol > 0: stop once N s_k < fwd_tol, which bounds
    the relative Frobenius error of X against the inverse."""
    d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    o = NNOpts(int(depth), float(tol), int(max_nests), d, float(refine_below), int(bulk_pieces), int(flags))
    o.x0_scalar = float(x0_scalar)
    o.fwd_tol = float(fwd_tol)
    if depth_schedule:
        arr = (c_int32 * len(depth_schedule))(*[int(x) for x in depth_schedule])
        o.depth_schedule = ctypes.cast(arr, POINTER(c_int32))
        o.schedule_len = len(depth_schedule)
        o._schedule_keepalive = arr  # the C side reads the array during the call
    return o


def workspace(n: int, dtype="f64", host=False, device=None):
    """Device workspace (a uint8 CUDA tensor) sized by nn_workspace_bytes[_host]."""
    import torch

    d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    nbytes = (lib().nn_workspace_bytes_host if host else lib().nn_workspace_bytes)(int(n), d)
    if nbytes == 0:
        raise ValueError("invalid size or dtype")
    return torch.empty(int(nbytes), dtype=torch.uint8, device=device or "cuda")


# ---- entry points (same names as the C ABI) -------------------------------------------

def nn_debug_withhold_signal(on: bool = True) -> int:
    """Arms the failure-detection hook for the next tensor-core GEMM launch (its bounded wait runs
    out and the call reports NN_ERR_TIMEOUT)."""
    return int(lib().nn_debug_withhold_signal(1 if on else 0))


def nn_set_gemm_variant(variant: int) -> int:
    """0 automatic, 1 single-CTA tiles, 3 2-SM MMA, 4 2-SM MMA with the last wave split into halves
    (tensor-core GEMM tiling)."""
    return int(lib().nn_set_gemm_variant(int(variant)))


def nn_set_spmv_variant(variant: int) -> int:
    """0 automatic (bulk-copy ring for one right-hand side), 1 staged loads (sparse products)."""
    return int(lib().nn_set_spmv_variant(int(variant)))


def nn_workspace_bytes(n: int, dtype) -> int:
    d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    return int(lib().nn_workspace_bytes(int(n), d))


def nn_workspace_bytes_host(n: int, dtype) -> int:
    d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    return int(lib().nn_workspace_bytes_host(int(n), d))


def nn_init_precond(A, kind, scalar, X0, workspace, stream=None) -> int:
    import torch

    pa, lda = _mat(A, "A", torch.float64)
    px, ldx = _mat(X0, "X0", torch.float64)
    k = PRECONDS[kind] if isinstance(kind, str) else int(kind)
    pw, nw = _ws(workspace)
    return lib().nn_init_precond(pa, A.shape[0], lda, k, float(scalar), px, ldx, pw, nw, _stream_ptr(stream))


def nn_invert(A, X0, opts: NNOpts, X, workspace, stream=None):
    """Returns (status, result dict). X receives the last iterate."""
    import torch

    pa, lda = _mat(A, "A", torch.float64)
    p0, ld0 = _mat(X0, "X0", torch.float64)
    px, ldx = _mat(X, "X", torch.float64)
    pw, nw = _ws(workspace)
    res = NNResult()
    st = lib().nn_invert(pa, A.shape[0], lda, p0, ld0, ctypes.byref(opts), px, ldx, ctypes.byref(res), pw, nw,
                         _stream_ptr(stream))
    return st, res.as_dict()


def nn_invert_host(A, X0, opts: NNOpts, X, workspace, stream=None):
    """Host-buffer variant: A, X0, X are C-contiguous float64 NumPy arrays (X is written)."""
    import numpy as np

    for name, arr in (("A", A), ("X0", X0), ("X", X)):
        if not (isinstance(arr, np.ndarray) and arr.dtype == np.float64 and arr.flags.c_contiguous):
            raise TypeError(f"{name} must be a C-contiguous float64 ndarray")
    pw, nw = _ws(workspace)
    res = NNResult()
    st = lib().nn_invert_host(c_void_p(A.ctypes.data), A.shape[0], c_void_p(X0.ctypes.data), ctypes.byref(opts),
                              c_void_p(X.ctypes.data), ctypes.byref(res), pw, nw, _stream_ptr(stream))
    return st, res.as_dict()


def nn_invert_host_pc(A, kind, scalar, opts: NNOpts, X, workspace, stream=None):
    """Host-buffer inversion with X_0 built on the device (kind, scalar as nn_init_precond):
    A and X are C-contiguous float64 NumPy arrays (X is written)."""
    import numpy as np

    for name, arr in (("A", A), ("X", X)):
        if not (isinstance(arr, np.ndarray) and arr.dtype == np.float64 and arr.flags.c_contiguous):
            raise TypeError(f"{name} must be a C-contiguous float64 ndarray")
    k = PRECONDS[kind] if isinstance(kind, str) else int(kind)
    pw, nw = _ws(workspace)
    res = NNResult()
    st = lib().nn_invert_host_pc(c_void_p(A.ctypes.data), A.shape[0], k, float(scalar), ctypes.byref(opts),
                                 c_void_p(X.ctypes.data), ctypes.byref(res), pw, nw, _stream_ptr(stream))
    return st, res.as_dict()


def nn_residual(A, X, dtype, workspace, stream=None):
    """Returns (status, ||I - A X||_F / N)."""
    import torch

    pa, lda = _mat(A, "A", torch.float64)
    px, ldx = _mat(X, "X", torch.float64)
    d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    pw, nw = _ws(workspace)
    out = c_double(0.0)
    st = lib().nn_residual(pa, lda, px, ldx, A.shape[0], d, ctypes.byref(out), pw, nw, _stream_ptr(stream))
    return st, out.value


# ---- general systems through the normal equations -----------------------------------------

def nn_normal_workspace_bytes(n: int, nrhs: int, is_complex: bool, dtype) -> int:
    d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    return int(lib().nn_normal_workspace_bytes(int(n), int(nrhs), int(bool(is_complex)), d))


def normal_workspace(n: int, nrhs: int, is_complex: bool, dtype, device=None):
    import torch

    nbytes = nn_normal_workspace_bytes(n, nrhs, is_complex, dtype)
    if nbytes == 0:
        raise ValueError("invalid sizes or dtype")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def nn_solve_normal(A, B, opts: NNOpts, X, workspace, stream=None):
    """A X = B through the normal equations. A (n x n), B and X (n x nrhs): row-major CUDA
    tensors, all float64 or all complex128. Returns (status, result dict of the inversion of W)."""
    import torch

    if A.dtype not in (torch.float64, torch.complex128):
        raise TypeError("A must be float64 or complex128")
    pa, lda = _mat(A, "A", A.dtype)
    pb, ldb = _mat(B, "B", A.dtype)
    px, ldx = _mat(X, "X", A.dtype)
    n, nrhs = A.shape[0], B.shape[1]
    if A.shape[1] != n or B.shape[0] != n or tuple(X.shape) != tuple(B.shape):
        raise ValueError("A must be n x n, B and X n x nrhs")
    pw, nw = _ws(workspace)
    res = NNResult()
    st = lib().nn_solve_normal(pa, n, lda, int(A.dtype == torch.complex128), pb, ldb, nrhs, ctypes.byref(opts), px,
                               ldx, ctypes.byref(res), pw, nw, _stream_ptr(stream))
    return st, res.as_dict()


# ---- sparse chain ----------------------------------------------------------------------

def _vec_dtype(t):
    import torch

    if t.dtype == torch.float64:
        return NN_F64
    if t.dtype == torch.float32:
        return NN_F32
    raise TypeError("values must be float64 or float32")


def nn_csr_workspace_bytes(n: int, nnz: int, nrhs: int, dtype) -> int:
    d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    return int(lib().nn_csr_workspace_bytes(int(n), int(nnz), int(nrhs), d))


def csr_workspace(n: int, nnz: int, nrhs: int, dtype, device=None):
    import torch

    nbytes = nn_csr_workspace_bytes(n, nnz, nrhs, dtype)
    if nbytes == 0:
        raise ValueError("invalid CSR sizes or dtype")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def _csr_args(row_ptr, col, val, B, X, double_float):
    import torch

    for name, t in (("row_ptr", row_ptr), ("col", col)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous int32 CUDA tensor")
    d = _vec_dtype(val)
    if double_float:
        if d != NN_F64:
            raise TypeError("double_float needs float64 values")
        d = NN_F64_DF
    for name, t in (("B", B), ("X", X)):
        if not (t.is_cuda and t.dtype == val.dtype and t.dim() == 2 and t.stride(1) == 1):
            raise TypeError(f"{name} must be a (nrhs, n) row-major CUDA tensor of the value dtype")
    n = row_ptr.numel() - 1
    nrhs = B.shape[0]
    if B.shape[1] != n or X.shape != B.shape:
        raise ValueError("B and X must be (nrhs, n)")
    # a dimension of extent 1 may carry any stride: the leading dimension is then n
    ldb = B.stride(0) if nrhs > 1 else n
    ldx = X.stride(0) if nrhs > 1 else n
    return d, n, nrhs, ldb, ldx


def nn_solve_csr(row_ptr, col, val, B, depth, nests, tol, X, workspace, stream=None, double_float=False):
    """CSR (int32 row_ptr/col, float val) on the device; B and X are (nrhs, n) row-major
    tensors, i.e. column-major n x nrhs blocks with leading dimension n. Returns (status, result).
    double_float=True runs FP64 data in double-float arithmetic (NN_F64_DF)."""
    d, n, nrhs, ldb, ldx = _csr_args(row_ptr, col, val, B, X, double_float)
    pw, nw = _ws(workspace)
    res = NNResult()
    st = lib().nn_solve_csr(c_void_p(row_ptr.data_ptr()), c_void_p(col.data_ptr()), c_void_p(val.data_ptr()), n,
                            val.numel(), d, c_void_p(B.data_ptr()), ldb, nrhs, int(depth), int(nests),
                            float(tol), c_void_p(X.data_ptr()), ldx, ctypes.byref(res), pw, nw,
                            _stream_ptr(stream))
    return st, res.as_dict()


def nn_solve_csr_sched(row_ptr, col, val, B, depths, tol, X, workspace, stream=None, double_float=False):
    """nn_solve_csr with a depth per factor (e.g. [2, 2, 1, 1, 1]: the sparse CNS construction)."""
    d, n, nrhs, ldb, ldx = _csr_args(row_ptr, col, val, B, X, double_float)
    arr = (c_int32 * max(len(depths), 1))(*[int(x) for x in depths])
    pw, nw = _ws(workspace)
    res = NNResult()
    st = lib().nn_solve_csr_sched(c_void_p(row_ptr.data_ptr()), c_void_p(col.data_ptr()), c_void_p(val.data_ptr()),
                                  n, val.numel(), d, c_void_p(B.data_ptr()), ldb, nrhs, arr, len(depths),
                                  float(tol), c_void_p(X.data_ptr()), ldx, ctypes.byref(res), pw, nw,
                                  _stream_ptr(stream))
    return st, res.as_dict()


def nn_solve(row_ptr, col, val, B, depth, tol, opts, X, workspace, stream=None):
    """The sparse chain with the solve interface's argument order: opts (make_opts) supplies the
    dtype ("f64", "f64_df" or "f32"), max_nests (factors) and an optional per-factor depth
    schedule. Tensors as nn_solve_csr. Returns (status, result)."""
    d, n, nrhs, ldb, ldx = _csr_args(row_ptr, col, val, B, X, opts.dtype == NN_F64_DF)
    if opts.dtype != d:
        raise TypeError("opts.dtype does not match the value tensor")
    pw, nw = _ws(workspace)
    res = NNResult()
    st = lib().nn_solve(c_void_p(row_ptr.data_ptr()), c_void_p(col.data_ptr()), c_void_p(val.data_ptr()), n,
                        val.numel(), c_void_p(B.data_ptr()), ldb, nrhs, int(depth), float(tol), ctypes.byref(opts),
                        c_void_p(X.data_ptr()), ldx, ctypes.byref(res), pw, nw, _stream_ptr(stream))
    return st, res.as_dict()


# ---- row strips of the sparse chain --------------------------------------------------------

def _ptr(t):
    return None if t is None else c_void_p(t.data_ptr())


def nn_csr_strip_workspace_bytes(n_local: int) -> int:
    return int(lib().nn_csr_strip_workspace_bytes(int(n_local)))


def nn_csr_strip_diag_inv(row_ptr, col_local, val, dinv_local, workspace, stream=None) -> int:
    """dinv_local = 1 / diag of the strip's rows (device tensors; val float64 or float32)."""
    pw, nw = _ws(workspace)
    return int(lib().nn_csr_strip_diag_inv(_ptr(row_ptr), _ptr(col_local), _ptr(val), row_ptr.numel() - 1,
                                           val.numel(), _vec_dtype(val), _ptr(dinv_local), pw, nw,
                                           _stream_ptr(stream)))


def nn_csr_strip_scale(col_local, val, dinv_ext, val_scaled, stream=None) -> int:
    return int(lib().nn_csr_strip_scale(_ptr(col_local), _ptr(val), val.numel(), _vec_dtype(val), _ptr(dinv_ext),
                                        _ptr(val_scaled), _stream_ptr(stream)))


def nn_csr_strip_product(row_ptr, col_local, val_scaled, v_ext, y, workspace, acc_in=None, acc_out=None,
                         stream=None) -> int:
    """y = v_ext[:n_local] - A'_strip v_ext (and acc_out = acc_in + y when acc_out is given)."""
    pw, nw = _ws(workspace)
    return int(lib().nn_csr_strip_product(_ptr(row_ptr), _ptr(col_local), _ptr(val_scaled), row_ptr.numel() - 1,
                                          val_scaled.numel(), _vec_dtype(val_scaled), _ptr(v_ext), _ptr(y),
                                          _ptr(acc_in), _ptr(acc_out), pw, nw, _stream_ptr(stream)))


def nn_csr_strip_residual(row_ptr, col_local, val_scaled, z_ext, b_local, workspace, stream=None):
    """(status, [sum r^2, sum b^2]) over the strip, r = b - A' z."""
    pw, nw = _ws(workspace)
    out = (c_double * 2)()
    st = lib().nn_csr_strip_residual(_ptr(row_ptr), _ptr(col_local), _ptr(val_scaled), row_ptr.numel() - 1,
                                     val_scaled.numel(), _vec_dtype(val_scaled), _ptr(z_ext), _ptr(b_local), out, pw,
                                     nw, _stream_ptr(stream))
    return int(st), [out[0], out[1]]


def nn_csr_strip_finish(z_local, dinv_local, x_local, stream=None) -> int:
    return int(lib().nn_csr_strip_finish(_ptr(z_local), _ptr(dinv_local), z_local.numel(), _vec_dtype(z_local),
                                         _ptr(x_local), _stream_ptr(stream)))


# ---- batched small complex inversions -------------------------------------------------------

def nn_batched_plan(sizes, cfg_by_u=None):
    """Host plan for a size list (NumPy int32 array); returns the int32 plan array."""
    import numpy as np

    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    count = sizes.shape[0]
    plan = np.zeros(int(lib().nn_batched_plan_size(count)), dtype=np.int32)
    cfg = None
    if cfg_by_u is not None:
        cfg = np.full(65, -1, dtype=np.int32)
        for u, c in dict(cfg_by_u).items():
            cfg[int(u)] = int(c)
    st = lib().nn_batched_plan(c_void_p(sizes.ctypes.data), count,
                               c_void_p(cfg.ctypes.data) if cfg is not None else c_void_p(0), c_void_p(plan.ctypes.data))
    if st != NN_OK:
        raise ValueError(f"nn_batched_plan failed ({STATUS_NAMES.get(st, st)})")
    return plan


def nn_batched_plan_classes(plan) -> int:
    """Mask of the tile classes that hold items, from a host plan (NumPy int32 array)."""
    import numpy as np

    plan = np.ascontiguousarray(plan, dtype=np.int32)
    return int(lib().nn_batched_plan_classes(c_void_p(plan.ctypes.data)))


def nn_batched_workspace_bytes(count: int) -> int:
    return int(lib().nn_batched_workspace_bytes(int(count)))


def nn_invert_batched_c64(A, offsets, sizes, plan, depth, nests, damping, X, residual, status, workspace,
                          stream=None, classes=0xFFFFFFFF) -> int:
    """A, X: complex64 CUDA tensors (packed); offsets int64, sizes int32, plan int32, residual float32,
    status int32 CUDA tensors; classes = nn_batched_plan_classes of the host plan (default: all).
    Enqueues only (graph-capturable); returns the status code."""
    import torch

    if A.dtype != torch.complex64 or X.dtype != torch.complex64 or not (A.is_cuda and X.is_cuda):
        raise TypeError("A and X must be complex64 CUDA tensors")
    checks = ((offsets, torch.int64), (sizes, torch.int32), (plan, torch.int32), (residual, torch.float32),
              (status, torch.int32))
    for t, dt in checks:
        if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError(f"expected contiguous CUDA {dt}")
    pw, nw = _ws(workspace)
    return lib().nn_invert_batched_c64(c_void_p(A.data_ptr()), c_void_p(offsets.data_ptr()),
                                       c_void_p(sizes.data_ptr()), sizes.numel(), c_void_p(plan.data_ptr()),
                                       int(classes) & 0xFFFFFFFF, int(depth), int(nests), float(damping),
                                       c_void_p(X.data_ptr()),
                                       c_void_p(residual.data_ptr()), c_void_p(status.data_ptr()), pw, nw,
                                       _stream_ptr(stream))


def nn_invert_batched(A, offsets, sizes, depth, nests, damping, plan, X, residual, status, workspace,
                      stream=None, classes=0xFFFFFFFF) -> int:
    """nn_invert_batched_c64 with the batched interface's argument order (same tensors)."""
    import torch

    if A.dtype != torch.complex64 or X.dtype != torch.complex64 or not (A.is_cuda and X.is_cuda):
        raise TypeError("A and X must be complex64 CUDA tensors")
    checks = ((offsets, torch.int64), (sizes, torch.int32), (plan, torch.int32), (residual, torch.float32),
              (status, torch.int32))
    for t, dt in checks:
        if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError(f"expected contiguous CUDA {dt}")
    pw, nw = _ws(workspace)
    return lib().nn_invert_batched(c_void_p(A.data_ptr()), c_void_p(offsets.data_ptr()), c_void_p(sizes.data_ptr()),
                                   sizes.numel(), int(depth), int(nests), float(damping), c_void_p(plan.data_ptr()),
                                   int(classes) & 0xFFFFFFFF, c_void_p(X.data_ptr()), c_void_p(residual.data_ptr()),
                                   c_void_p(status.data_ptr()), pw, nw, _stream_ptr(stream))


# ---- residual without allocation ---------------------------------------------------------

def nn_residual_noalloc(A, X, stream=None):
    """FP64 s = ||I - A X||_F / N using the library's fixed device scratch (no workspace).

    For callers that cannot allocate device memory; N <= NN_RESIDUAL_NOALLOC_MAX_N.
    Returns (status, s)."""
    import torch

    pa, lda = _mat(A, "A", torch.float64)
    px, ldx = _mat(X, "X", torch.float64)
    out = c_double(0.0)
    st = lib().nn_residual_noalloc(pa, lda, px, ldx, A.shape[0], ctypes.byref(out), _stream_ptr(stream))
    return st, out.value


# ---- serving -------------------------------------------------------------------------------

def nn_server_request_bytes(n, nrhs, dtype) -> int:
    d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    return int(lib().nn_server_request_bytes(int(n), int(nrhs), d))


class Server:
    """Marshalling wrapper of nn_server_*: keeps the host arrays of in-flight requests alive."""

    def __init__(self, arena, max_active=4, depth=2, tol=1e-6, max_nests=64):
        self.arena = arena
        opts = NNServerOpts(c_void_p(arena.data_ptr()), arena.numel() * arena.element_size(), int(max_active),
                            int(depth), float(tol), int(max_nests))
        h = c_void_p()
        st = lib().nn_server_create(ctypes.byref(opts), ctypes.byref(h))
        if st != NN_OK:
            raise RuntimeError(f"nn_server_create failed ({STATUS_NAMES.get(st, st)})")
        self.h = h
        self.live = {}

    def submit(self, rid, A, B=None, Y=None, X=None, dtype="f32", precond="trace", pc_scalar=1.0) -> int:
        import numpy as np

        for name, arr in (("A", A), ("B", B), ("Y", Y), ("X", X)):
            if arr is not None and not (isinstance(arr, np.ndarray) and arr.dtype == np.float64
                                        and arr.flags.c_contiguous):
                raise TypeError(f"{name} must be a C-contiguous float64 ndarray")
        d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        k = PRECONDS[precond] if isinstance(precond, str) else int(precond)
        nrhs = 0 if B is None else B.shape[1]
        req = NNRequest(int(rid), A.shape[0], c_void_p(A.ctypes.data), nrhs,
                        c_void_p(B.ctypes.data) if B is not None else c_void_p(0),
                        c_void_p(Y.ctypes.data) if Y is not None else c_void_p(0),
                        c_void_p(X.ctypes.data) if X is not None else c_void_p(0), d, k, float(pc_scalar))
        st = lib().nn_server_submit(self.h, ctypes.byref(req))
        if st == NN_OK:
            self.live[int(rid)] = (A, B, Y, X)
        return st

    def poll(self, max_out=256):
        buf = (NNCompletion * max_out)()
        cnt = c_int(0)
        lib().nn_server_poll(self.h, buf, max_out, ctypes.byref(cnt))
        out = []
        for i in range(cnt.value):
            c = buf[i]
            self.live.pop(int(c.id), None)
            out.append({"id": c.id, "status": c.status, "nests": c.nests, "residual": c.residual,
                        "t_submit": c.t_submit, "t_start": c.t_start, "t_done": c.t_done,
                        "launches": c.launches})
        return out

    def wait_idle(self, timeout_s=0.0) -> int:
        return lib().nn_server_wait_idle(self.h, float(timeout_s))

    def stats(self):
        used, peak = c_size_t(), c_size_t()
        pend, act = c_int(), c_int()
        lib().nn_server_stats(self.h, ctypes.byref(used), ctypes.byref(peak), ctypes.byref(pend), ctypes.byref(act))
        return {"arena_used": used.value, "arena_peak": peak.value, "pending": pend.value, "active": act.value}

    def close(self):
        if self.h:
            lib().nn_server_destroy(self.h)
            self.h = None
