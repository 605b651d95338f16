"""Python binding of the M-HDC SpMV library (include/mhdc.h).

Argument marshalling only: every function passes device pointers (from torch
tensors), sizes and the current CUDA stream to the C ABI of the same name;
every step of the computation runs in the library's sm_103a kernels.  There
is no CPU path: if the compiled library is missing, or no GPU is present, the
compute calls raise.

Method: Fukaya et al., "Accelerating the SpMV kernel on standard CPUs by
exploiting the partially diagonal structures" (arXiv 2105.04937), Sec. 4.3.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import SO, build as _build_library  # noqa: F401  (re-exported for build steps)

__all__ = [
    "MHDC_F64", "MHDC_F32", "MHDC_BF16", "MhdcError", "Matrix", "lib", "mhdc_build",
    "hdc_build", "mhdc_build_dia", "mhdc_dia_spmv", "mhdc_spmv_host_async", "mhdc_host_wait",
    "Sell", "sell_build", "sell_spmv", "sell_info", "sell_export", "sell_destroy", "mhdc_spmv",
    "mhdc_spmv_host", "mhdc_spmm", "mhdc_spmm_set_variant", "mhdc_spmm_tune",
    "MHDC_NUM_SPMM_VARIANTS", "csr_spmv", "mhdc_export",
    "mhdc_info", "mhdc_stats", "mhdc_destroy", "mhdc_strerror", "mhdc_stream_bench", "DTYPES",
    "mhdc_set_variant", "mhdc_tune", "MHDC_NUM_VARIANTS", "NATIVE_VARIANTS",
    "EMULATED_VARIANTS", "XW_VARIANTS", "FIRST_EMULATED_VARIANT", "mhdc_check",
    "mhdc_read_bench", "mhdc_read_bench_ctas", "mhdc_build_noalloc",
    "mhdc_fma_bench", "Batch", "mhdc_batch_create", "mhdc_batch_spmv", "mhdc_batch_spmv_graph",
    "mhdc_batch_destroy", "pointer_array", "MHDC_NUM_FEATURES", "MHDC_NUM_CANDIDATES",
    "MHDC_SELECT_PAPER", "MHDC_SELECT_MLP", "MHDC_SELECT_AUTOTUNE", "MHDC_SELECT_MODEL",
    "mhdc_candidate", "mhdc_features", "mhdc_autotune", "mhdc_select", "Mlp",
    "mhdc_mlp_create", "mhdc_mlp_forward", "mhdc_mlp_grad", "mhdc_mlp_train_step",
    "mhdc_mlp_get_params", "mhdc_mlp_set_params", "mhdc_mlp_destroy", "mhdc_num_candidates",
    "mhdc_mlp_num_params", "mhdc_debug_fail_alloc", "mhdc_debug_alloc_stats", "mhdc_set_checked",
]

MHDC_F64, MHDC_F32, MHDC_BF16 = 0, 1, 2
DTYPES = {"f64": MHDC_F64, "f32": MHDC_F32, "bf16": MHDC_BF16}
(MHDC_OK, MHDC_ERR_INVALID_ARG, MHDC_ERR_BAD_CSR, MHDC_ERR_OOM, MHDC_ERR_CUDA,
 MHDC_ERR_UNSUPPORTED, MHDC_ERR_DEVICE_CHECK, MHDC_ERR_TIMEOUT) = 0, -1, -2, -3, -4, -5, -6, -7
_NP_STORE = {MHDC_F64: np.float64, MHDC_F32: np.float32, MHDC_BF16: np.uint16}

_lock = threading.Lock()
_lib = None


class MhdcError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: {mhdc_strerror(code)} ({code})" + (f": {detail}" if detail else ""))


class _Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("nnz_rem", C.c_int64), ("P", C.c_int64),
                ("n_blocks", C.c_int64), ("n_b", C.c_int32), ("dtype", C.c_int32),
                ("mode", C.c_int32), ("variant", C.c_int32), ("emulated_ok", C.c_int32),
                ("reserved", C.c_int32), ("theta", C.c_double),
                ("alpha", C.c_double), ("beta", C.c_double), ("bytes_model", C.c_int64),
                ("bytes_device", C.c_int64)]


_P, _I64, _I32, _D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
_SIGS = {
    "mhdc_build": [_I64, _P, _P, _P, _I32, _D, _I32, _P, C.POINTER(C.c_void_p)],
    "hdc_build": [_I64, _P, _P, _P, _I32, _D, _I32, _P, C.POINTER(C.c_void_p)],
    "mhdc_build_dia": [_I64, _I32, _P, _P, _I32, _D, _I32, _P, C.POINTER(C.c_void_p)],
    "sell_build": [_I64, _P, _P, _P, _I32, _I32, _P, C.POINTER(C.c_void_p)],
    "sell_spmv": [_P, _P, _P, _P],
    "sell_info": [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64)],
    "sell_export": [_P, _P, _P, _P, _P, _P],
    "sell_destroy": [_P],
    "mhdc_spmv": [_P, _P, _P, _P],
    "mhdc_spmv_host": [_P, _P, _P, _P],
    "mhdc_spmv_host_async": [_P, _P, _P],
    "mhdc_host_wait": [_P],
    "mhdc_dia_spmv": [_P, _P, _P, _P],
    "mhdc_spmm": [_P, _I32, _P, _I64, _P, _I64, _P],
    "mhdc_spmm_set_variant": [_P, _I32],
    "mhdc_spmm_tune": [_P, _I32, _P, _I64, _P, _I64, _P, C.POINTER(C.c_int32),
                       C.POINTER(C.c_float)],
    "csr_spmv": [_I64, _P, _P, _P, _P, _P, _P],
    "mhdc_export": [_P, _P, _P, _P, _P, _P, _P],
    "mhdc_info": [_P, C.POINTER(_Info)],
    "mhdc_stats": [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int64),
                   C.POINTER(C.c_int64)],
    "mhdc_destroy": [_P],
    "mhdc_strerror": [C.c_int],
    "mhdc_last_error": [],
    "mhdc_stream_bench": [_I64, _P, _P, _P, _P, _I32, _P],
    "mhdc_set_variant": [_P, _I32],
    "mhdc_check": [_P],
    "mhdc_set_checked": [_P, _I32],
    "mhdc_read_bench": [_I64, _P, _P, _P],
    "mhdc_read_bench_ctas": [],
    "mhdc_fma_bench": [_I32, _I32, _P, _P],
    "mhdc_batch_create": [_I32, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)],
    "mhdc_batch_spmv": [_P, _P, _P, _P],
    "mhdc_batch_spmv_graph": [_P, _P, _P, _P],
    "mhdc_batch_destroy": [_P],
    "mhdc_num_candidates": [],
    "mhdc_candidate": [_I32, _P],
    "mhdc_features": [_I64, _P, _P, _P, _P],
    "mhdc_autotune": [_I64, _P, _P, _P, _I32, _P, _P],
    "mhdc_select": [_I64, _P, _P, _P, _D, _I32, _P, _P, _P],
    "mhdc_mlp_create": [_I32, _I32, _I32, C.c_uint64, C.POINTER(C.c_void_p)],
    "mhdc_mlp_num_params": [_P],
    "mhdc_mlp_get_params": [_P, _P],
    "mhdc_mlp_set_params": [_P, _P],
    "mhdc_mlp_forward": [_P, _I32, _P, _P, _P],
    "mhdc_mlp_grad": [_P, _I32, _P, _P, _P, _P, _P, _P],
    "mhdc_mlp_train_step": [_P, _I32, _P, _P, _P, C.c_float, _P, _P],
    "mhdc_mlp_destroy": [_P],
    "mhdc_build_noalloc": [_I64, _P, _P, _P, _I32, _D, _I32, _P, _P, _P, _I64, _P, _P, _P, _I64,
                           C.POINTER(C.c_int64), C.POINTER(C.c_int64), _P],
    "mhdc_tune": [_P, _P, _P, _P, C.POINTER(C.c_int32), C.POINTER(C.c_float)],
    "mhdc_debug_fail_alloc": [_I64],
    "mhdc_debug_alloc_stats": [C.POINTER(_I64), C.POINTER(_I64)],
}

MHDC_NUM_VARIANTS = 20
MHDC_NUM_SPMM_VARIANTS = 4
MHDC_NUM_FEATURES = 64
MHDC_NUM_CANDIDATES = 45
MHDC_SELECT_PAPER, MHDC_SELECT_MLP, MHDC_SELECT_AUTOTUNE, MHDC_SELECT_MODEL = 0, 1, 2, 4
FIRST_EMULATED_VARIANT = 10
EMULATED_VARIANTS = tuple(range(10, 16))  # FP64 handles: FP32-pair arithmetic
NATIVE_VARIANTS = tuple(range(0, 10)) + tuple(range(16, 20))  # the handle's own arithmetic
XW_VARIANTS = tuple(range(16, 20))        # values and x staged in shared memory by TMA


def lib(build_if_missing: bool = False):
    """The loaded library; raises if it has not been compiled (see build.py)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO):
                if not build_if_missing:
                    raise RuntimeError(
                        f"M-HDC CUDA library not built ({SO} missing): run "
                        "paper_2105_04937_gb300.build.build() (or __graft_entry__.build())")
                _build_library()
            L = C.CDLL(SO)
            for name, args in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = (C.c_char_p if name in ("mhdc_strerror", "mhdc_last_error") else
                             C.c_int64 if name == "mhdc_mlp_num_params" else C.c_int)
            _lib = L
    return _lib


def mhdc_strerror(code: int) -> str:
    return lib().mhdc_strerror(code).decode()


def _check(rc: int, where: str):
    if rc != 0:
        raise MhdcError(rc, where, lib().mhdc_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def _check_dev(t, dtype, n=None, name="array"):
    import torch
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n}")
    del torch


class Matrix:
    """Owner of an mhdc_handle (freed by destroy() or when collected)."""

    def __init__(self, handle: int, n: int):
        self.handle = handle
        self.n = n
        self._info = None

    @property
    def info(self) -> dict:
        if self._info is None:
            self._info = mhdc_info(self)
        return self._info

    @property
    def dtype(self) -> int:
        return self.info["dtype"]

    def destroy(self):
        if self.handle:
            lib().mhdc_destroy(C.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


def _build(fn, n, row_ptr, col, val, n_b, theta, dtype, stream):
    import torch
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    _check_dev(row_ptr, torch.int32, n + 1, "row_ptr")
    _check_dev(col, torch.int32, None, "col")
    _check_dev(val, torch.float64, None, "val")
    h = C.c_void_p()
    rc = getattr(lib(), fn)(n, _ptr(row_ptr), _ptr(col), _ptr(val), int(n_b), float(theta),
                            int(dtype), _stream(stream), C.byref(h))
    _check(rc, fn)
    return Matrix(h.value, n)


def mhdc_build(n, row_ptr, col, val, n_b, theta, dtype="f64", stream=None) -> Matrix:
    """CSR (device int32 row_ptr/col, float64 val) -> M-HDC handle (Sec. 4.3)."""
    return _build("mhdc_build", n, row_ptr, col, val, n_b, theta, dtype, stream)


def hdc_build(n, row_ptr, col, val, n_b, theta, dtype="f64", stream=None) -> Matrix:
    """CSR -> HDC (global selection, Sec. 3.4) stored blocked for the B-HDC kernel."""
    return _build("hdc_build", n, row_ptr, col, val, n_b, theta, dtype, stream)


def mhdc_build_dia(n, offsets, dia_val, n_b, theta, dtype="f64", stream=None) -> Matrix:
    """DIA input (device int32 offsets[nd], float64 dia_val[nd, n] with
    dia_val[d, i] = a(i, i + offsets[d])) -> M-HDC handle, without CSR."""
    import torch
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    nd = int(offsets.numel())
    _check_dev(offsets, torch.int32, nd, "offsets")
    _check_dev(dia_val, torch.float64, nd * n, "dia_val")
    h = C.c_void_p()
    rc = lib().mhdc_build_dia(n, nd, _ptr(offsets), _ptr(dia_val), int(n_b), float(theta),
                              int(dtype), _stream(stream), C.byref(h))
    _check(rc, "mhdc_build_dia")
    return Matrix(h.value, n)


class Sell:
    """A SELL-C-sigma handle (device memory freed by destroy() or on collection)."""

    def __init__(self, handle: int, n: int):
        self.handle = handle
        self.n = n

    @property
    def info(self) -> dict:
        return sell_info(self)

    def destroy(self):
        if self.handle:
            lib().sell_destroy(C.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sell_build(n, row_ptr, col, val, C_=32, sigma=256, stream=None) -> Sell:
    """CSR (device int32 row_ptr/col, float64 val) -> SELL-C-sigma handle."""
    import torch
    _check_dev(row_ptr, torch.int32, n + 1, "row_ptr")
    _check_dev(col, torch.int32, None, "col")
    _check_dev(val, torch.float64, None, "val")
    h = C.c_void_p()
    _check(lib().sell_build(n, _ptr(row_ptr), _ptr(col), _ptr(val), int(C_), int(sigma),
                            _stream(stream), C.byref(h)), "sell_build")
    return Sell(h.value, n)


def sell_spmv(S: Sell, x, y, stream=None):
    """y = A x with the SELL-C-sigma kernel (FP64)."""
    import torch
    _check_dev(x, torch.float64, S.n, "x")
    _check_dev(y, torch.float64, S.n, "y")
    _check(lib().sell_spmv(C.c_void_p(S.handle), _ptr(x), _ptr(y), _stream(stream)), "sell_spmv")
    return y


def sell_info(S: Sell) -> dict:
    v = [C.c_int64() for _ in range(4)]
    _check(lib().sell_info(C.c_void_p(S.handle), *[C.byref(a) for a in v]), "sell_info")
    return dict(zip(("n", "nnz", "slots", "chunks"), (a.value for a in v)))


def sell_export(S: Sell) -> dict:
    inf = sell_info(S)
    n, c, s = inf["n"], inf["chunks"], inf["slots"]
    out = {"perm": np.zeros(n, np.int32), "rowlen": np.zeros(n, np.int32),
           "chunk_ptr": np.zeros(c + 1, np.int32), "col": np.zeros(max(s, 1), np.int32),
           "val": np.zeros(max(s, 1), np.float64)}
    _check(lib().sell_export(C.c_void_p(S.handle), *[out[k].ctypes.data_as(C.c_void_p)
                                                      for k in ("perm", "rowlen", "chunk_ptr",
                                                                "col", "val")]), "sell_export")
    out["col"], out["val"] = out["col"][:s], out["val"][:s]
    return out


def sell_destroy(S: Sell):
    S.destroy()


def _xy_types(A: Matrix):
    import torch
    d = A.dtype
    xt = {MHDC_F64: torch.float64, MHDC_F32: torch.float32, MHDC_BF16: torch.bfloat16}[d]
    yt = torch.float64 if d == MHDC_F64 else torch.float32
    return xt, yt


def mhdc_spmv(A: Matrix, x, y, stream=None):
    """y = A x on the device (Fig. 13)."""
    xt, yt = _xy_types(A)
    _check_dev(x, xt, A.n, "x")
    _check_dev(y, yt, A.n, "y")
    _check(lib().mhdc_spmv(C.c_void_p(A.handle), _ptr(x), _ptr(y), _stream(stream)), "mhdc_spmv")
    return y


def mhdc_spmv_host_async(A: Matrix, x, y):
    """Queue y = A x on pinned host tensors (three calls in flight; see the C
    header for when x and y may be reused).  mhdc_host_wait(A) drains."""
    xt, yt = _xy_types(A)
    for t, dt, nm in ((x, xt, "x"), (y, yt, "y")):
        if t.is_cuda or t.dtype != dt or not t.is_contiguous() or t.numel() < A.n:
            raise ValueError(f"{nm} must be a contiguous host tensor of {dt} with n elements")
    _check(lib().mhdc_spmv_host_async(C.c_void_p(A.handle), _ptr(x), _ptr(y)),
           "mhdc_spmv_host_async")
    return y


def mhdc_host_wait(A: Matrix):
    _check(lib().mhdc_host_wait(C.c_void_p(A.handle)), "mhdc_host_wait")


def mhdc_dia_spmv(A: Matrix, x, y, stream=None):
    """y = A x in the unblocked DIA order (Fig. 5); A must come from hdc_build."""
    xt, yt = _xy_types(A)
    _check_dev(x, xt, A.n, "x")
    _check_dev(y, yt, A.n, "y")
    _check(lib().mhdc_dia_spmv(C.c_void_p(A.handle), _ptr(x), _ptr(y), _stream(stream)),
           "mhdc_dia_spmv")
    return y


def mhdc_spmv_host(A: Matrix, x, y, stream=None):
    """y = A x with host (CPU, preferably pinned) torch tensors x and y."""
    xt, yt = _xy_types(A)
    for t, dt, nm in ((x, xt, "x"), (y, yt, "y")):
        if t.is_cuda or t.dtype != dt or not t.is_contiguous() or t.numel() < A.n:
            raise ValueError(f"{nm} must be a contiguous host tensor of {dt} with n elements")
    _check(lib().mhdc_spmv_host(C.c_void_p(A.handle), _ptr(x), _ptr(y), _stream(stream)),
           "mhdc_spmv_host")
    return y


def _spmm_args(A: Matrix, X, Y):
    xt, yt = _xy_types(A)
    for t, dt, nm in ((X, xt, "X"), (Y, yt, "Y")):
        if not t.is_cuda or t.dtype != dt:
            raise TypeError(f"{nm} must be a CUDA tensor of {dt}")
        if t.dim() != 2 or t.stride(1) != 1 or t.shape[0] < A.n:
            raise ValueError(f"{nm} must be n x k with unit column stride")
    if X.shape[1] != Y.shape[1]:
        raise ValueError("X and Y must have the same number of columns")
    return X.shape[1]


def mhdc_spmm(A: Matrix, X, Y, stream=None):
    """Y = A X for row-major n x k device tensors X and Y."""
    k = _spmm_args(A, X, Y)
    _check(lib().mhdc_spmm(C.c_void_p(A.handle), k, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0),
                           _stream(stream)), "mhdc_spmm")
    return Y


def mhdc_spmm_set_variant(A: Matrix, v: int):
    """SpMM tile shape v (0..MHDC_NUM_SPMM_VARIANTS-1, -1: default)."""
    _check(lib().mhdc_spmm_set_variant(C.c_void_p(A.handle), int(v)), "mhdc_spmm_set_variant")


def mhdc_spmm_tune(A: Matrix, X, Y, stream=None):
    """Time every SpMM tile shape on (X, Y); keep the fastest.  Returns
    (best, per-shape microseconds)."""
    k = _spmm_args(A, X, Y)
    best = C.c_int32(-1)
    times = (C.c_float * MHDC_NUM_SPMM_VARIANTS)()
    _check(lib().mhdc_spmm_tune(C.c_void_p(A.handle), k, _ptr(X), X.stride(0), _ptr(Y),
                                Y.stride(0), _stream(stream), C.byref(best), times),
           "mhdc_spmm_tune")
    return best.value, list(times)


def csr_spmv(n, row_ptr, col, val, x, y, stream=None):
    """The plain FP64 CSR kernel (Fig. 2) on device tensors (the CSR is not
    validated: pass arrays that mhdc_build would accept)."""
    import torch
    _check_dev(row_ptr, torch.int32, n + 1, "row_ptr")
    _check_dev(col, torch.int32, None, "col")
    _check_dev(val, torch.float64, None, "val")
    _check_dev(x, torch.float64, n, "x")
    _check_dev(y, torch.float64, n, "y")
    _check(lib().csr_spmv(n, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(x), _ptr(y),
                          _stream(stream)), "csr_spmv")
    return y


def mhdc_stats(A: Matrix) -> dict:
    """alpha, beta, P and the model bytes of one product (Sec. 5.3)."""
    a, b = C.c_double(), C.c_double()
    p, by = C.c_int64(), C.c_int64()
    _check(lib().mhdc_stats(C.c_void_p(A.handle), C.byref(a), C.byref(b), C.byref(p), C.byref(by)),
           "mhdc_stats")
    return {"alpha": a.value, "beta": b.value, "P": p.value, "bytes": by.value}


def mhdc_info(A: Matrix) -> dict:
    inf = _Info()
    _check(lib().mhdc_info(C.c_void_p(A.handle), C.byref(inf)), "mhdc_info")
    return {name: getattr(inf, name) for name, _ in _Info._fields_ if name != "reserved"}


def mhdc_export(A: Matrix) -> dict:
    """Copy the handle's arrays to host numpy arrays (parity checks)."""
    inf = A.info
    sd = _NP_STORE[inf["dtype"]]
    out = dict(
        dia_ptr=np.zeros(inf["n_blocks"] + 1, np.int32),
        dia_offset=np.zeros(max(1, inf["P"]), np.int32),
        dia_val=np.zeros(max(1, inf["P"] * inf["n_b"]), sd),
        csr_row_ptr=np.zeros(inf["n"] + 1, np.int32),
        csr_col=np.zeros(max(1, inf["nnz_rem"]), np.int32),
        csr_val=np.zeros(max(1, inf["nnz_rem"]), sd),
    )
    rc = lib().mhdc_export(C.c_void_p(A.handle), *(out[k].ctypes.data_as(C.c_void_p) for k in
                                                   ("dia_ptr", "dia_offset", "dia_val",
                                                    "csr_row_ptr", "csr_col", "csr_val")))
    _check(rc, "mhdc_export")
    out["dia_offset"] = out["dia_offset"][:inf["P"]]
    out["dia_val"] = out["dia_val"][:inf["P"] * inf["n_b"]]
    out["csr_col"] = out["csr_col"][:inf["nnz_rem"]]
    out["csr_val"] = out["csr_val"][:inf["nnz_rem"]]
    return out


def mhdc_destroy(A: Matrix):
    A.destroy()


def mhdc_stream_bench(A, B, I, Cv, indirect: bool, stream=None):
    """C += A * B (or A * B[I]) on device float64 tensors (Sec. 6.2)."""
    import torch
    N = Cv.numel()
    for t, nm in ((A, "A"), (B, "B"), (Cv, "C")):
        _check_dev(t, torch.float64, N, nm)
    if indirect:
        _check_dev(I, torch.int32, N, "I")
    _check(lib().mhdc_stream_bench(N, _ptr(A), _ptr(B), _ptr(I) if indirect else None, _ptr(Cv),
                                   1 if indirect else 0, _stream(stream)), "mhdc_stream_bench")
    return Cv


def mhdc_set_variant(A: Matrix, v: int):
    """Select the SpMV tile shape (-1: default from n_b)."""
    _check(lib().mhdc_set_variant(C.c_void_p(A.handle), int(v)), "mhdc_set_variant")
    A._info = None


def mhdc_tune(A: Matrix, x, y, stream=None):
    """Time every tile shape on (x, y); keep the fastest.  Returns
    (best id, list of mean times in microseconds)."""
    xt, yt = _xy_types(A)
    _check_dev(x, xt, A.n, "x")
    _check_dev(y, yt, A.n, "y")
    best = C.c_int32(-1)
    times = (C.c_float * MHDC_NUM_VARIANTS)()
    _check(lib().mhdc_tune(C.c_void_p(A.handle), _ptr(x), _ptr(y), _stream(stream),
                           C.byref(best), times), "mhdc_tune")
    A._info = None
    return best.value, [float(t) for t in times]


def mhdc_set_checked(A: Matrix, on: bool = True):
    """Products of this handle run the bounds-checked kernel (see mhdc.h)."""
    _check(lib().mhdc_set_checked(C.c_void_p(A.handle), 1 if on else 0), "mhdc_set_checked")


def mhdc_check(A: Matrix):
    """Raise MhdcError(MHDC_ERR_TIMEOUT) if a bounded device wait gave up."""
    _check(lib().mhdc_check(C.c_void_p(A.handle)), "mhdc_check")


def mhdc_read_bench_ctas() -> int:
    return int(lib().mhdc_read_bench_ctas())


def mhdc_read_bench(A, out, stream=None):
    """Read-only bandwidth probe: out[c] = XOR of the 64-bit words of CTA c's
    share of A (A float64, out int64)."""
    import torch
    _check_dev(A, torch.float64, None, "A")
    _check_dev(out, torch.int64, mhdc_read_bench_ctas(), "out")
    _check(lib().mhdc_read_bench(A.numel(), _ptr(A), _ptr(out), _stream(stream)), "mhdc_read_bench")
    return out


def _noalloc_check(n, nnz, row_ptr, col, val, n_b, dtype, dia_ptr, dia_offset, dia_val,
                   csr_row_ptr, csr_col, csr_val):
    """Argument checks of mhdc_build_noalloc, done before anything runs on the
    GPU: the C layer receives raw pointers and cannot check lengths or
    placement, and a short or host-side array would be written out of bounds.
    nnz = row_ptr[n] (read by the caller)."""
    import torch
    if n < 1 or n_b < 1:
        raise ValueError("n and n_b must be >= 1")
    if nnz < 0:
        raise ValueError("row_ptr[n] must be >= 0")
    store = {MHDC_F64: (torch.float64,), MHDC_F32: (torch.float32,),
             MHDC_BF16: (torch.bfloat16, torch.int16)}[dtype]
    nb = (n + n_b - 1) // n_b
    _check_dev(row_ptr, torch.int32, n + 1, "row_ptr")
    _check_dev(col, torch.int32, nnz, "col")
    _check_dev(val, torch.float64, nnz, "val")
    _check_dev(dia_ptr, torch.int32, nb + 1, "dia_ptr")
    _check_dev(dia_offset, torch.int32, None, "dia_offset")
    _check_dev(csr_row_ptr, torch.int32, n + 1, "csr_row_ptr")
    _check_dev(csr_col, torch.int32, None, "csr_col")
    for t, nm in ((dia_val, "dia_val"), (csr_val, "csr_val")):
        if t.dtype not in store:
            raise TypeError(f"{nm} must be {' or '.join(map(str, store))} for this dtype, "
                            f"got {t.dtype}")
        _check_dev(t, t.dtype, None, nm)
    cap_P = dia_offset.numel()
    if dia_val.numel() < cap_P * n_b:
        raise ValueError("dia_val must hold dia_offset.numel() * n_b values")
    dev = row_ptr.device
    for t, nm in ((col, "col"), (val, "val"), (dia_ptr, "dia_ptr"), (dia_offset, "dia_offset"),
                  (dia_val, "dia_val"), (csr_row_ptr, "csr_row_ptr"), (csr_col, "csr_col"),
                  (csr_val, "csr_val")):
        if t.device != dev:
            raise ValueError(f"{nm} is on {t.device}, row_ptr on {dev}")
    return cap_P, min(csr_col.numel(), csr_val.numel())


def mhdc_build_noalloc(n, row_ptr, col, val, n_b, theta, dtype, dia_ptr, dia_offset, dia_val,
                       csr_row_ptr, csr_col, csr_val, stream=None):
    """mhdc_build into caller-owned device tensors, allocating no device memory.

    Output tensors: dia_ptr int32[ceil(n/n_b)+1], dia_offset int32[cap_P],
    dia_val (float64 / float32 / bfloat16 or int16 bits)[cap_P * n_b],
    csr_row_ptr int32[n+1], csr_col int32[cap_rem], csr_val[cap_rem]; every
    tensor on row_ptr's device.  Returns (P, nnz_rem).  Limits and sharing
    rules: see include/mhdc.h."""
    import torch
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    _check_dev(row_ptr, torch.int32, n + 1, "row_ptr")
    with torch.cuda.device(row_ptr.device):
        nnz = int(row_ptr[n].item()) if n >= 1 else 0
    cap_P, cap_rem = _noalloc_check(n, nnz, row_ptr, col, val, int(n_b), dtype, dia_ptr,
                                    dia_offset, dia_val, csr_row_ptr, csr_col, csr_val)
    P = C.c_int64(0)
    R = C.c_int64(0)
    with torch.cuda.device(row_ptr.device):
        rc = lib().mhdc_build_noalloc(n, _ptr(row_ptr), _ptr(col), _ptr(val), int(n_b),
                                      float(theta), int(dtype), _ptr(dia_ptr), _ptr(dia_offset),
                                      _ptr(dia_val), cap_P, _ptr(csr_row_ptr), _ptr(csr_col),
                                      _ptr(csr_val), cap_rem, C.byref(P), C.byref(R),
                                      _stream(stream))
    _check(rc, "mhdc_build_noalloc")
    return P.value, R.value


def mhdc_debug_fail_alloc(n: int):
    """Make the library's n-th device allocation attempt from now on fail as
    out of memory (host-side injection; 0 disarms)."""
    _check(lib().mhdc_debug_fail_alloc(int(n)), "mhdc_debug_fail_alloc")


def mhdc_debug_alloc_stats() -> tuple[int, int]:
    """(allocation attempts since the last arming, live allocations)."""
    a, l_ = C.c_int64(0), C.c_int64(0)
    lib().mhdc_debug_alloc_stats(C.byref(a), C.byref(l_))
    return a.value, l_.value


def mhdc_fma_bench(fp64: bool, iters: int, out, stream=None):
    """FMA-throughput probe; out: float64 (fp64) or float32 tensor of
    mhdc_read_bench_ctas() * 256 elements.  FMAs = that count * 8 * iters."""
    import torch
    _check_dev(out, torch.float64 if fp64 else torch.float32, mhdc_read_bench_ctas() * 256, "out")
    _check(lib().mhdc_fma_bench(1 if fp64 else 0, int(iters), _ptr(out), _stream(stream)),
           "mhdc_fma_bench")
    return out


class Batch:
    """Owner of an mhdc_batch_handle; keeps its matrices alive."""

    def __init__(self, handle: int, mats):
        self.handle = handle
        self.mats = list(mats)

    def destroy(self):
        if self.handle:
            lib().mhdc_batch_destroy(C.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def mhdc_batch_create(mats) -> Batch:
    """Batch of Matrix handles of one dtype for one-launch products."""
    arr = (C.c_void_p * len(mats))(*[m.handle for m in mats])
    h = C.c_void_p()
    _check(lib().mhdc_batch_create(len(mats), arr, C.byref(h)), "mhdc_batch_create")
    return Batch(h.value, mats)


def pointer_array(tensors):
    """Device int64 tensor holding the data pointers of CUDA tensors."""
    import torch
    return torch.tensor([t.data_ptr() for t in tensors], dtype=torch.int64, device="cuda")


def _batch_args(B, xs, ys):
    import torch
    for a, nm in ((xs, "xs"), (ys, "ys")):
        if not a.is_cuda or a.dtype != torch.int64 or a.numel() < len(B.mats):
            raise ValueError(f"{nm} must be a CUDA int64 tensor of {len(B.mats)} device pointers")
    return C.c_void_p(B.handle), _ptr(xs), _ptr(ys)


def mhdc_batch_spmv(B: Batch, xs, ys, stream=None):
    """y_i = A_i x_i for every matrix of B in one launch; xs, ys from pointer_array()."""
    _check(lib().mhdc_batch_spmv(*_batch_args(B, xs, ys), _stream(stream)), "mhdc_batch_spmv")


def mhdc_batch_spmv_graph(B: Batch, xs, ys, stream=None):
    """mhdc_batch_spmv replayed from a CUDA graph captured on first use."""
    _check(lib().mhdc_batch_spmv_graph(*_batch_args(B, xs, ys), _stream(stream)),
           "mhdc_batch_spmv_graph")


def mhdc_batch_destroy(B: Batch):
    B.destroy()


class _Params(C.Structure):
    _fields_ = [("n_b", C.c_int32), ("dtype", C.c_int32), ("theta", C.c_double),
                ("variant", C.c_int32), ("reserved", C.c_int32)]


_DT_NAME = {MHDC_F64: "f64", MHDC_F32: "f32", MHDC_BF16: "bf16"}


def _params_dict(p: _Params) -> dict:
    return {"n_b": p.n_b, "theta": p.theta, "dtype": _DT_NAME[p.dtype], "variant": p.variant}


def mhdc_num_candidates() -> int:
    return int(lib().mhdc_num_candidates())


def mhdc_candidate(idx: int) -> dict:
    p = _Params()
    _check(lib().mhdc_candidate(int(idx), C.byref(p)), "mhdc_candidate")
    return _params_dict(p)


def mhdc_features(n, row_ptr, col, stream=None) -> np.ndarray:
    """The selector's feature vector (MHDC_NUM_FEATURES floats) of a CSR matrix."""
    import torch
    _check_dev(row_ptr, torch.int32, n + 1, "row_ptr")
    f = np.zeros(MHDC_NUM_FEATURES, dtype=np.float32)
    _check(lib().mhdc_features(n, _ptr(row_ptr), _ptr(col), _stream(stream),
                               f.ctypes.data_as(C.c_void_p)), "mhdc_features")
    return f


def mhdc_autotune(n, row_ptr, col, val, reps=10, stream=None) -> np.ndarray:
    """Mean time (us) of every candidate, -1 where it could not be built."""
    import torch
    _check_dev(row_ptr, torch.int32, n + 1, "row_ptr")
    t = np.zeros(MHDC_NUM_CANDIDATES, dtype=np.float32)
    _check(lib().mhdc_autotune(n, _ptr(row_ptr), _ptr(col), _ptr(val), int(reps), _stream(stream),
                               t.ctypes.data_as(C.c_void_p)), "mhdc_autotune")
    return t


def mhdc_select(n, row_ptr, col, val, tol, flags=MHDC_SELECT_PAPER, mlp=None, stream=None) -> dict:
    import torch
    _check_dev(row_ptr, torch.int32, n + 1, "row_ptr")
    p = _Params()
    _check(lib().mhdc_select(n, _ptr(row_ptr), _ptr(col), _ptr(val), float(tol), int(flags),
                             C.c_void_p(mlp.handle if mlp is not None else 0), _stream(stream),
                             C.byref(p)), "mhdc_select")
    return _params_dict(p)


class Mlp:
    """Owner of an mhdc_mlp_handle (the selector network)."""

    def __init__(self, handle: int, n_in: int, n_hidden: int, n_out: int):
        self.handle, self.n_in, self.n_hidden, self.n_out = handle, n_in, n_hidden, n_out

    @property
    def num_params(self) -> int:
        return mhdc_mlp_num_params(self)

    def destroy(self):
        if self.handle:
            lib().mhdc_mlp_destroy(C.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def mhdc_mlp_create(n_in, n_hidden, n_out, seed=0) -> Mlp:
    h = C.c_void_p()
    _check(lib().mhdc_mlp_create(int(n_in), int(n_hidden), int(n_out), int(seed), C.byref(h)),
           "mhdc_mlp_create")
    return Mlp(h.value, n_in, n_hidden, n_out)


def mhdc_mlp_num_params(M: Mlp) -> int:
    return int(lib().mhdc_mlp_num_params(C.c_void_p(M.handle)))


def mhdc_mlp_get_params(M: Mlp) -> np.ndarray:
    p = np.zeros(M.num_params, dtype=np.float32)
    _check(lib().mhdc_mlp_get_params(C.c_void_p(M.handle), p.ctypes.data_as(C.c_void_p)),
           "mhdc_mlp_get_params")
    return p


def mhdc_mlp_set_params(M: Mlp, p):
    p = np.ascontiguousarray(p, dtype=np.float32)
    if p.size != M.num_params:
        raise ValueError("wrong parameter count")
    _check(lib().mhdc_mlp_set_params(C.c_void_p(M.handle), p.ctypes.data_as(C.c_void_p)),
           "mhdc_mlp_set_params")


def _mlp_batch(M, X, T=None, Mask=None):
    import torch
    _check_dev(X, torch.float32, None, "X")
    B = X.shape[0]
    if X.dim() != 2 or X.shape[1] != M.n_in:
        raise ValueError("X must be batch x n_in")
    for t, nm in ((T, "T"), (Mask, "M")):
        if t is not None:
            _check_dev(t, torch.float32, B * M.n_out, nm)
    return B


def mhdc_mlp_forward(M: Mlp, X, stream=None):
    import torch
    B = _mlp_batch(M, X)
    Y = torch.empty((B, M.n_out), dtype=torch.float32, device=X.device)
    _check(lib().mhdc_mlp_forward(C.c_void_p(M.handle), B, _ptr(X), _ptr(Y), _stream(stream)),
           "mhdc_mlp_forward")
    return Y


def mhdc_mlp_grad(M: Mlp, X, T, Mask, stream=None):
    """(gradient of the masked MSE as a float32 numpy array, loss)."""
    B = _mlp_batch(M, X, T, Mask)
    g = np.zeros(M.num_params, dtype=np.float32)
    loss = C.c_float(0)
    _check(lib().mhdc_mlp_grad(C.c_void_p(M.handle), B, _ptr(X), _ptr(T), _ptr(Mask),
                               g.ctypes.data_as(C.c_void_p), C.byref(loss), _stream(stream)),
           "mhdc_mlp_grad")
    return g, float(loss.value)


def mhdc_mlp_train_step(M: Mlp, X, T, Mask, lr, stream=None, want_loss=True):
    B = _mlp_batch(M, X, T, Mask)
    loss = C.c_float(0)
    _check(lib().mhdc_mlp_train_step(C.c_void_p(M.handle), B, _ptr(X), _ptr(T), _ptr(Mask),
                                     float(lr), _stream(stream),
                                     C.byref(loss) if want_loss else None), "mhdc_mlp_train_step")
    return float(loss.value) if want_loss else None


def mhdc_mlp_destroy(M: Mlp):
    M.destroy()
