"""CPU oracle for the M-HDC SpMV library (ctypes binding of mhdc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product package, and sharing no
code with it.  All arithmetic is FP64 in plain C (see mhdc_oracle.c for the
paper passages each function follows); this module only marshals arrays.

Also here (plain numpy, FP64): the per-row error bounds used as tolerances.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhdc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

DTYPES = {"f64": 0, "f32": 1, "bf16": 2}
STORE_NP = {"f64": np.float64, "f32": np.float32, "bf16": np.uint16}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math: the FP order is the
    source order)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


P = C.c_void_p
I64 = C.c_int64
I32 = C.c_int32
D = C.c_double


def _declare(L):
    sig = {
        "orc_csr_check": (C.c_int, [I64, P, P]),
        "orc_csr_spmv": (None, [I64, P, P, P, P, P, C.c_int]),
        "orc_csr_absrow": (None, [I64, P, P, P, P, P, C.c_int]),
        "orc_round_f32": (None, [I64, P, P]),
        "orc_round_bf16": (None, [I64, P, P]),
        "orc_bf16_to_f64": (None, [I64, P, P]),
        "orc_select": (I64, [I64, P, P, I64, D, C.c_int, P, P, I64]),
        "orc_fill": (I64, [I64, P, P, P, I64, C.c_int, P, P, P, P, P, P]),
        "orc_hdc_global": (I64, [I64, P, P, P, D, P, I64, P, P, P, P, P]),
        "orc_mhdc_spmv": (None, [I64, I64, P, P, P, P, P, P, P, P, C.c_int]),
        "orc_mhdc_spmv_range": (None, [I64, I64, I64, I64, P, P, P, P, P, P, P, P, C.c_int]),
        "orc_mhdc_to_coo": (I64, [I64, I64, P, P, P, P, P, P, I64, P, P, P]),
        "orc_mhdc_absrow": (None, [I64, I64, P, P, P, P, P, P, P, P, P]),
        "orc_stream_direct": (None, [I64, P, P, P]),
        "orc_dia_to_csr": (I64, [I64, I64, P, P, P, P, P, I64]),
        "orc_stream_indirect": (None, [I64, P, P, P, P]),
        "orc_max_threads": (C.c_int, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(C.c_void_p)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(lib().orc_max_threads())


# --------------------------------------------------------------------------
# CSR (Sec. 3.2, Fig. 2)
# --------------------------------------------------------------------------

def csr_check(n, row_ptr, col) -> int:
    """0 if the CSR arrays are valid, else 1..4 (see mhdc_oracle.c)."""
    rp, c = _i32(row_ptr), _i32(col)
    if rp.size != n + 1:
        return 1
    if c.size < int(rp[-1]):
        return 2
    return int(lib().orc_csr_check(n, _p(rp), _p(c if c.size else np.zeros(1, np.int32))))


def csr_spmv(A, x, nthreads: int = 0) -> np.ndarray:
    x = _f64(x)
    y = np.empty(A.n, dtype=np.float64)
    lib().orc_csr_spmv(A.n, _p(_i32(A.row_ptr)), _p(_i32(A.col)), _p(_f64(A.val)), _p(x), _p(y),
                       nthreads)
    return y


def csr_absrow(A, x, nthreads: int = 0) -> np.ndarray:
    out = np.empty(A.n)
    lib().orc_csr_absrow(A.n, _p(_i32(A.row_ptr)), _p(_i32(A.col)), _p(_f64(A.val)),
                         _p(_f64(x)), _p(out), nthreads)
    return out


# --------------------------------------------------------------------------
# Storage rounding
# --------------------------------------------------------------------------

def round_f32(v) -> np.ndarray:
    v = _f64(v)
    out = np.empty(v.size, dtype=np.float32)
    lib().orc_round_f32(v.size, _p(v), _p(out))
    return out


def round_bf16(v) -> np.ndarray:
    """BF16 bit patterns (uint16) of v, rounded FP64 -> FP32 -> BF16."""
    v = _f64(v)
    out = np.empty(v.size, dtype=np.uint16)
    lib().orc_round_bf16(v.size, _p(v), _p(out))
    return out


def bf16_to_f64(b) -> np.ndarray:
    b = np.ascontiguousarray(b, dtype=np.uint16)
    out = np.empty(b.size)
    lib().orc_bf16_to_f64(b.size, _p(b), _p(out))
    return out


def store(v, dtype: str) -> np.ndarray:
    """v rounded to the storage dtype (as that dtype's numpy array)."""
    if dtype == "f64":
        return _f64(v).copy()
    if dtype == "f32":
        return round_f32(v)
    return round_bf16(v)


def widen(a, dtype: str) -> np.ndarray:
    """Stored values of dtype back to FP64 (exact)."""
    if dtype == "bf16":
        return bf16_to_f64(a)
    return np.asarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Conversion (Sec. 3.4, 4.3; Figs. 7, 12)
# --------------------------------------------------------------------------

def select(A, bl: int, theta: float, mode: str = "block"):
    n_blocks = (A.n + bl - 1) // bl
    dia_ptr = np.zeros(n_blocks + 1, dtype=np.int32)
    cap = max(1, A.nnz)
    if mode == "global" and n_blocks > 1:
        # every block gets the same list: size it from the single-block call
        _, one = select(A, max(1, A.n), theta, "global")
        cap = max(1, one.size * n_blocks)
    dia_offset = np.zeros(cap, dtype=np.int32)
    Pt = lib().orc_select(A.n, _p(_i32(A.row_ptr)), _p(_i32(A.col) if A.nnz else
                                                      np.zeros(1, np.int32)),
                          bl, float(theta), 1 if mode == "global" else 0,
                          _p(dia_ptr), _p(dia_offset), cap)
    if Pt < 0:
        raise RuntimeError("oracle select: capacity exceeded")
    return dia_ptr, dia_offset[:Pt].copy()


def convert(A, bl: int, theta: float, dtype: str = "f64", mode: str = "block") -> dict:
    """CSR -> M-HDC (mode "block") or blocked HDC (mode "global")."""
    if bl < 1:
        raise ValueError("bl must be >= 1")
    dia_ptr, dia_offset = select(A, bl, theta, mode)
    Pt = int(dia_ptr[-1])
    sd = STORE_NP[dtype]
    dia_val = np.zeros(max(1, Pt * bl), dtype=sd)
    csr_row_ptr = np.zeros(A.n + 1, dtype=np.int32)
    csr_col = np.zeros(max(1, A.nnz), dtype=np.int32)
    csr_val = np.zeros(max(1, A.nnz), dtype=sd)
    col = _i32(A.col) if A.nnz else np.zeros(1, np.int32)
    val = _f64(A.val) if A.nnz else np.zeros(1)
    nr = lib().orc_fill(A.n, _p(_i32(A.row_ptr)), _p(col), _p(val), bl, DTYPES[dtype],
                        _p(dia_ptr), _p(dia_offset if Pt else np.zeros(1, np.int32)),
                        _p(dia_val), _p(csr_row_ptr), _p(csr_col), _p(csr_val))
    return dict(n=A.n, bl=bl, theta=theta, dtype=dtype, mode=mode, dia_ptr=dia_ptr,
                dia_offset=dia_offset, dia_val=dia_val[:Pt * bl].copy(),
                csr_row_ptr=csr_row_ptr, csr_col=csr_col[:nr].copy(),
                csr_val=csr_val[:nr].copy(), nnz_rem=int(nr), P=Pt)


def hdc_global(A, theta: float) -> dict:
    """HDC as printed in the paper (Fig. 7): diagonals n long, indexed by row."""
    cap = max(1, min(2 * A.n - 1, A.nnz))
    dia_offset = np.zeros(cap, dtype=np.int32)
    dia_val = np.zeros(cap * A.n)
    csr_row_ptr = np.zeros(A.n + 1, dtype=np.int32)
    csr_col = np.zeros(max(1, A.nnz), dtype=np.int32)
    csr_val = np.zeros(max(1, A.nnz))
    nr = np.zeros(1, dtype=np.int64)
    nd = lib().orc_hdc_global(A.n, _p(_i32(A.row_ptr)), _p(_i32(A.col)), _p(_f64(A.val)),
                              float(theta), _p(dia_offset), cap, _p(dia_val), _p(csr_row_ptr),
                              _p(csr_col), _p(csr_val), _p(nr))
    r = int(nr[0])
    return dict(dia_offset=dia_offset[:nd].copy(), dia_val=dia_val[:nd * A.n].reshape(nd, A.n),
                csr_row_ptr=csr_row_ptr, csr_col=csr_col[:r].copy(), csr_val=csr_val[:r].copy())


def _wide_arrays(M):
    dt = M["dtype"]
    dv = widen(M["dia_val"], dt) if M["P"] else np.zeros(1)
    cv = widen(M["csr_val"], dt) if M["nnz_rem"] else np.zeros(1)
    cc = M["csr_col"] if M["nnz_rem"] else np.zeros(1, np.int32)
    do = M["dia_offset"] if M["P"] else np.zeros(1, np.int32)
    return _f64(dv), _f64(cv), _i32(cc), _i32(do)


def mhdc_spmv(M: dict, x, nthreads: int = 0) -> np.ndarray:
    """Fig. 13 in FP64 on the stored values (reduced dtypes widened exactly)."""
    dv, cv, cc, do = _wide_arrays(M)
    x = _f64(x)
    y = np.empty(M["n"])
    lib().orc_mhdc_spmv(M["n"], M["bl"], _p(_i32(M["dia_ptr"])), _p(do), _p(dv),
                        _p(_i32(M["csr_row_ptr"])), _p(cc), _p(cv), _p(x), _p(y), nthreads)
    return y


class Prepared:
    """An M-HDC structure with its arrays widened to FP64 once, for repeated
    timed products (the CPU baseline)."""

    def __init__(self, M: dict):
        self.M = M
        self.dv, self.cv, self.cc, self.do = _wide_arrays(M)
        self.dp = _i32(M["dia_ptr"])
        self.crp = _i32(M["csr_row_ptr"])

    def spmv_blocks(self, x, y, ib_begin: int, ib_end: int, nthreads: int = 0):
        lib().orc_mhdc_spmv_range(self.M["n"], self.M["bl"], ib_begin, ib_end, _p(self.dp),
                                  _p(self.do), _p(self.dv), _p(self.crp), _p(self.cc),
                                  _p(self.cv), _p(x), _p(y), nthreads)


def mhdc_to_coo(M: dict):
    dv, cv, cc, do = _wide_arrays(M)
    cap = M["P"] * M["bl"] + M["nnz_rem"] + 1
    ro = np.empty(cap, dtype=np.int64)
    co = np.empty(cap, dtype=np.int32)
    vo = np.empty(cap)
    m = lib().orc_mhdc_to_coo(M["n"], M["bl"], _p(_i32(M["dia_ptr"])), _p(do), _p(dv),
                              _p(_i32(M["csr_row_ptr"])), _p(cc), _p(cv), cap, _p(ro), _p(co),
                              _p(vo))
    if m < 0:
        raise RuntimeError("oracle round trip: capacity exceeded")
    return ro[:m], co[:m], vo[:m]


def mhdc_absrow(M: dict, x):
    dv, cv, cc, do = _wide_arrays(M)
    a = np.empty(M["n"])
    t = np.empty(M["n"], dtype=np.int64)
    lib().orc_mhdc_absrow(M["n"], M["bl"], _p(_i32(M["dia_ptr"])), _p(do), _p(dv),
                          _p(_i32(M["csr_row_ptr"])), _p(cc), _p(cv), _p(_f64(x)), _p(a), _p(t))
    return a, t


# --------------------------------------------------------------------------
# Tolerances
# --------------------------------------------------------------------------

FP64_ROW_TOL = 1e-12          # |y_i - y*_i| <= 1e-12 * sum_j |a_ij||x_j|
U_STORE = {"f64": 0.0, "f32": 2.0 ** -24, "bf16": (1 + 2.0 ** -24) * (1 + 2.0 ** -8) - 1}
U_ACC = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -24}

# FP32 / BF16 products sum a CSR remainder row (Fig. 13, first loop) with more
# than REM_LONG entries in FP64 and round that sum once into the FP32
# accumulator, where it counts as one term; FP64 handles are unaffected.
REM_LONG = 64


def gamma(k, u):
    k = np.asarray(k, dtype=np.float64)
    return k * u / (1.0 - k * u)


def long_remainder(M: dict) -> np.ndarray:
    """Per row of the converted matrix M: its remainder length L where a
    reduced-precision product sums the remainder in FP64 (L > REM_LONG),
    else 0; all zero for FP64 handles."""
    L = np.diff(np.asarray(M["csr_row_ptr"], dtype=np.int64))
    if M["dtype"] == "f64":
        return np.zeros_like(L)
    return np.where(L > REM_LONG, L, 0)


def _acc_factor(terms, dtype: str, long_rem):
    """(1 + gamma_{k+1}(u_acc)) (1 + gamma_L(2^-53)) - 1 for a row summed as
    k terms in the accumulator (Higham, Accuracy and Stability of Numerical
    Algorithms, Sec. 3.1: k FMAs into a sum starting at zero, plus one
    rounding kept as a margin).  A row with a long remainder (long_rem = L > 0)
    has k = terms - L + 1: its diagonal terms and the remainder's FP64 sum
    (error gamma_L(2^-53), products exact in FP64) rounded once."""
    terms = np.asarray(terms, dtype=np.float64)
    if long_rem is None:
        return gamma(terms + 1, U_ACC[dtype])
    lr = np.asarray(long_rem, dtype=np.float64)
    k = np.where(lr > 0, terms - lr + 1, terms)
    g = gamma(k + 1, U_ACC[dtype])
    return np.where(lr > 0, (1 + g) * (1 + gamma(lr, 2.0 ** -53)) - 1, g)


def bound_vs_exact(absrow, terms, dtype: str, long_rem=None) -> np.ndarray:
    """Per-row bound on |y_computed - y_exact| where y_exact uses the
    unrounded FP64 matrix and x: storage rounding of a and x (unit roundoff
    u_s each) and the accumulation bound f of _acc_factor:
    [(1 + u_s)^2 (1 + f) - 1] * sum_j |a_ij x_j|.  long_rem: per-row output
    of long_remainder (None: every row summed in the accumulator)."""
    if dtype == "f64":
        return FP64_ROW_TOL * np.asarray(absrow)
    us = U_STORE[dtype]
    f = _acc_factor(terms, dtype, long_rem)
    return ((1 + us) ** 2 * (1 + f) - 1) * np.asarray(absrow)


def bound_vs_stored(absrow_stored, terms, dtype: str, long_rem=None) -> np.ndarray:
    """Per-row bound on |y_computed - y_stored| where y_stored is the FP64
    product of the stored (rounded) values: f * sum |a^ x^| (f of _acc_factor)."""
    if dtype == "f64":
        return FP64_ROW_TOL * np.asarray(absrow_stored)
    return _acc_factor(terms, dtype, long_rem) * np.asarray(absrow_stored)


# --------------------------------------------------------------------------
# Memory benchmarks (Sec. 6.2)
# --------------------------------------------------------------------------

def dia_to_csr(n, offsets, dia_val):
    """DIA arrays (Sec. 3.3, Fig. 4: dia_val[d, i] = a(i, i + offsets[d])) as
    CSR (row_ptr, col, val); zeros and out-of-range positions are not entries."""
    off = _i32(offsets)
    dv = _f64(dia_val).reshape(-1)
    nd = off.size
    assert dv.size == nd * n
    rp = np.zeros(n + 1, dtype=np.int32)
    nnz = lib().orc_dia_to_csr(n, nd, _p(off), _p(dv), _p(rp), None, None, 0)
    if nnz < 0:
        raise ValueError("offsets must be strictly increasing")
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    val = np.zeros(max(nnz, 1), dtype=np.float64)
    got = lib().orc_dia_to_csr(n, nd, _p(off), _p(dv), _p(rp), _p(col), _p(val), nnz)
    assert got == nnz
    return rp, col[:nnz], val[:nnz]


def stream_direct(A, B, Cv):
    Cv = _f64(Cv).copy()
    lib().orc_stream_direct(Cv.size, _p(_f64(A)), _p(_f64(B)), _p(Cv))
    return Cv


def stream_indirect(A, B, I, Cv):
    Cv = _f64(Cv).copy()
    lib().orc_stream_indirect(Cv.size, _p(_f64(A)), _p(_f64(B)), _p(_i32(I)), _p(Cv))
    return Cv
