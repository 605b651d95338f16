"""The memory-traffic performance models of Sec. 5 (host arithmetic only).

Every volume is in units of b_fp * n bytes (b_fp: bytes of one stored value,
n: rows), and a kernel's predicted speed relative to another is the inverse
ratio of their volumes (Sec. 5.1: P_A / P_B = V_B / V_A).  b = b_int / b_fp is
the index-to-value size ratio (1/2 for FP64 values with INT32 indices).

Stencil matrices (Sec. 5.2): nd full diagonals, nnz = nd n; gamma is the
share of x accesses that reach main memory (1/nd <= gamma <= 1).
General matrices (Sec. 5.3): c = nnz / n, beta the CSR rate (share of the
nonzeros left in the CSR part), alpha the filling rate of the DIA part,
v_x the x traffic of the CSR kernel per row (>= 1).  The M-HDC model is the
B-HDC one with the block-wise alpha and beta (Sec. 5.3.3-5.3.4).
"""
from __future__ import annotations

B_FP64_INT32 = 0.5


def b_ratio(dtype: str) -> float:
    """b_int / b_fp for INT32 indices and values of `dtype`."""
    return {"f64": 4 / 8, "f32": 4 / 4, "bf16": 4 / 2}[dtype]


# ------------------------------------------------------------ stencil (Sec. 5.2)

def volume_csr_stencil(nd: float, gamma: float, b: float = B_FP64_INT32) -> float:
    """CSR kernel: val and col_ind (nd n each), row_ptr (n), x (gamma nd n), y (n)."""
    return nd + b * nd + b + gamma * nd + 1


def volume_dia_stencil(nd: float, b: float = B_FP64_INT32) -> float:
    """Unblocked DIA kernel (Fig. 5): val (nd n), every x access from main memory
    (nd n), y zeroed once and read and written per diagonal ((1 + 2 nd) n)."""
    return nd + nd + 1 + 2 * nd


def volume_bdia_stencil(nd: float, gamma: float, b: float = B_FP64_INT32) -> float:
    """B-DIA kernel (Fig. 9): val (nd n), x (gamma nd n), y written once (n)."""
    return nd + gamma * nd + 1


def stencil_speedups(nd: float, gamma: float, b: float = B_FP64_INT32) -> dict:
    """Predicted relative performance of the three stencil kernels (Sec. 5.2.4-5.2.6)."""
    vc = volume_csr_stencil(nd, gamma, b)
    vd = volume_dia_stencil(nd, b)
    vb = volume_bdia_stencil(nd, gamma, b)
    return {"dia_over_csr": vc / vd, "bdia_over_csr": vc / vb, "bdia_over_dia": vd / vb}


# ------------------------------------------------------------ general (Sec. 5.3)

def volume_csr(c: float, b: float = B_FP64_INT32, v_x: float = 1.0) -> float:
    """CSR kernel on a general matrix: val, col_ind (c n each), row_ptr, x (v_x n), y."""
    return c + b * c + b + v_x + 1


def volume_hdc(alpha: float, beta: float, c: float, b: float = B_FP64_INT32, v_x: float = 1.0,
               dv_x: float = 0.0) -> float:
    """B-HDC / M-HDC kernel: the CSR part (beta c values and indices, row_ptr),
    the DIA part ((1 - beta) c / alpha stored values), x (v_x + dv_x), y."""
    return beta * (c + b * c) + b + (1 - beta) * c / alpha + v_x + dv_x + 1


def rp_est(alpha: float, beta: float, c: float, b: float = B_FP64_INT32, v_x: float = 1.0) -> float:
    """Estimated relative performance of the (B/M-)HDC kernel over CSR (Sec. 5.3.2
    and 5.3.4, with dv_x = 0: an upper estimate)."""
    return volume_csr(c, b, v_x) / volume_hdc(alpha, beta, c, b, v_x)


def relative_error(est: float, exe: float) -> float:
    """RE = (RP_est - RP_exe) / RP_exe (Sec. 6.4.3)."""
    return (est - exe) / exe
