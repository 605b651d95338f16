"""Helpers for the GPU parity tests: move synthetic matrices to the device,
call the library through its C ABI (Python binding), and compare with the
oracle."""
import numpy as np

import oracle

VALUE_KEYS = ("dia_val", "csr_val")
INDEX_KEYS = ("dia_ptr", "dia_offset", "csr_row_ptr", "csr_col")


def torch():
    import torch as t
    return t


def dev_csr(A):
    t = torch()
    return (t.from_numpy(np.ascontiguousarray(A.row_ptr, np.int32)).cuda(),
            t.from_numpy(np.ascontiguousarray(A.col, np.int32)).cuda(),
            t.from_numpy(np.ascontiguousarray(A.val, np.float64)).cuda())


def x_device(x64, dtype):
    """x rounded to the storage dtype by the oracle, as a device tensor."""
    t = torch()
    s = oracle.store(x64, dtype)
    if dtype == "bf16":
        return t.from_numpy(s.view(np.int16)).cuda().view(t.bfloat16), oracle.widen(s, dtype)
    return t.from_numpy(s).cuda(), oracle.widen(s, dtype)


def y_empty(n, dtype):
    t = torch()
    return t.full((max(n, 1),), float("nan"), dtype=t.float64 if dtype == "f64" else t.float32,
                  device="cuda")[:n]


def bits(a):
    a = np.asarray(a)
    return a.view({8: np.uint64, 4: np.uint32, 2: np.uint16}[a.dtype.itemsize])


def build(mh, A, n_b, theta, dtype="f64", mode="block"):
    rp, col, val = dev_csr(A)
    fn = mh.mhdc_build if mode == "block" else mh.hdc_build
    return fn(A.n, rp, col, val, n_b, theta, dtype)


def assert_same_structure(E, M, ctx=""):
    for k in INDEX_KEYS:
        assert np.array_equal(E[k], M[k]), (ctx, k, E[k][:20], M[k][:20])
    for k in VALUE_KEYS:
        assert E[k].shape == M[k].shape, (ctx, k)
        assert np.array_equal(bits(E[k]), bits(M[k])), (ctx, k)


def check_build(mh, A, n_b, theta, dtype="f64", mode="block"):
    """Build on the GPU, export, and require bit-exact equality with the oracle."""
    M = oracle.convert(A, n_b, theta, dtype, mode)
    h = build(mh, A, n_b, theta, dtype, mode)
    E = mh.mhdc_export(h)
    assert_same_structure(E, M, (A.n, n_b, theta, dtype, mode))
    inf = h.info
    assert inf["P"] == M["P"] and inf["nnz_rem"] == M["nnz_rem"] and inf["nnz"] == A.nnz
    return h, M


def check_spmv(mh, h, M, A, x64, dtype):
    """mhdc_spmv against the oracle: within the stated per-row bounds both
    against the FP64 product of the stored values and against the exact
    (unrounded) FP64 product."""
    xd, xs = x_device(x64, dtype)
    y = y_empty(A.n, dtype)
    mh.mhdc_spmv(h, xd, y)
    torch().cuda.synchronize()
    mh.mhdc_check(h)
    yg = y.double().cpu().numpy()
    assert np.all(np.isfinite(yg))
    y_st = oracle.mhdc_spmv(M, xs)
    abs_st, terms = oracle.mhdc_absrow(M, xs)
    lr = oracle.long_remainder(M)
    err = np.abs(yg - y_st)
    bnd = oracle.bound_vs_stored(abs_st, terms, dtype, lr)
    bad = np.nonzero(err > bnd)[0]
    assert bad.size == 0, ("vs stored", dtype, bad[:5], err[bad[:5]], bnd[bad[:5]])
    y_ex = oracle.csr_spmv(A, x64)
    abs_ex = oracle.csr_absrow(A, x64)
    bnd = oracle.bound_vs_exact(abs_ex, terms, dtype, lr)
    err = np.abs(yg - y_ex)
    bad = np.nonzero(err > bnd)[0]
    assert bad.size == 0, ("vs exact", dtype, bad[:5], err[bad[:5]], bnd[bad[:5]])
    return yg


def check_spmm(mh, h, M, A, X64, dtype, pad=0):
    """mhdc_spmm against the oracle column by column (same bounds as SpMV).
    X64: n x k float64; pad > 0 stores X and Y with leading dimension k + pad."""
    t = torch()
    n, k = X64.shape
    Xs = oracle.store(X64.ravel(), dtype).reshape(n, k)
    Xw = oracle.widen(Xs.ravel(), dtype).reshape(n, k)
    ld = k + pad
    if dtype == "bf16":
        base = t.zeros((n, ld), dtype=t.int16)
        base[:, :k] = t.from_numpy(Xs.view(np.int16))
        Xd = base.cuda().view(t.bfloat16)
    else:
        base = t.zeros((n, ld), dtype=t.float64 if dtype == "f64" else t.float32)
        base[:, :k] = t.from_numpy(Xs)
        Xd = base.cuda()
    yt = t.float64 if dtype == "f64" else t.float32
    Yfull = t.full((n, ld), float("nan"), dtype=yt, device="cuda")
    Yd = Yfull[:, :k]
    Xv = Xd[:, :k]
    mh.mhdc_spmm(h, Xv, Yd)
    t.cuda.synchronize()
    Y = Yfull.double().cpu().numpy()
    if pad:
        assert np.all(np.isnan(Y[:, k:])), "mhdc_spmm wrote outside the k columns"
    lr = oracle.long_remainder(M)
    for c in range(k):
        yg = Y[:, c]
        y_st = oracle.mhdc_spmv(M, Xw[:, c])
        abs_st, terms = oracle.mhdc_absrow(M, Xw[:, c])
        assert np.all(np.abs(yg - y_st) <= oracle.bound_vs_stored(abs_st, terms, dtype, lr)), \
            (dtype, k, c)
        x64 = np.ascontiguousarray(X64[:, c])
        bnd = oracle.bound_vs_exact(oracle.csr_absrow(A, x64), terms, dtype, lr)
        assert np.all(np.abs(yg - oracle.csr_spmv(A, x64)) <= bnd), (dtype, k, c)
