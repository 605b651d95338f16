"""The bounds-checked product (mhdc_set_checked), on in-bounds inputs only.

With checking on, every index the product computes is compared with its
array's extent before the access.  On valid handles no check may fire
(mhdc_check stays OK) and y must equal the unchecked default product bit for
bit, over tile edges, ragged last blocks, vector and element layouts,
remainder-heavy and long remainder rows, misaligned x and the host-buffer
entry point.  No test here hands the kernel an out-of-range structure.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_build, check_spmv, torch, x_device, y_empty

pytestmark = pytest.mark.gpu

DTYPES = ("f64", "f32", "bf16")


@pytest.fixture(scope="module")
def mh():
    t = torch()
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2105_04937_gb300 as m
    m.lib()
    return m


def long_row_matrix():
    # rows of 70 and 130 remainder entries (FP64 accumulation for reduced
    # precision) among ordinary stencil rows
    A = synth.config_matrix("stencil7_32", scale=0.25)
    rows = [[] for _ in range(A.n)]
    for i in range(A.n):
        a, b = A.row_ptr[i], A.row_ptr[i + 1]
        rows[i] = list(zip(A.col[a:b].tolist(), A.val[a:b].tolist()))
    rng = synth.Rng(41, 2)
    for i, L in ((5, 70), (A.n // 2, 130), (A.n - 1, 66)):
        cols = sorted(set(int(c) for c in rng.integers(L * 2, 0, A.n)) | {c for c, _ in rows[i]})
        have = dict(rows[i])
        rows[i] = [(c, have.get(c, float(v))) for c, v in zip(cols, rng.uniform(len(cols), -1, 1))]
    rp = np.zeros(A.n + 1, dtype=np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c, _ in r], dtype=np.int32)
    val = np.array([v for r in rows for _, v in r], dtype=np.float64)
    return synth.CSR(A.n, rp, col, val)


CASES = [("stencil27_48", lambda: synth.config_matrix("stencil27_128", scale=0.375), 4096),
         ("stencil27_48_ragged", lambda: synth.config_matrix("stencil27_128", scale=0.375), 1000),
         ("odd_block", lambda: synth.config_matrix("stencil7_32", scale=0.5), 999),
         ("scattered", lambda: synth.config_matrix("scattered_4m", scale=1 / 256), 2048),
         ("random", lambda: synth.random_sparse(333, 0.05, seed=12, diag_bias=0.5), 37),
         ("long_rows", long_row_matrix, 512)]


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("name,make,n_b", CASES, ids=[c[0] for c in CASES])
def test_checked_product_equals_unchecked(mh, dt, name, make, n_b):
    t = torch()
    A = make()
    h, M = check_build(mh, A, n_b, 0.6, dt)
    x64 = synth.uniform_vector(A.n, 17)
    xd, _ = x_device(x64, dt)
    mh.mhdc_set_variant(h, -1)
    y0 = y_empty(A.n, dt)
    mh.mhdc_spmv(h, xd, y0)
    mh.mhdc_set_checked(h, True)
    y1 = y_empty(A.n, dt)
    mh.mhdc_spmv(h, xd, y1)
    # x one element off the allocation's alignment
    buf = t.zeros(A.n + 1, dtype=xd.dtype, device="cuda")
    buf[1:] = xd
    y2 = y_empty(A.n, dt)
    mh.mhdc_spmv(h, buf[1:], y2)
    t.cuda.synchronize()
    mh.mhdc_check(h)                 # no check fired
    assert t.equal(y1, y0), name
    assert t.equal(y2, y0), name
    check_spmv(mh, h, M, A, x64, dt)  # the checked product against the oracle
    mh.mhdc_check(h)
    mh.mhdc_set_checked(h, False)
    h.destroy()


def test_checked_host_entry_point(mh):
    t = torch()
    A = synth.config_matrix("stencil27_128", scale=0.25)
    h, M = check_build(mh, A, 4096, 0.6, "f64")
    x = t.from_numpy(synth.uniform_vector(A.n, 3)).pin_memory()
    y = t.empty(A.n, dtype=t.float64).pin_memory()
    mh.mhdc_set_checked(h, True)
    mh.mhdc_spmv_host(h, x, y)
    mh.mhdc_check(h)
    ref = oracle.mhdc_spmv(M, x.numpy())
    tol = oracle.FP64_ROW_TOL * oracle.csr_absrow(A, x.numpy())
    assert np.all(np.abs(y.numpy() - ref) <= tol)
    assert mh.lib().mhdc_set_checked(ctypes.c_void_p(h.handle), 2) == mh.MHDC_ERR_INVALID_ARG
    h.destroy()
