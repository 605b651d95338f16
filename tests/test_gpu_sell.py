"""GPU tests of the SELL-C-sigma baseline: the layout against a host
re-derivation of its definition (sorting inside sigma windows, chunks of C
rows padded to their longest row, column-by-column storage), and the
product bit-identical to the CSR kernel and within the oracle's bound."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev_csr, torch, y_empty

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    t = torch()
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2105_04937_gb300 as m
    m.lib()
    return m


def expected_layout(A, C, sigma):
    lens = np.diff(A.row_ptr).astype(np.int64)
    perm = []
    for w0 in range(0, A.n, sigma):
        idx = np.arange(w0, min(w0 + sigma, A.n))
        if sigma > 1:
            idx = idx[np.lexsort((idx, -lens[idx]))]  # longest first, ties by row
        perm += idx.tolist()
    perm = np.array(perm, dtype=np.int64)
    rowlen = lens[perm]
    chunks = -(-A.n // C)
    widths = np.array([rowlen[c * C:(c + 1) * C].max(initial=0) for c in range(chunks)])
    chunk_ptr = np.concatenate([[0], np.cumsum(widths * C)])
    col = np.zeros(chunk_ptr[-1], np.int64)
    val = np.zeros(chunk_ptr[-1])
    for pos, i in enumerate(perm):
        c, r = divmod(pos, C)
        a, b = A.row_ptr[i], A.row_ptr[i + 1]
        q = chunk_ptr[c] + r + C * np.arange(b - a)
        col[q] = A.col[a:b]
        val[q] = A.val[a:b]
    return perm, rowlen, chunk_ptr, col, val


def check_sell(mh, A, C, sigma, x):
    t = torch()
    rp, col, val = dev_csr(A)
    S = mh.sell_build(A.n, rp, col, val, C, sigma)
    E = mh.sell_export(S)
    perm, rowlen, chunk_ptr, ecol, evalue = expected_layout(A, C, sigma)
    assert np.array_equal(E["perm"], perm), (C, sigma)
    assert np.array_equal(E["rowlen"], rowlen)
    assert np.array_equal(E["chunk_ptr"], chunk_ptr)
    assert np.array_equal(E["col"], ecol) and np.array_equal(E["val"].view(np.uint64),
                                                             evalue.view(np.uint64))
    assert S.info["nnz"] == A.nnz and S.info["slots"] == chunk_ptr[-1]
    xd = t.from_numpy(x).cuda()
    y1, y2 = y_empty(A.n, "f64"), y_empty(A.n, "f64")
    mh.sell_spmv(S, xd, y1)
    mh.csr_spmv(A.n, rp, col, val, xd, y2)
    t.cuda.synchronize()
    assert t.equal(y1, y2), (C, sigma)
    ref = oracle.csr_spmv(A, x)
    assert np.all(np.abs(y1.cpu().numpy() - ref) <= oracle.FP64_ROW_TOL * oracle.csr_absrow(A, x))
    S.destroy()


@pytest.mark.parametrize("seed", range(3))
def test_sell_random_small(mh, seed):
    A = synth.random_sparse(150 + 37 * seed, 0.05, seed=seed, diag_bias=0.6)
    x = synth.uniform_vector(A.n, seed)
    for C in (1, 8, 32, 33):
        for sigma in (1, 32, 64, 100, 4096):
            check_sell(mh, A, C, sigma, x)


def test_sell_structured_and_empty_rows(mh):
    d = np.zeros((300, 300))
    d[5, 7] = 1.5
    d[299, 0] = -2.0
    d[100, 50:90] = 0.25
    cases = [synth.config_matrix("stencil7_32"), synth.config_matrix("scattered_4m", 1 / 64),
             synth.from_dense(d),
             synth.stencil_3d(20, 19, 17, 27, seed=3, drop_rate=0.4, drop_block=256,
                              offband_poisson=2.0)]
    for A in cases:
        x = synth.loguniform_vector(A.n, 4)
        for C, sigma in ((32, 1), (32, 256), (32, 8192), (16, 512)):
            check_sell(mh, A, C, sigma, x)


def test_sell_full_size_bit_identical_to_csr(mh):
    t = torch()
    A = synth.config_matrix("stencil27_128")
    rp, col, val = dev_csr(A)
    S = mh.sell_build(A.n, rp, col, val, 32, 256)
    x = t.from_numpy(synth.uniform_vector(A.n, 2)).cuda()
    y1, y2 = y_empty(A.n, "f64"), y_empty(A.n, "f64")
    mh.sell_spmv(S, x, y1)
    mh.csr_spmv(A.n, rp, col, val, x, y2)
    t.cuda.synchronize()
    assert t.equal(y1, y2)
    inf = S.info
    assert inf["nnz"] == A.nnz and inf["slots"] >= A.nnz and inf["chunks"] == A.n // 32


def test_sell_bad_arguments(mh):
    t = torch()
    A = synth.example_matrix()
    rp, col, val = dev_csr(A)
    for C, sigma in ((0, 1), (2000, 1), (32, 0), (32, 9000)):
        with pytest.raises(mh.MhdcError) as e:
            mh.sell_build(A.n, rp, col, val, C, sigma)
        assert e.value.code == mh.MHDC_ERR_INVALID_ARG


def test_sell_fewer_rows_than_a_chunk(mh):
    # n < C: one partial chunk; n = 1
    for n in (1, 5, 31):
        d = np.zeros((n, n))
        d[np.arange(n), np.arange(n)] = 2.0
        d[0, n - 1] = -1.0 if n > 1 else 2.0
        A = synth.from_dense(d)
        check_sell(mh, A, 32, 64, synth.uniform_vector(n, n))
