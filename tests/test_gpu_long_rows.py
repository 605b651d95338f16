"""GPU tests of the long-remainder-row rule of the reduced-precision products:
a CSR remainder row (Fig. 13, first loop) with more than 64 entries is summed
in FP64 and rounded once into the FP32 accumulator.

Rows built as 2^25 followed by ones (x = 1) make the rule visible exactly:
FP32 accumulation loses every +1 (ulp(2^25) = 4), FP64 keeps them, and with
diagonal values 4, 8, 4 every later FP32 step is exact.  So a row with 64
remainder entries (not long) must come out as 2^25 + 16 and a row with 65 as
2^25 + 64 + 16, in every kernel: every tile shape of mhdc_spmv, the DIA-order
product, SpMM and the batched launch.  Random x then checks every row against
the oracle's bound for this arithmetic."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_build, check_spmm, check_spmv, torch, x_device, y_empty

pytestmark = pytest.mark.gpu

BIG = 2.0 ** 25


@pytest.fixture(scope="module")
def mh():
    t = torch()
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2105_04937_gb300 as m
    m.lib()
    return m


def long_row_matrix():
    """n = 3000, tridiagonal 4 / 8 / 4 plus remainder rows of 2^25 and ones
    (first entry in column order 2^25) and two random long rows.  Returns
    the CSR and {row: (exact sum with x = 1 in FP64, FP32 kernel result)}."""
    n = 3000
    d = np.zeros((n, n))
    i = np.arange(n)
    d[i, i] = 8.0
    d[i[1:], i[1:] - 1] = 4.0
    d[i[:-1], i[:-1] + 1] = 4.0
    expect = {}

    def ones_row(r, c0, ones):
        d[r, c0] = BIG
        d[r, c0 + 1:c0 + 1 + ones] = 1.0
        diag = d[r, max(r - 1, 0):r + 2].sum()
        L = ones + 1
        fp32 = BIG + (ones if L > 64 else 0) + diag
        expect[r] = (BIG + ones + diag, fp32)

    ones_row(1000, 0, 63)      # 64 entries: FP32 accumulation
    ones_row(1500, 0, 64)      # 65 entries: FP64
    ones_row(5, 2000, 64)      # first block
    ones_row(2999, 0, 64)      # last row, ragged last block, two diagonal terms
    ones_row(0, 1000, 300)     # first row, 301 entries
    rng = synth.Rng(7, 31)
    for r in (2000, 2101):
        pool = np.setdiff1d(np.arange(n), [r - 1, r, r + 1])
        cols = np.sort(pool[np.argsort(rng.unit(pool.size))[:500]])
        d[r, cols] = rng.uniform(500, -1, 1) * 10.0 ** rng.uniform(500, -2, 2)
    return synth.from_dense(d), expect


def assert_rows(y, expect, dt, ctx):
    yv = y.double().cpu().numpy()
    for r, (e64, e32) in expect.items():
        want = e64 if dt == "f64" else e32
        assert yv[r] == want, (ctx, dt, r, yv[r], want)


@pytest.mark.parametrize("dt", ("f64", "f32", "bf16"))
def test_long_rows_every_variant(mh, dt):
    t = torch()
    A, expect = long_row_matrix()
    h, M = check_build(mh, A, 256, 0.6, dt)
    lr = oracle.long_remainder(M)
    if dt != "f64":
        assert lr[1000] == 0 and lr[1500] == 65 and lr[0] == 301 and lr[2000] == 500
    ones, _ = x_device(np.ones(A.n), dt)
    vs = (-1,) + tuple(mh.NATIVE_VARIANTS)
    for v in vs:
        mh.mhdc_set_variant(h, v)
        y = y_empty(A.n, dt)
        mh.mhdc_spmv(h, ones, y)
        t.cuda.synchronize()
        assert_rows(y, expect, dt, ("variant", v))
        check_spmv(mh, h, M, A, synth.loguniform_vector(A.n, 3), dt)


@pytest.mark.parametrize("dt", ("f64", "f32", "bf16"))
def test_long_rows_dia_order_spmm_and_batch(mh, dt):
    t = torch()
    A, expect = long_row_matrix()
    ones, _ = x_device(np.ones(A.n), dt)
    # DIA order on a global-selection handle, bit-identical to the blocked kernel
    hg, Mg = check_build(mh, A, 256, 0.6, dt, mode="global")
    y1, y2 = y_empty(A.n, dt), y_empty(A.n, dt)
    mh.mhdc_dia_spmv(hg, ones, y1)
    mh.mhdc_spmv(hg, ones, y2)
    t.cuda.synchronize()
    assert_rows(y1, expect, dt, "dia order")
    assert t.equal(y1, y2)
    # SpMM: every column a copy of the ones vector, then random columns
    h, M = check_build(mh, A, 256, 0.6, dt)
    for k in (1, 3, 8, 16):
        X = np.ones((A.n, k))
        Xs = oracle.store(X.ravel(), dt)
        if dt == "bf16":
            Xd = t.from_numpy(Xs.view(np.int16)).cuda().view(t.bfloat16).reshape(A.n, k)
        else:
            Xd = t.from_numpy(Xs).cuda().reshape(A.n, k)
        Y = t.full((A.n, k), float("nan"), dtype=t.float64 if dt == "f64" else t.float32,
                   device="cuda")
        mh.mhdc_spmm(h, Xd, Y)
        t.cuda.synchronize()
        for c in range(k):
            assert_rows(Y[:, c], expect, dt, ("spmm", k, c))
    rng = synth.Rng(5, 17)
    check_spmm(mh, h, M, A, rng.uniform(A.n * 5, -1, 1).reshape(A.n, 5), dt)
    # one persistent launch over the matrix twice (blocked and global handles)
    B = mh.mhdc_batch_create([h, hg])
    ys = [y_empty(A.n, dt), y_empty(A.n, dt)]
    mh.mhdc_batch_spmv(B, mh.pointer_array([ones, ones]), mh.pointer_array(ys))
    t.cuda.synchronize()
    for y in ys:
        assert_rows(y, expect, dt, "batch")
    B.destroy()
