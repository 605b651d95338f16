"""GPU parity of the unblocked DIA-order product (Fig. 5, mhdc_dia_spmv):
bit-identical to the blocked product on the same global-selection handle and,
through it, within the stated bounds of the oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_build, check_spmv, dev_csr, torch, x_device, y_empty

pytestmark = pytest.mark.gpu

DTYPES = ("f64", "f32", "bf16")


@pytest.fixture(scope="module")
def mh():
    t = torch()
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2105_04937_gb300 as m
    m.lib()
    return m


def dia_matches_blocked(mh, h, M, A, x64, dt):
    """mhdc_spmv within the oracle's bounds, and mhdc_dia_spmv bit-identical to it."""
    yb = check_spmv(mh, h, M, A, x64, dt)
    xd, _ = x_device(x64, dt)
    y = y_empty(A.n, dt)
    mh.mhdc_dia_spmv(h, xd, y)
    torch().cuda.synchronize()
    yd = y.double().cpu().numpy()
    assert np.array_equal(yd.view(np.uint64), yb.view(np.uint64)), (A.n, h.info["n_b"], dt)


@pytest.mark.parametrize("seed", range(6))
def test_random_small_every_block_size(mh, seed):
    rng = synth.Rng(seed, 9)
    n = int(rng.integers(1, 1, 300)[0])
    A = synth.random_sparse(n, 0.03, seed=100 + seed, diag_bias=0.7)
    x = synth.uniform_vector(n, seed)
    for n_b in sorted({1, 3, 8, 64, 100, n, 2 * n + 1}):
        for theta in (0.0, 0.02, 0.5):
            for dt in DTYPES:
                h, M = check_build(mh, A, n_b, theta, dt, mode="global")
                dia_matches_blocked(mh, h, M, A, x, dt)


def test_paper_stencils_b_dia(mh):
    # theta = 0 keeps every nonempty diagonal in every block: B-DIA (Figs. 8-9)
    for dim in (1, 2, 3):
        A = synth.paper_stencil(50000, dim)
        x = synth.uniform_vector(A.n, dim)
        for n_b in (10, 500, 4096, 5000):
            for dt in DTYPES:
                h, M = check_build(mh, A, n_b, 0.0, dt, mode="global")
                assert h.info["nnz_rem"] == 0
                dia_matches_blocked(mh, h, M, A, x, dt)


def test_dia_with_remainder_and_ragged_tail(mh):
    A = synth.stencil_3d(30, 29, 23, 27, seed=4, drop_rate=0.3, drop_block=1024,
                         offband_poisson=0.7)
    x = synth.loguniform_vector(A.n, 8)
    for n_b in (1000, 1024, 4099):
        for dt in DTYPES:
            h, M = check_build(mh, A, n_b, 0.6, dt, mode="global")
            assert h.info["nnz_rem"] > 0
            dia_matches_blocked(mh, h, M, A, x, dt)


def test_dia_paper_stencil_large(mh):
    # 3D 7-point stencil with n = 2e7 (x, y 160 MB each: beyond L2)
    t = torch()
    A = synth.paper_stencil(20_000_000, 3)
    rp, col, val = dev_csr(A)
    h = mh.hdc_build(A.n, rp, col, val, 4096, 0.0, "f64")
    assert h.info["nnz_rem"] == 0 and h.info["P"] == 7 * h.info["n_blocks"]
    x = synth.uniform_vector(A.n, 77)
    xd = t.from_numpy(x).cuda()
    y1, y2, y3 = (y_empty(A.n, "f64") for _ in range(3))
    mh.mhdc_spmv(h, xd, y1)
    mh.mhdc_dia_spmv(h, xd, y2)
    mh.csr_spmv(A.n, rp, col, val, xd, y3)
    t.cuda.synchronize()
    assert t.equal(y1, y2)
    ref = oracle.csr_spmv(A, x)
    tol = oracle.FP64_ROW_TOL * oracle.csr_absrow(A, x)
    assert np.all(np.abs(y2.cpu().numpy() - ref) <= tol)
    assert np.all(np.abs(y3.cpu().numpy() - ref) <= tol)


def test_dia_rejects_block_mode_and_handles_empty(mh):
    t = torch()
    A = synth.example_matrix()
    rp, col, val = dev_csr(A)
    h = mh.mhdc_build(A.n, rp, col, val, 4, 0.6)
    x = t.zeros(A.n, dtype=t.float64, device="cuda")
    y = t.zeros(A.n, dtype=t.float64, device="cuda")
    with pytest.raises(mh.MhdcError) as e:
        mh.mhdc_dia_spmv(h, x, y)
    assert e.value.code == mh.MHDC_ERR_UNSUPPORTED
    z = t.zeros(1, dtype=t.int32, device="cuda")
    h0 = mh.hdc_build(0, z, z, t.zeros(1, dtype=t.float64, device="cuda"), 16, 0.6)
    mh.mhdc_dia_spmv(h0, x[:0], y[:0])
    # a matrix without entries: y = 0
    E = synth.CSR(300, np.zeros(301, np.int32), np.zeros(0, np.int32), np.zeros(0))
    h, M = check_build(mh, E, 64, 0.5, "f64", mode="global")
    dia_matches_blocked(mh, h, M, E, synth.uniform_vector(300, 1), "f64")
