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


# ---------------------------------------------------------------- DIA input (mhdc_build_dia)

def _dia_case(mh, n, offs, val, n_b, theta, dt, x=None):
    """mhdc_build_dia against the oracle's conversion of the same entries
    (oracle.dia_to_csr, then oracle.convert): every array bit-exact, then
    the product within the stated bounds."""
    from gpu_util import assert_same_structure
    t = torch()
    rp, col, v = oracle.dia_to_csr(n, offs, val)
    A = synth.CSR(n, rp, col, v, {})
    M = oracle.convert(A, n_b, theta, dt)
    h = mh.mhdc_build_dia(n, t.from_numpy(np.ascontiguousarray(offs, np.int32)).cuda(),
                          t.from_numpy(np.ascontiguousarray(val, np.float64)).cuda(), n_b, theta, dt)
    assert_same_structure(mh.mhdc_export(h), M, (n, n_b, theta, dt))
    inf = h.info
    assert inf["nnz"] == A.nnz and inf["P"] == M["P"] and inf["nnz_rem"] == M["nnz_rem"]
    if x is not None:
        check_spmv(mh, h, M, A, x, dt)
    return h


@pytest.mark.parametrize("seed", range(4))
def test_dia_input_random(mh, seed):
    rng = synth.Rng(seed, 23)
    n = int(rng.integers(1, 2, 260)[0])
    k = int(rng.integers(1, 1, 12)[0])
    offs = sorted({int(o) for o in rng.integers(k, -(n - 1), n)} | {0, n - 1, -(n - 1)})
    x = synth.uniform_vector(n, seed)
    for zr in (0.0, 0.3, 0.9):
        off, val = synth.dia_matrix(n, offs, seed=seed, zero_rate=zr)
        for n_b in sorted({1, 3, 8, 64, 100, n, 2 * n + 1}):
            for theta in (0.0, 0.5, 0.9):
                for dt in ("f64", "f32", "bf16"):
                    _dia_case(mh, n, off, val, n_b, theta, dt, x if theta == 0.5 else None)


def test_dia_input_paper_stencils(mh):
    for dim in (1, 2, 3):
        n = 50000
        off, val = synth.dia_matrix(n, synth.paper_stencil_offsets(n, dim), seed=dim,
                                    zero_rate=0.1)
        x = synth.uniform_vector(n, dim)
        for n_b in (10, 500, 4096):
            for dt in ("f64", "f32", "bf16"):
                _dia_case(mh, n, off, val, n_b, 0.6, dt, x)


def test_dia_input_large_equals_csr_build(mh):
    # 3D 7-point stencil, n = 1e7, 5% zeros: the handle from DIA input equals
    # the handle built from the CSR of the same entries
    t = torch()
    n = 10_000_000
    off, val = synth.dia_matrix(n, synth.paper_stencil_offsets(n, 3), seed=5, zero_rate=0.05)
    rp, col, v = oracle.dia_to_csr(n, off, val)
    h1 = mh.mhdc_build_dia(n, t.from_numpy(off).cuda(), t.from_numpy(val).cuda(), 4096, 0.6)
    h2 = mh.mhdc_build(n, t.from_numpy(rp).cuda(), t.from_numpy(col).cuda(), t.from_numpy(v).cuda(),
                       4096, 0.6)
    E1, E2 = mh.mhdc_export(h1), mh.mhdc_export(h2)
    for k in E1:
        assert np.array_equal(np.asarray(E1[k]).view(np.uint8), np.asarray(E2[k]).view(np.uint8)), k
    A = synth.CSR(n, rp, col, v, {})
    x = synth.uniform_vector(n, 6)
    y = y_empty(n, "f64")
    mh.mhdc_spmv(h1, t.from_numpy(x).cuda(), y)
    ref = oracle.csr_spmv(A, x)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= oracle.FP64_ROW_TOL * oracle.csr_absrow(A, x))


def test_dia_input_rejects_bad_offsets(mh):
    t = torch()
    n = 100
    _, val = synth.dia_matrix(n, [-1, 0, 1], seed=1)
    dv = t.from_numpy(val).cuda()
    for offs in ([0, -1, 1], [-1, 0, 0], [-100, 0, 1], [-1, 0, 100]):
        with pytest.raises(mh.MhdcError) as e:
            mh.mhdc_build_dia(n, t.tensor(offs, dtype=t.int32, device="cuda"), dv, 16, 0.5)
        assert e.value.code == mh.MHDC_ERR_INVALID_ARG
    # no diagonals at all: every row empty
    h = mh.mhdc_build_dia(n, t.zeros(0, dtype=t.int32, device="cuda"),
                          t.zeros(1, dtype=t.float64, device="cuda"), 16, 0.5)
    assert h.info["nnz"] == 0 and h.info["P"] == 0
    y = y_empty(n, "f64")
    mh.mhdc_spmv(h, t.ones(n, dtype=t.float64, device="cuda"), y)
    assert t.all(y == 0)


def test_dia_input_block_wider_than_matrix_and_single_row(mh):
    for n, offs in ((1, [0]), (7, [-6, -1, 0, 6]), (300, [-299, -150, 0, 1, 299])):
        off, val = synth.dia_matrix(n, offs, seed=n, zero_rate=0.2)
        x = synth.uniform_vector(n, 3)
        for n_b in (1, n, 4 * n + 3):
            for dt in ("f64", "bf16"):
                _dia_case(mh, n, off, val, n_b, 0.5, dt, x)
