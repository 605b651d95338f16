"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Conversion (mhdc_build / hdc_build): every array bit-exact.  Products:
FP64 within 1e-12 * sum_j |a_ij||x_j| per row; FP32/BF16 within the stated
per-row bound (rounding of the stored values and FP32 accumulation).
"""
import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden
from gpu_util import (build, check_build, check_spmm, check_spmv, dev_csr, torch, x_device,
                      y_empty)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    t = torch()
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2105_04937_gb300 as m
    m.lib()  # raises if the library was not built
    return m


DTYPES = ("f64", "f32", "bf16")


# ---------------------------------------------------------------- worked example

def test_example_matches_fig12_on_gpu(mh):
    g = read_golden("example_mhdc_bl4_theta06.txt")
    A = synth.example_matrix()
    h = build(mh, A, 4, 0.6)
    E = mh.mhdc_export(h)
    assert E["dia_ptr"].tolist() == g["dia_ptr"]
    assert E["dia_offset"].tolist() == g["dia_col_offset"]
    assert E["dia_val"].tolist() == sum((g[f"dia_val{k}"] for k in range(5)), [])
    assert E["csr_val"].tolist() == g["csr_val"]
    assert E["csr_col"].tolist() == g["csr_col_ind"]
    assert E["csr_row_ptr"].tolist() == g["csr_row_ptr"]
    # the model statistics of this example (Sec. 5.3): P = 5 partial diagonals
    # of 4 slots, alpha = stored entries / slots, beta = remainder share
    st = mh.mhdc_stats(h)
    P, rem = len(g["dia_col_offset"]), len(g["csr_val"])
    assert st["P"] == P and st["alpha"] == (A.nnz - rem) / (P * 4) and st["beta"] == rem / A.nnz
    assert st["bytes"] == h.info["bytes_model"]


@pytest.mark.parametrize("mode", ["block", "global"])
def test_example_every_block_size(mh, mode):
    A = synth.example_matrix()
    x = np.arange(1.0, 9.0)
    for bl in range(1, 11):
        for theta in (0.0, 0.3, 0.6, 1.0, 1.5):
            h, M = check_build(mh, A, bl, theta, "f64", mode)
            y = check_spmv(mh, h, M, A, x, "f64")
            dense = np.zeros((8, 8))
            dense[A.rows(), A.col] = A.val
            assert y.tolist() == (dense @ x).tolist()


# ---------------------------------------------------------------- random small

@pytest.mark.parametrize("seed", range(8))
def test_random_small(mh, seed):
    rng = synth.Rng(seed, 5)
    n = int(rng.integers(1, 1, 300)[0])
    A = synth.random_sparse(n, 0.03, seed=seed, diag_bias=0.7)
    x = synth.uniform_vector(n, seed)
    for n_b in sorted({1, 3, 8, 64, 100, n, 2 * n + 1}):
        for theta in (0.0, 0.5, 0.9):
            for dt in DTYPES:
                h, M = check_build(mh, A, n_b, theta, dt)
                check_spmv(mh, h, M, A, x, dt)


# ---------------------------------------------------------------- workloads

@pytest.mark.parametrize("dt", DTYPES)
def test_stencil7_32_full(mh, dt):
    # 7-point FDM on 32^3, n_b = 1024, theta = 0.6 (the small workload)
    A = synth.config_matrix("stencil7_32")
    h, M = check_build(mh, A, 1024, 0.6, dt)
    assert M["nnz_rem"] == 0 and M["P"] == 222
    check_spmv(mh, h, M, A, synth.uniform_vector(A.n, 0), dt)


@pytest.mark.parametrize("n_b", [256, 1000, 4096, 8192, 12345])
def test_stencil27_scaled(mh, n_b):
    A = synth.config_matrix("stencil27_128", scale=0.375)   # 48^3 rows, 27-point
    x = synth.uniform_vector(A.n, 1)
    for dt in DTYPES:
        for theta in (0.5, 0.9):
            h, M = check_build(mh, A, n_b, theta, dt)
            check_spmv(mh, h, M, A, x, dt)
    h, M = check_build(mh, A, n_b, 0.6, "f64", "global")
    check_spmv(mh, h, M, A, x, "f64")


@pytest.mark.parametrize("n_b", [2048, 8192])
def test_scattered_scaled(mh, n_b):
    # n_b = 8192 has > 12288 distinct offsets per block: the global-table path
    A = synth.config_matrix("scattered_4m", scale=1 / 64)
    x = synth.loguniform_vector(A.n, 2)
    for dt in DTYPES:
        h, M = check_build(mh, A, n_b, 0.6, dt)
        check_spmv(mh, h, M, A, x, dt)


def test_paper_stencils(mh):
    for dim in (1, 2, 3):
        A = synth.paper_stencil(50000, dim)
        x = synth.uniform_vector(A.n, dim)
        for n_b in (10, 500, 5000):
            h, M = check_build(mh, A, n_b, 0.6, "f64")
            check_spmv(mh, h, M, A, x, "f64")


# ---------------------------------------------------------------- full size

def test_stencil27_128_full_size(mh):
    # the benchmark workload, in the benchmark's configuration
    A = synth.config_matrix("stencil27_128")
    h, M = check_build(mh, A, 4096, 0.6, "f64")
    check_spmv(mh, h, M, A, synth.uniform_vector(A.n, 1), "f64")
    # HDC over the same matrix (blocked, global selection)
    h2, M2 = check_build(mh, A, 4096, 0.6, "f64", "global")
    check_spmv(mh, h2, M2, A, synth.uniform_vector(A.n, 1), "f64")


@pytest.mark.parametrize("dt", DTYPES)
def test_scattered_4m_full_size(mh, dt):
    A = synth.config_matrix("scattered_4m")
    h, M = check_build(mh, A, 2048, 0.6, dt)
    check_spmv(mh, h, M, A, synth.loguniform_vector(A.n, 2), dt)


# ---------------------------------------------------------------- CSR baseline

@pytest.mark.parametrize("name,scale", [("stencil7_32", 1.0), ("stencil27_128", 1.0),
                                        ("scattered_4m", 1.0)])
def test_csr_spmv(mh, name, scale):
    A = synth.config_matrix(name, scale)
    x = synth.uniform_vector(A.n, 3)
    rp, col, val = dev_csr(A)
    t = torch()
    xd = t.from_numpy(x).cuda()
    y = y_empty(A.n, "f64")
    mh.csr_spmv(A.n, rp, col, val, xd, y)
    yg = y.cpu().numpy()
    ref = oracle.csr_spmv(A, x)
    assert np.all(np.abs(yg - ref) <= oracle.FP64_ROW_TOL * oracle.csr_absrow(A, x))


def test_csr_spmv_row_lengths(mh):
    # every lanes-per-row choice (mean row length 1 .. 60)
    t = torch()
    for density in (0.0005, 0.002, 0.004, 0.008, 0.02, 0.06):
        A = synth.random_sparse(1000, density, seed=7, diag_bias=0.5)
        x = synth.uniform_vector(A.n, 3)
        rp, col, val = dev_csr(A)
        y = y_empty(A.n, "f64")
        mh.csr_spmv(A.n, rp, col, val, t.from_numpy(x).cuda(), y)
        ref = oracle.csr_spmv(A, x)
        assert np.all(np.abs(y.cpu().numpy() - ref) <= oracle.FP64_ROW_TOL * oracle.csr_absrow(A, x))


# ---------------------------------------------------------------- edge cases

def test_empty_matrix(mh):
    A = synth.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    t = torch()
    rp = t.zeros(1, dtype=t.int32, device="cuda")
    col = t.zeros(1, dtype=t.int32, device="cuda")
    val = t.zeros(1, dtype=t.float64, device="cuda")
    h = mh.mhdc_build(0, rp, col, val, 16, 0.6)
    assert h.info["P"] == 0 and h.info["nnz"] == 0
    x = t.zeros(1, dtype=t.float64, device="cuda")
    y = t.zeros(1, dtype=t.float64, device="cuda")
    mh.mhdc_spmv(h, x[:0], y[:0])
    del A


def test_matrix_without_entries_and_empty_rows(mh):
    n = 777
    A = synth.CSR(n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    h, M = check_build(mh, A, 64, 0.5)
    y = check_spmv(mh, h, M, A, synth.uniform_vector(n, 0), "f64")
    assert np.all(y == 0.0)
    # only a few rows hold entries
    d = np.zeros((n, n))
    d[5, 7] = 1.5
    d[700, 3] = -2.0
    d[776, 776] = 3.0
    B = synth.from_dense(d)
    for n_b in (1, 64, 777, 1000):
        h, M = check_build(mh, B, n_b, 0.0)
        check_spmv(mh, h, M, B, synth.uniform_vector(n, 1), "f64")


def test_bad_csr_is_rejected(mh):
    A = synth.example_matrix()
    t = torch()
    cases = []
    col = A.col.copy(); col[5] = 8; cases.append((A.row_ptr, col))
    col = A.col.copy(); col[1] = 0; cases.append((A.row_ptr, col))
    col = A.col.copy(); col[0], col[1] = col[1], col[0]; cases.append((A.row_ptr, col))
    rp = A.row_ptr.copy(); rp[3], rp[4] = rp[4], rp[3]; cases.append((rp, A.col))
    rp = A.row_ptr.copy(); rp[0] = 1; cases.append((rp, A.col))
    for rp, col in cases:
        with pytest.raises(mh.MhdcError) as e:
            mh.mhdc_build(8, t.from_numpy(rp.astype(np.int32)).cuda(),
                          t.from_numpy(col.astype(np.int32)).cuda(),
                          t.from_numpy(A.val).cuda(), 4, 0.6)
        assert e.value.code == -2
    rp_d, col_d, val_d = dev_csr(A)
    for kw in (dict(n_b=0), dict(theta=-1.0), dict(theta=float("nan")), dict(dtype=7)):
        args = dict(n_b=4, theta=0.6, dtype="f64")
        args.update(kw)
        with pytest.raises(mh.MhdcError) as e:
            mh.mhdc_build(8, rp_d, col_d, val_d, args["n_b"], args["theta"], args["dtype"])
        assert e.value.code == -1


def test_misaligned_x_gives_identical_result(mh):
    A = synth.config_matrix("stencil27_128", scale=0.25)
    t = torch()
    for dt in DTYPES:
        h = build(mh, A, 4096, 0.6, dt)
        xd, _ = x_device(synth.uniform_vector(A.n, 9), dt)
        buf = t.zeros(A.n + 1, dtype=xd.dtype, device="cuda")
        buf[1:] = xd
        for v in range(-1, mh.MHDC_NUM_VARIANTS):
            mh.mhdc_set_variant(h, v)
            y1 = y_empty(A.n, dt)
            y2 = y_empty(A.n, dt)
            mh.mhdc_spmv(h, xd, y1)
            mh.mhdc_spmv(h, buf[1:], y2)
            assert t.equal(y1, y2), (dt, v)
        # an x far outside the emulation window sends the rows that read it
        # down the native path, which also reads the unaligned x: those rows
        # equal native FP64 bit for bit, the others stay within tolerance
        if dt == "f64":
            j = A.n // 2
            buf[1 + j] = 1e300
            xal = buf[1:].clone()
            rows_of = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
            reads_j = t.from_numpy(np.unique(rows_of[A.col == j])).cuda()
            xh = xal.cpu().numpy()
            tol = t.from_numpy(oracle.FP64_ROW_TOL * oracle.csr_absrow(A, xh)).cuda()
            for v in mh.EMULATED_VARIANTS:
                mh.mhdc_set_variant(h, v)
                y1 = y_empty(A.n, dt)
                mh.mhdc_spmv(h, buf[1:], y1)
                y3 = y_empty(A.n, dt)
                mh.mhdc_spmv(h, xal, y3)
                assert t.equal(y1, y3), v
                mh.mhdc_set_variant(h, -1)
                y2 = y_empty(A.n, dt)
                mh.mhdc_spmv(h, buf[1:], y2)
                assert t.equal(y1[reads_j], y2[reads_j]), v
                assert bool(((y1 - y2).abs() <= 2 * tol).all()), v
        mh.mhdc_check(h)


def test_staged_x_variants_edge_cases(mh):
    # variants 16-19 (values and x windows in shared memory): bit-identical to
    # the register kernel on small and ragged shapes -- n not a multiple of
    # the 16-byte vector, n_b below and above the unit size, windows reaching
    # outside [0, n), diagonals far apart (one window each), global selection
    t = torch()
    cases = []
    for seed in range(4):
        rng = synth.Rng(seed, 41)
        n = int(rng.integers(1, 1, 3000)[0])
        A = synth.random_sparse(n, 0.01, seed=200 + seed, diag_bias=0.7)
        cases += [(A, n_b, th, mode) for n_b in (8, 64, 1024, 3 * n + 8)
                  for th, mode in ((0.0, "block"), (0.02, "block"), (0.5, "global"))]
    cases += [(synth.paper_stencil(50001, d), n_b, 0.0, "block") for d in (1, 3) for n_b in (16, 4096)]
    cases.append((synth.config_matrix("stencil27_128", 0.25), 4096, 0.6, "block"))
    cases.append((synth.config_matrix("scattered_4m", 1 / 128), 2048, 0.6, "block"))
    for A, n_b, th, mode in cases:
        for dt in DTYPES:
            h, M = check_build(mh, A, n_b, th, dt, mode)
            xd, _ = x_device(synth.loguniform_vector(A.n, 3), dt)
            mh.mhdc_set_variant(h, 1)
            y0 = y_empty(A.n, dt)
            mh.mhdc_spmv(h, xd, y0)
            for v in mh.XW_VARIANTS:
                mh.mhdc_set_variant(h, v)
                y = y_empty(A.n, dt)
                mh.mhdc_spmv(h, xd, y)
                t.cuda.synchronize()
                mh.mhdc_check(h)
                assert t.equal(y, y0), (A.n, n_b, th, mode, dt, v)
            check_spmv(mh, h, M, A, synth.uniform_vector(A.n, 4), dt)


def test_repeatable_and_host_path(mh):
    A = synth.config_matrix("stencil27_128", scale=0.25)
    t = torch()
    for dt in DTYPES:
        h = build(mh, A, 2048, 0.6, dt)
        xd, _ = x_device(synth.uniform_vector(A.n, 4), dt)
        y1 = y_empty(A.n, dt)
        y2 = y_empty(A.n, dt)
        mh.mhdc_spmv(h, xd, y1)
        mh.mhdc_spmv(h, xd, y2)
        assert t.equal(y1, y2)
        xh = xd.cpu().pin_memory()
        yh = t.empty(A.n, dtype=y1.dtype).pin_memory()
        mh.mhdc_spmv_host(h, xh, yh)
        assert t.equal(yh, y1.cpu())


def test_host_async_pipeline(mh):
    # ten products on host buffers through the pipelined entry point, with a
    # ring of four buffer pairs (a pair is reused four calls later, after the
    # call that used it has been reported complete by a later call)
    t = torch()
    A = synth.config_matrix("stencil27_128", scale=0.25)
    for dt in DTYPES:
        h = build(mh, A, 4096, 0.6, dt)
        K, R = 10, 4
        xs = [x_device(synth.uniform_vector(A.n, 40 + k), dt)[0] for k in range(K)]
        ref = []
        for xd in xs:
            y = y_empty(A.n, dt)
            mh.mhdc_spmv(h, xd, y)
            ref.append(y.cpu())
        ring_x = [t.empty_like(xs[0], device="cpu").pin_memory() for _ in range(R)]
        ring_y = [t.empty(A.n, dtype=ref[0].dtype).pin_memory() for _ in range(R)]
        got = [None] * K
        for k in range(K):
            if k >= R:
                got[k - R] = ring_y[k % R].clone()   # finished: three calls were queued since
            ring_x[k % R].copy_(xs[k].cpu())
            mh.mhdc_spmv_host_async(h, ring_x[k % R], ring_y[k % R])
        mh.mhdc_host_wait(h)
        for k in range(K - R, K):
            got[k] = ring_y[k % R].clone()
        for k in range(K):
            assert t.equal(got[k], ref[k]), (dt, k)


def test_stream_bench(mh):
    t = torch()
    N = 1 << 20
    Av = t.arange(N, dtype=t.float64, device="cuda")
    Bv = t.full((N,), 2.0, dtype=t.float64, device="cuda")
    I = t.arange(N, dtype=t.int32, device="cuda")
    for ind in (False, True):
        Cv = t.ones(N, dtype=t.float64, device="cuda")
        mh.mhdc_stream_bench(Av, Bv, I, Cv, ind)
        ref = oracle.stream_indirect(Av.cpu().numpy(), Bv.cpu().numpy(), I.cpu().numpy(),
                                     np.ones(N)) if ind else \
            oracle.stream_direct(Av.cpu().numpy(), Bv.cpu().numpy(), np.ones(N))
        assert np.array_equal(Cv.cpu().numpy(), ref)


def test_every_variant_is_bit_identical_and_tune_picks_one(mh):
    t = torch()
    for name, scale, n_b in (("stencil27_128", 0.375, 4096), ("scattered_4m", 1 / 64, 2048),
                             ("stencil7_32", 1.0, 1024)):
        A = synth.config_matrix(name, scale)
        for dt in DTYPES:
            h, M = check_build(mh, A, n_b, 0.6, dt)
            xd, _ = x_device(synth.uniform_vector(A.n, 5), dt)
            ys = []
            # variants 0-9 share the arithmetic; 10-15 emulate FP64 (FP64
            # handles) and fall back to the default elsewhere
            vs = (-1,) + (mh.NATIVE_VARIANTS if dt == "f64" else tuple(range(mh.MHDC_NUM_VARIANTS)))
            for v in vs:
                mh.mhdc_set_variant(h, v)
                y = y_empty(A.n, dt)
                mh.mhdc_spmv(h, xd, y)
                ys.append(y)
            for y in ys[1:]:
                assert t.equal(y, ys[0]), (name, dt)
            mh.mhdc_set_variant(h, -1)
            check_spmv(mh, h, M, A, synth.uniform_vector(A.n, 5), dt)
            best, times = mh.mhdc_tune(h, xd, ys[0])
            assert 0 <= best < mh.MHDC_NUM_VARIANTS and h.info["variant"] == best
            assert all(tt > 0 for tt in times)
            if best not in mh.EMULATED_VARIANTS or dt != "f64":
                y = y_empty(A.n, dt)
                mh.mhdc_spmv(h, xd, y)
                assert t.equal(y, ys[1])
            else:  # an emulated variant won: the FP64 tolerance holds
                check_spmv(mh, h, M, A, synth.uniform_vector(A.n, 5), dt)
    with pytest.raises(mh.MhdcError):
        mh.mhdc_set_variant(h, mh.MHDC_NUM_VARIANTS)


def test_persistent_tiles_on_a_remainder_heavy_matrix(mh):
    # A matrix whose CSR remainder holds 21 % of the nonzeros (enough 8-warp
    # CTAs) runs its one-vector tiles (variants 0 and 5, and the emulated 10
    # and 11) with persistent tile scheduling: the same bits as the tiles that
    # take one tile a warp (variants 1-4, 6-9; emulated 12), launch after
    # launch (the tile counter is cleared by each launch), and within the
    # oracle's bound.
    t = torch()
    A = synth.config_matrix("scattered_4m", 1 / 4)
    x = synth.loguniform_vector(A.n, 2)
    for dt in DTYPES:
        h, M = check_build(mh, A, 2048, 0.6, dt)
        assert M["nnz_rem"] * 20 >= A.nnz
        xd, _ = x_device(x, dt)
        ref = None
        for v in mh.NATIVE_VARIANTS:
            mh.mhdc_set_variant(h, v)
            for rep in range(3):
                y = y_empty(A.n, dt)
                mh.mhdc_spmv(h, xd, y)
                if ref is None:
                    ref = y
                assert t.equal(y, ref), (dt, v, rep)
        mh.mhdc_set_variant(h, 5)
        check_spmv(mh, h, M, A, x, dt)
        if dt == "f64":
            ys = []
            for v in (10, 11, 12):
                mh.mhdc_set_variant(h, v)
                for rep in range(3):
                    y = y_empty(A.n, dt)
                    mh.mhdc_spmv(h, xd, y)
                    ys.append(y)
            for y in ys[1:]:
                assert t.equal(y, ys[0])
            mh.mhdc_set_variant(h, 11)
            check_spmv(mh, h, M, A, x, dt)
        mh.mhdc_check(h)
        h.destroy()


def test_read_bench_xor(mh):
    t = torch()
    N = (1 << 22) + 6
    A = t.from_numpy(synth.uniform_vector(N, 8)).cuda()
    out = t.zeros(mh.mhdc_read_bench_ctas(), dtype=t.int64, device="cuda")
    mh.mhdc_read_bench(A, out)
    got = np.bitwise_xor.reduce(out.cpu().numpy().view(np.uint64))
    ref = np.bitwise_xor.reduce(A.cpu().numpy().view(np.uint64))
    assert got == ref


def test_fma_probe_values(mh):
    t = torch()
    ctas = mh.mhdc_read_bench_ctas()
    for fp64 in (True, False):
        out = t.zeros(ctas * 256, dtype=t.float64 if fp64 else t.float32, device="cuda")
        mh.mhdc_fma_bench(fp64, 3, out)
        tid = np.tile(np.arange(256), ctas).astype(np.float64)
        # c_k = k/8 + tid + 3 * (1 + tid) * 0.5; out = sum_k c_k
        ref = sum(k * 0.125 + tid + 3 * (1.0 + tid) * 0.5 for k in range(8))
        assert np.allclose(out.cpu().numpy(), ref, rtol=1e-6)


# ---------------------------------------------------------------- emulated FP64

def _emulated_cases():
    yield "example", synth.example_matrix(), 4, np.arange(1.0, 9.0)
    for seed in range(3):
        A = synth.random_sparse(150 + 40 * seed, 0.03, seed=seed, diag_bias=0.7)
        yield f"random{seed}", A, 8, synth.uniform_vector(A.n, seed)
    A = synth.config_matrix("stencil7_32")
    yield "stencil7_32", A, 1024, synth.uniform_vector(A.n, 0)
    A = synth.config_matrix("stencil27_128", scale=0.375)
    for n_b in (256, 1000, 4096, 12346):
        yield f"stencil27_48^3_nb{n_b}", A, n_b, synth.uniform_vector(A.n, 1)
    A = synth.config_matrix("scattered_4m", scale=1 / 64)
    yield "scattered", A, 2048, synth.loguniform_vector(A.n, 2)
    A = synth.paper_stencil(50000, 3)
    yield "paper3d", A, 500, synth.uniform_vector(A.n, 3)


def test_emulated_fp64_meets_the_fp64_tolerance(mh):
    for name, A, n_b, x in _emulated_cases():
        for mode in ("block", "global"):
            h, M = check_build(mh, A, n_b, 0.6, "f64", mode)
            assert h.info["emulated_ok"] == -1, name   # made on first use
            mh.mhdc_set_variant(h, mh.FIRST_EMULATED_VARIANT)
            assert h.info["emulated_ok"] == 1, name
            for v in mh.EMULATED_VARIANTS:
                mh.mhdc_set_variant(h, v)
                check_spmv(mh, h, M, A, x, "f64")


def test_emulated_fp64_full_size(mh):
    A = synth.config_matrix("stencil27_128")
    h, M = check_build(mh, A, 4096, 0.6, "f64")
    mh.mhdc_set_variant(h, mh.FIRST_EMULATED_VARIANT)
    assert h.info["emulated_ok"] == 1
    for v in mh.EMULATED_VARIANTS:
        mh.mhdc_set_variant(h, v)
        check_spmv(mh, h, M, A, synth.uniform_vector(A.n, 1), "f64")


def _native_and_emulated(mh, h, x):
    t = torch()
    mh.mhdc_set_variant(h, -1)
    y0 = y_empty(h.n, "f64")
    mh.mhdc_spmv(h, x, y0)
    out = []
    for v in mh.EMULATED_VARIANTS:
        mh.mhdc_set_variant(h, v)
        y = y_empty(h.n, "f64")
        mh.mhdc_spmv(h, x, y)
        out.append(y)
    t.cuda.synchronize()
    return y0, out


def test_emulated_fp64_falls_back_outside_its_window(mh):
    # An x outside the window is marked NaN by the split, so exactly the rows
    # that read it (through an entry or a padded slot of its column) come out
    # NaN in FP32 pairs and are recomputed with native FP64 arithmetic: the
    # rows holding an entry in that column equal native FP64 bit for bit (NaN
    # where native has NaN), every other row stays within the FP64 tolerance.
    t = torch()
    A = synth.config_matrix("stencil27_128", scale=0.25)
    h = build(mh, A, 4096, 0.6, "f64")
    mh.mhdc_set_variant(h, mh.FIRST_EMULATED_VARIANT)
    assert h.info["emulated_ok"] == 1
    base = synth.uniform_vector(A.n, 6)
    y0, ys = _native_and_emulated(mh, h, t.from_numpy(base).cuda())
    for v, y in zip(mh.EMULATED_VARIANTS, ys):
        assert not t.equal(y, y0), v
    j = A.n // 3
    rows_of = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    reads_j = np.unique(rows_of[A.col == j])
    assert reads_j.size > 1
    for bad in (1e30, -3e19, 1e-20, 2.0 ** -60, float("inf"), float("nan")):
        xb = base.copy()
        xb[j] = bad
        xd = t.from_numpy(xb).cuda()
        y0, ys = _native_and_emulated(mh, h, xd)
        a = y0.cpu().numpy()
        with np.errstate(invalid="ignore", over="ignore"):
            tol = oracle.FP64_ROW_TOL * oracle.csr_absrow(A, xb)
        fin = np.isfinite(a) & np.isfinite(tol)
        for v, y in zip(mh.EMULATED_VARIANTS, ys):
            b = y.cpu().numpy()
            assert np.array_equal(np.isnan(a), np.isnan(b)), (bad, v)
            assert np.array_equal(a[reads_j], b[reads_j], equal_nan=True), (bad, v)
            assert np.all(np.abs(a[fin] - b[fin]) <= 2 * tol[fin]), (bad, v)
        mh.mhdc_check(h)
    # a good x again: every row emulated (some rows differ from native FP64)
    xd = t.from_numpy(base).cuda()
    y0, ys = _native_and_emulated(mh, h, xd)
    for v, y in zip(mh.EMULATED_VARIANTS, ys):
        assert not t.equal(y, y0), v
    M = oracle.convert(A, 4096, 0.6, "f64")
    for v in mh.EMULATED_VARIANTS:
        mh.mhdc_set_variant(h, v)
        check_spmv(mh, h, M, A, base, "f64")


def test_emulated_chain_and_graph_replay(mh):
    # Products whose x is the previous product's y, launched back to back
    # (the split and the product are programmatic dependent launches, no host
    # wait between calls), equal the same chain with a device
    # synchronisation after every product, bit for bit.  So does the chain
    # captured in a CUDA graph and replayed twice: the window word and the
    # CTA ticket are left clear by every product, so a replayed product sees
    # the state a direct call sees.  Three products a chain (an odd count),
    # one-warp and 8-warp CTAs (the two matrix sizes), every emulated
    # variant; the first product differs from native FP64 as in the test
    # above, so the emulated arithmetic ran.
    t = torch()
    steps = 3
    for scale in (0.25, 0.75):
        A = synth.config_matrix("stencil27_128", scale=scale)
        h = build(mh, A, 4096, 0.6, "f64")
        x0 = t.from_numpy(synth.uniform_vector(A.n, 6)).cuda()
        mh.mhdc_set_variant(h, -1)
        y_native = y_empty(A.n, "f64")
        mh.mhdc_spmv(h, x0, y_native)
        for v in mh.EMULATED_VARIANTS:
            mh.mhdc_set_variant(h, v)

            def chain(sync):
                a, b = x0.clone(), t.empty_like(x0)
                firsts = []
                for _ in range(steps):
                    mh.mhdc_spmv(h, a, b)
                    if sync:
                        t.cuda.synchronize()
                        if not firsts:
                            firsts.append(b.clone())
                    a, b = b, a
                t.cuda.synchronize()
                return a.clone(), (firsts[0] if firsts else None)

            ref, first = chain(True)
            assert not t.equal(first, y_native), (scale, v)
            got, _ = chain(False)
            assert t.equal(got, ref), (scale, v)
            a, b = x0.clone(), t.empty_like(x0)
            g = t.cuda.CUDAGraph()
            with t.cuda.graph(g):
                mh.mhdc_spmv(h, a, b)
                mh.mhdc_spmv(h, b, a)
                mh.mhdc_spmv(h, a, b)
            for _ in range(2):
                a.copy_(x0)
                g.replay()
                t.cuda.synchronize()
                assert t.equal(b, ref), (scale, v)
            mh.mhdc_check(h)
        h.destroy()


def test_emulated_fp64_disabled_by_values_or_row_length(mh):
    t = torch()
    A = synth.config_matrix("stencil7_32", scale=0.5)
    tiny = synth.CSR(A.n, A.row_ptr, A.col, A.val * 1e-17)
    long_rows = synth.random_sparse(300, 0.3, seed=3)          # ~90 terms per row
    for M_ in (tiny, long_rows):
        h = build(mh, M_, 64, 0.6, "f64")
        mh.mhdc_set_variant(h, mh.FIRST_EMULATED_VARIANT)
        assert h.info["emulated_ok"] == 0
        xd = t.from_numpy(synth.uniform_vector(M_.n, 2)).cuda()
        y0, ys = _native_and_emulated(mh, h, xd)
        for y in ys:
            assert t.equal(y, y0)


# ---------------------------------------------------------------- SpMM

@pytest.mark.parametrize("dt", DTYPES)
def test_spmm_matches_columnwise_oracle(mh, dt):
    cases = [(synth.config_matrix("stencil27_128", scale=0.25), 4096),
             (synth.config_matrix("scattered_4m", scale=1 / 256), 2048),
             (synth.random_sparse(123, 0.05, seed=4, diag_bias=0.5), 10),
             (synth.config_matrix("stencil7_32", scale=0.5), 999)]
    for A, n_b in cases:
        h, M = check_build(mh, A, n_b, 0.6, dt)
        for k in (1, 2, 3, 4, 5, 8, 13, 16, 17, 33):
            X = synth.uniform_vector(A.n * k, 40 + k).reshape(A.n, k)
            check_spmm(mh, h, M, A, X, dt)
        X = synth.uniform_vector(A.n * 6, 77).reshape(A.n, 6)
        check_spmm(mh, h, M, A, X, dt, pad=3)


def test_spmm_full_size_fp32_k16(mh):
    # the 128^3 27-point matrix with 16 right-hand sides in FP32
    A = synth.config_matrix("stencil27_128")
    h, M = check_build(mh, A, 4096, 0.6, "f32")
    X = synth.uniform_vector(A.n * 16, 5).reshape(A.n, 16)
    check_spmm(mh, h, M, A, X, "f32")


@pytest.mark.parametrize("dt", DTYPES)
def test_spmm_every_tile_shape(mh, dt):
    # every SpMM tile shape sums each (row, column) in the same order: the
    # shapes agree bit for bit, and each meets the column-wise bounds; X and Y
    # with a padded leading dimension take the element-by-element path
    t = torch()
    cases = [(synth.config_matrix("stencil27_128", scale=0.2), 1000),
             (synth.random_sparse(301, 0.04, seed=8, diag_bias=0.6), 37),
             (synth.config_matrix("scattered_4m", scale=1 / 512), 2048)]
    for A, n_b in cases:
        h, M = check_build(mh, A, n_b, 0.6, dt)
        for k in (2, 4, 8, 12, 16, 20):
            X = synth.uniform_vector(A.n * k, 90 + k).reshape(A.n, k)
            Ys = []
            for v in range(mh.MHDC_NUM_SPMM_VARIANTS):
                mh.mhdc_spmm_set_variant(h, v)
                check_spmm(mh, h, M, A, X, dt, pad=1 if k == 12 else 0)
                xd, _ = x_device(X.ravel(), dt)
                Xd = xd.view(A.n, k)
                Y = t.empty((A.n, k), dtype=t.float64 if dt == "f64" else t.float32,
                            device="cuda")
                mh.mhdc_spmm(h, Xd, Y)
                Ys.append(Y)
            t.cuda.synchronize()
            for v in range(1, len(Ys)):
                assert t.equal(Ys[v], Ys[0]), (n_b, k, v)
        best, times = mh.mhdc_spmm_tune(h, Xd, Ys[0])
        assert 0 <= best < mh.MHDC_NUM_SPMM_VARIANTS and all(tm > 0 for tm in times)
        mh.mhdc_spmm_set_variant(h, -1)
        with pytest.raises(mh.MhdcError):
            mh.mhdc_spmm_set_variant(h, mh.MHDC_NUM_SPMM_VARIANTS)


def test_spmm_k64_and_bad_args(mh):
    t = torch()
    A = synth.config_matrix("stencil7_32", scale=0.25)
    h, M = check_build(mh, A, 64, 0.6, "f64")
    X = synth.uniform_vector(A.n * 64, 9).reshape(A.n, 64)
    check_spmm(mh, h, M, A, X, "f64")
    Xd = t.zeros((A.n, 65), dtype=t.float64, device="cuda")
    Yd = t.zeros((A.n, 65), dtype=t.float64, device="cuda")
    with pytest.raises(mh.MhdcError):
        mh.mhdc_spmm(h, Xd, Yd)


# ---------------------------------------------------------------- batched

def _batch_case(mh, dt, seed):
    rng = synth.Rng(seed, 17)
    mats, hs, Ms, xs = [], [], [], []
    for q in range(10):
        e = [int(v) for v in rng.integers(3, 6, 20)]
        if q % 3 == 2:
            A = synth.random_sparse(200 + 17 * q, 0.04, seed=seed * 100 + q, diag_bias=0.6)
            n_b = 37 if q % 2 else 64        # odd n_b: element loads
        else:
            A = synth.stencil_3d(*e, 27 if q % 2 else 7, seed=seed * 100 + q, drop_rate=0.2,
                                 drop_block=256)
            n_b = (256, 1024, 100)[q % 3]
        h, M = check_build(mh, A, n_b, 0.6, dt)
        mats.append(A); hs.append(h); Ms.append(M)
        xs.append(synth.uniform_vector(A.n, seed * 100 + q))
    return mats, hs, Ms, xs


@pytest.mark.parametrize("dt", DTYPES)
def test_batch_matches_oracle_and_graph_replays(mh, dt):
    t = torch()
    mats, hs, Ms, xs = _batch_case(mh, dt, 1)
    B = mh.mhdc_batch_create(hs)
    xd = [x_device(x, dt)[0] for x in xs]
    ys = [y_empty(A.n, dt) for A in mats]
    XP, YP = mh.pointer_array(xd), mh.pointer_array(ys)
    for rep in range(2):     # the counter is reset by each launch
        mh.mhdc_batch_spmv(B, XP, YP)
        t.cuda.synchronize()
        for A, M, x, y in zip(mats, Ms, xs, ys):
            xs_w = oracle.widen(oracle.store(x, dt), dt)
            ref = oracle.mhdc_spmv(M, xs_w)
            a, terms = oracle.mhdc_absrow(M, xs_w)
            bnd = oracle.bound_vs_stored(a, terms, dt, oracle.long_remainder(M))
            assert np.all(np.abs(y.double().cpu().numpy() - ref) <= bnd)
    direct = [y.clone() for y in ys]
    for rep in range(3):
        for y in ys:
            y.fill_(float("nan"))
        mh.mhdc_batch_spmv_graph(B, XP, YP)
        t.cuda.synchronize()
        for y, d in zip(ys, direct):
            assert t.equal(y, d)
    # new x contents, same pointer arrays: the graph reads them at run time
    for x in xd:
        x.mul_(2)
    mh.mhdc_batch_spmv_graph(B, XP, YP)
    t.cuda.synchronize()
    for y, d in zip(ys, direct):
        assert t.allclose(y.double(), 2 * d.double(), rtol=1e-6 if dt != "f64" else 1e-15, atol=0)
    # one handle at a time gives the same bits
    for h, x, y in zip(hs, xd, ys):
        yy = y_empty(h.n, dt)
        mh.mhdc_set_variant(h, 5)
        mh.mhdc_spmv(h, x, yy)
        if h.info["n_b"] % {"f64": 2, "f32": 4, "bf16": 8}[dt] == 0:
            assert t.equal(yy, y)
    B.destroy()


def test_batch_64_stencils_full_size(mh):
    # 64 seeded 7-/27-point stencils, grid edges uniform in [16, 96], FP64
    t = torch()
    mats = synth.batch_matrices(64, 16, 96, seed=3)
    hs, xd, ys, xs = [], [], [], []
    for i, A in enumerate(mats):
        rp, col, val = dev_csr(A)
        hs.append(mh.mhdc_build(A.n, rp, col, val, 4096, 0.6, "f64"))
        xs.append(synth.uniform_vector(A.n, 500 + i))
        xd.append(t.from_numpy(xs[-1]).cuda())
        ys.append(y_empty(A.n, "f64"))
    B = mh.mhdc_batch_create(hs)
    mh.mhdc_batch_spmv_graph(B, mh.pointer_array(xd), mh.pointer_array(ys))
    t.cuda.synchronize()
    for A, x, y in zip(mats, xs, ys):
        ref = oracle.csr_spmv(A, x)
        assert np.all(np.abs(y.cpu().numpy() - ref) <= oracle.FP64_ROW_TOL * oracle.csr_absrow(A, x))
    B.destroy()
