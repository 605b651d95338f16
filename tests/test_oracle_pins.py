"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these retypes the oracle's own code: the expected values come from
the paper's worked example (tests/golden, Figs. 3, 4, 7, 12), from a dense
brute-force re-derivation of the selection rule, from closed forms of the
7-point Laplacian, from numpy / torch rounding, and from invariants.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden


# ---------------------------------------------------------------- worked example

def test_example_csr_matches_fig3():
    g = read_golden("example_csr.txt")
    A = synth.example_matrix()
    assert A.val.tolist() == g["val"]
    assert A.col.tolist() == g["col_ind"]
    assert A.row_ptr.tolist() == g["row_ptr"]
    assert oracle.csr_check(A.n, A.row_ptr, A.col) == 0


def test_example_dia_matches_fig4():
    # DIA = every nonzero diagonal line: HDC with a threshold that keeps any
    # diagonal holding at least one nonzero.
    g = read_golden("example_dia.txt")
    H = oracle.hdc_global(synth.example_matrix(), 1e-9)
    assert H["dia_offset"].tolist() == g["offset"]
    for k in range(5):
        assert H["dia_val"][k].tolist() == g[f"val{k}"]
    assert H["csr_col"].size == 0


def test_dia_input_of_fig4_gives_the_csr_of_fig3():
    g = read_golden("example_dia.txt")
    c = read_golden("example_csr.txt")
    dv = np.array([g[f"val{k}"] for k in range(5)], dtype=np.float64)
    rp, col, val = oracle.dia_to_csr(8, g["offset"], dv)
    assert rp.tolist() == c["row_ptr"] and col.tolist() == c["col_ind"] and val.tolist() == c["val"]


@pytest.mark.parametrize("seed", range(5))
def test_dia_input_round_trip_through_a_dense_matrix(seed):
    # a random sparse matrix written out as DIA by a dense scan (every offset
    # with a nonzero, a(i, i+d) or 0), read back: the same CSR
    A = synth.random_sparse(60 + 13 * seed, 0.05, seed=seed, diag_bias=0.5)
    d = np.zeros((A.n, A.n))
    for i in range(A.n):
        d[i, A.col[A.row_ptr[i]:A.row_ptr[i + 1]]] = A.val[A.row_ptr[i]:A.row_ptr[i + 1]]
    offs = sorted({int(j - i) for i, j in zip(*np.nonzero(d))})
    dv = np.zeros((len(offs), A.n))
    for k, o in enumerate(offs):
        for i in range(A.n):
            if 0 <= i + o < A.n:
                dv[k, i] = d[i, i + o]
    rp, col, val = oracle.dia_to_csr(A.n, offs, dv)
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
    assert np.array_equal(val, A.val)
    with pytest.raises(ValueError):
        oracle.dia_to_csr(A.n, offs[::-1], dv)


def test_example_hdc_matches_fig7():
    g = read_golden("example_hdc_theta06.txt")
    H = oracle.hdc_global(synth.example_matrix(), g["theta"][0])
    assert H["dia_offset"].tolist() == g["dia_offset"]
    assert H["dia_val"][0].tolist() == g["dia_val0"]
    assert H["dia_val"][1].tolist() == g["dia_val1"]
    assert H["csr_val"].tolist() == g["csr_val"]
    assert H["csr_col"].tolist() == g["csr_col_ind"]
    assert H["csr_row_ptr"].tolist() == g["csr_row_ptr"]


def test_example_mhdc_matches_fig12():
    g = read_golden("example_mhdc_bl4_theta06.txt")
    M = oracle.convert(synth.example_matrix(), g["bl"][0], g["theta"][0])
    bl = g["bl"][0]
    assert M["dia_ptr"].tolist() == g["dia_ptr"]
    assert M["dia_offset"].tolist() == g["dia_col_offset"]
    for k in range(5):
        assert M["dia_val"][k * bl:(k + 1) * bl].tolist() == g[f"dia_val{k}"]
    assert M["csr_val"].tolist() == g["csr_val"]
    assert M["csr_col"].tolist() == g["csr_col_ind"]
    assert M["csr_row_ptr"].tolist() == g["csr_row_ptr"]


def test_example_blocked_hdc_is_fig7_cut_into_blocks():
    # The B-HDC kernel (Fig. 10) walks the global diagonals block by block:
    # the blocked layout must hold Fig. 7's rows cut into bl-long pieces.
    g = read_golden("example_hdc_theta06.txt")
    M = oracle.convert(synth.example_matrix(), 4, 0.6, mode="global")
    assert M["dia_ptr"].tolist() == [0, 2, 4]
    assert M["dia_offset"].tolist() == [0, 2, 0, 2]
    full = [g["dia_val0"], g["dia_val1"]]
    for ib in range(2):
        for d in range(2):
            p = 2 * ib + d
            assert M["dia_val"][p * 4:(p + 1) * 4].tolist() == full[d][4 * ib:4 * ib + 4]
    assert M["csr_val"].tolist() == g["csr_val"]
    assert M["csr_row_ptr"].tolist() == g["csr_row_ptr"]


def test_example_spmv_all_formats():
    A = synth.example_matrix()
    dense = np.zeros((8, 8))
    dense[A.rows(), A.col] = A.val
    x = np.arange(1.0, 9.0)
    y = dense @ x  # small integers: exact
    assert oracle.csr_spmv(A, x).tolist() == y.tolist()
    for bl in range(1, 9):
        for theta in (0.0, 0.3, 0.6, 1.0):
            for mode in ("block", "global"):
                M = oracle.convert(A, bl, theta, mode=mode)
                assert oracle.mhdc_spmv(M, x).tolist() == y.tolist(), (bl, theta, mode)


# ---------------------------------------------------------------- brute force

def dense_convert(dense, bl, theta, mode):
    """Selection re-derived by scanning every (block, offset) of a dense matrix."""
    n = dense.shape[0]
    nb = (n + bl - 1) // bl
    dia_ptr, dia_offset, dia_val = [0], [], []
    rem_rows, rem_cols, rem_vals = [], [], []
    glob = []
    if mode == "global":
        for d in range(-(n - 1), n):
            c = sum(1 for i in range(n) if 0 <= i + d < n and dense[i, i + d] != 0)
            if c >= 1 and c >= theta * n:
                glob.append(d)
    for ib in range(nb):
        r0, r1 = ib * bl, min(n, ib * bl + bl)
        rows = r1 - r0
        if mode == "global":
            sel = list(glob)
        else:
            sel = []
            for d in range(-(n - 1), n):
                c = sum(1 for i in range(r0, r1) if 0 <= i + d < n and dense[i, i + d] != 0)
                if c >= 1 and c >= theta * rows:
                    sel.append(d)
        for d in sel:
            seg = [dense[i, i + d] if (i < n and 0 <= i + d < n) else 0.0
                   for i in range(r0, r0 + bl)]
            dia_val.extend(seg)
            dia_offset.append(d)
        dia_ptr.append(len(dia_offset))
        for i in range(r0, r1):
            for j in range(n):
                if dense[i, j] != 0 and (j - i) not in sel:
                    rem_rows.append(i)
                    rem_cols.append(j)
                    rem_vals.append(dense[i, j])
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    for i in rem_rows:
        row_ptr[i + 1] += 1
    return dict(dia_ptr=dia_ptr, dia_offset=dia_offset, dia_val=dia_val,
                csr_row_ptr=np.cumsum(row_ptr).tolist(), csr_col=rem_cols, csr_val=rem_vals)


@pytest.mark.parametrize("seed", range(6))
def test_conversion_matches_dense_brute_force(seed):
    rng = synth.Rng(seed, 99)
    n = int(rng.integers(1, 2, 24)[0])
    A = synth.random_sparse(n, 0.15, seed=seed, diag_bias=0.5)
    dense = np.zeros((n, n))
    dense[A.rows(), A.col] = A.val
    for bl in sorted({1, 2, 3, n // 2 + 1, n - 1 if n > 1 else 1, n, n + 3}):
        for theta in (0.0, 0.1, 0.34, 0.5, 0.6, 0.75, 1.0):
            for mode in ("block", "global"):
                M = oracle.convert(A, bl, theta, mode=mode)
                E = dense_convert(dense, bl, theta, mode)
                ctx = (n, bl, theta, mode)
                assert M["dia_ptr"].tolist() == E["dia_ptr"], ctx
                assert M["dia_offset"].tolist() == E["dia_offset"], ctx
                assert M["dia_val"].tolist() == E["dia_val"], ctx
                assert M["csr_row_ptr"].tolist() == E["csr_row_ptr"], ctx
                assert M["csr_col"].tolist() == E["csr_col"], ctx
                assert M["csr_val"].tolist() == E["csr_val"], ctx


@pytest.mark.parametrize("seed", range(4))
def test_spmv_matches_dense_matvec(seed):
    n = 40 + 7 * seed
    A = synth.random_sparse(n, 0.1, seed=100 + seed, diag_bias=0.6)
    dense = np.zeros((n, n))
    dense[A.rows(), A.col] = A.val
    x = synth.uniform_vector(n, seed)
    y = dense @ x
    scale = np.abs(dense) @ np.abs(x)
    tol = 1e-13 * scale + 1e-300
    assert np.all(np.abs(oracle.csr_spmv(A, x) - y) <= tol)
    for bl in (1, 5, 16, n):
        for theta in (0.2, 0.6):
            M = oracle.convert(A, bl, theta)
            assert np.all(np.abs(oracle.mhdc_spmv(M, x) - y) <= tol)
            # absrow of the structure equals the dense |A||x| (padding adds 0)
            a, t = oracle.mhdc_absrow(M, x)
            assert np.allclose(a, scale, rtol=1e-13, atol=0)


def check_csr_absrow():
    """sum_j |a_ij| |x_j| per row (the scale of every per-row tolerance, Sec.
    3.1's y = A x) against the dense |A| |x|.  Integer values and x of both
    signs make the dense product exact, so the comparison is equality: a
    doubled scale, a dropped absolute value or a missed entry all fail."""
    for seed in range(4):
        n = 30 + 11 * seed
        A = synth.random_sparse(n, 0.15, seed=200 + seed, diag_bias=0.4)
        rng = synth.Rng(300 + seed, 1)
        A.val = np.round(rng.uniform(A.nnz, -9, 9)) + np.where(rng.unit(A.nnz) < 0.5, 0.5, -0.5)
        x = np.round(rng.uniform(n, -7, 7)) - 0.25
        dense = np.zeros((n, n))
        dense[A.rows(), A.col] = A.val
        assert np.array_equal(oracle.csr_absrow(A, x), np.abs(dense) @ np.abs(x)), seed
    # float data: the same within rounding of the two summation orders
    A = synth.config_matrix("stencil7_32", scale=0.25)
    x = synth.uniform_vector(A.n, 9)
    dense_rows = np.zeros(A.n)
    np.add.at(dense_rows, A.rows(), np.abs(A.val) * np.abs(x[A.col]))
    assert np.allclose(oracle.csr_absrow(A, x), dense_rows, rtol=1e-14, atol=0)


def test_csr_absrow_matches_dense():
    check_csr_absrow()


def check_mhdc_absrow_terms():
    """Terms per row of an M-HDC structure, the k of the gamma_k bounds: every
    remainder entry of the row plus one per selected diagonal of its block,
    out-of-range positions included (Fig. 13 runs the diagonal loop over the
    whole block; the kernels add 0 * 0 there).  The selection and the
    remainder come from the dense brute-force re-derivation, and |A||x| from
    the dense matrix, so neither side reuses the oracle's conversion."""
    for seed in range(5):
        rng = synth.Rng(seed, 77)
        n = int(rng.integers(1, 8, 40)[0])
        A = synth.random_sparse(n, 0.2, seed=50 + seed, diag_bias=0.6)
        dense = np.zeros((n, n))
        dense[A.rows(), A.col] = A.val
        x = synth.uniform_vector(n, 40 + seed)
        clipped_terms = 0
        for bl in sorted({1, 3, 7, n // 2 + 1, n, n + 2}):
            for theta in (0.2, 0.5, 0.9):
                E = dense_convert(dense, bl, theta, "block")
                M = oracle.convert(A, bl, theta)
                a, t = oracle.mhdc_absrow(M, x)
                want = np.zeros(n, dtype=np.int64)
                for i in range(n):
                    ib = i // bl
                    sel = E["dia_offset"][E["dia_ptr"][ib]:E["dia_ptr"][ib + 1]]
                    rem = sum(1 for j in range(n) if dense[i, j] != 0 and (j - i) not in sel)
                    want[i] = rem + len(sel)
                    clipped_terms += sum(1 for d in sel if not 0 <= i + d < n)
                assert t.tolist() == want.tolist(), (seed, n, bl, theta)
                assert np.allclose(a, np.abs(dense) @ np.abs(x), rtol=1e-13, atol=0)
        # the cases above include diagonals that leave the matrix
        assert clipped_terms > 0


def test_mhdc_absrow_terms_match_dense_count():
    check_mhdc_absrow_terms()


# ---------------------------------------------------------------- invariants

def _nonzero_set(A):
    return set(zip(A.rows().tolist(), A.col.tolist(), A.val.tolist()))


@pytest.mark.parametrize("name,bl,theta", [
    ("stencil7_32", 1024, 0.6), ("stencil7_32", 100, 0.9), ("stencil7_32", 7, 0.3),
])
def test_round_trip_and_fill(name, bl, theta):
    A = synth.config_matrix(name, scale=0.5)
    for mode in ("block", "global"):
        M = oracle.convert(A, bl, theta, mode=mode)
        r, c, v = oracle.mhdc_to_coo(M)
        assert set(zip(r.tolist(), c.tolist(), v.tolist())) == _nonzero_set(A)
        assert r.size == A.nnz
        if mode == "block":
            # every kept partial diagonal has filling rate >= theta (Sec. 6.4.3)
            n = A.n
            for ib in range(len(M["dia_ptr"]) - 1):
                rows = min(bl, n - ib * bl)
                for p in range(M["dia_ptr"][ib], M["dia_ptr"][ib + 1]):
                    filled = np.count_nonzero(M["dia_val"][p * bl:p * bl + rows])
                    assert filled >= 1 and filled >= theta * rows


def test_scattered_round_trip_small():
    A = synth.config_matrix("scattered_4m", scale=1 / 256)
    M = oracle.convert(A, 2048, 0.6)
    r, c, v = oracle.mhdc_to_coo(M)
    assert set(zip(r.tolist(), c.tolist(), v.tolist())) == _nonzero_set(A)
    assert M["nnz_rem"] > 0 and M["P"] > 0


def test_block_equal_n_is_hdc_selection():
    # B-HDC is M-HDC with bl = n in terms of alpha and beta (Fig. 28 caption)
    for name in ("stencil7_32", "stencil27_128"):
        A = synth.config_matrix(name, scale=0.125 if name == "stencil27_128" else 0.5)
        for theta in (0.5, 0.7, 0.9):
            Mb = oracle.convert(A, A.n, theta, mode="block")
            Mg = oracle.convert(A, A.n, theta, mode="global")
            for k in ("dia_ptr", "dia_offset", "dia_val", "csr_row_ptr", "csr_col", "csr_val"):
                assert np.array_equal(Mb[k], Mg[k]), (name, theta, k)


def test_block_of_one_row_keeps_everything_in_dia():
    A = synth.random_sparse(30, 0.2, seed=5)
    for theta in (0.0, 0.5, 1.0):
        M = oracle.convert(A, 1, theta)
        assert M["nnz_rem"] == 0
        assert M["P"] == A.nnz
        assert M["dia_val"].tolist() == A.val.tolist()


def test_smaller_theta_or_block_lowers_csr_rate():
    # trend stated in Sec. 6.4.3: smaller bl and/or theta give a lower CSR rate
    A = synth.config_matrix("stencil27_128", scale=0.125)
    betas = [oracle.convert(A, 4096, t)["nnz_rem"] for t in (0.5, 0.7, 0.9)]
    assert betas == sorted(betas)
    betas = [oracle.convert(A, bl, 0.9)["nnz_rem"] for bl in (64, 512, 4096)]
    assert betas[0] <= betas[-1]


# ---------------------------------------------------------------- closed forms

def laplacian7(e):
    A = synth.stencil_3d(e, e, e, 7, seed=0)
    r = A.rows()
    A.val = np.where(A.col == r, 6.0, -1.0)
    return A


def test_laplacian_of_constant_vector():
    e = 10
    A = laplacian7(e)
    i = np.arange(A.n)
    x, y, z = i % e, (i // e) % e, i // (e * e)
    missing = sum(((c == 0) | (c == e - 1)).astype(int) for c in (x, y, z))
    ones = np.ones(A.n)
    assert oracle.csr_spmv(A, ones).tolist() == missing.astype(float).tolist()
    for bl in (1, 37, 100, 1000):
        for theta in (0.5, 0.95):
            M = oracle.convert(A, bl, theta)
            assert oracle.mhdc_spmv(M, ones).tolist() == missing.astype(float).tolist()


@pytest.mark.parametrize("p", [(1, 1, 1), (2, 3, 1), (5, 4, 7)])
def test_laplacian_sine_eigenvector(p):
    e = 12
    A = laplacian7(e)
    i = np.arange(A.n)
    coords = (i % e, (i // e) % e, i // (e * e))
    v = np.ones(A.n)
    lam = 0.0
    for c, pd in zip(coords, p):
        v *= np.sin(pd * math.pi * (c + 1) / (e + 1))
        lam += 2.0 - 2.0 * math.cos(pd * math.pi / (e + 1))
    tol = 1e-13 * 12
    assert np.max(np.abs(oracle.csr_spmv(A, v) - lam * v)) < tol
    M = oracle.convert(A, 144, 0.6)
    assert np.max(np.abs(oracle.mhdc_spmv(M, v) - lam * v)) < tol


# ---------------------------------------------------------------- rounding

def _edge_doubles():
    f32max = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    sub = 2.0 ** -149
    vals = [0.0, -0.0, 1.0, -1.0, 1 + 2 ** -24, 1 + 2 ** -23 + 2 ** -24, 1 + 3 * 2 ** -24,
            f32max, f32max * (1 + 2 ** -25), f32max * (1 + 2 ** -23), 1e300, -1e300,
            tiny, tiny * (1 - 2 ** -25), sub, sub / 2, sub * 0.5000001, sub * 1.5, sub * 2.5,
            sub / 3, 1e-320, 5e-324, float("inf"), -float("inf"), 3.14159, 1e-3, 1e3]
    return np.array(vals)


def test_round_f32_matches_numpy_cast():
    rng = synth.Rng(7, 1)
    x = np.concatenate([_edge_doubles(), rng.uniform(20000, -1, 1) * 10.0 ** rng.uniform(20000, -50, 50),
                        rng.uniform(2000, -1, 1) * 2.0 ** -140])
    ours = oracle.round_f32(x)
    ref = x.astype(np.float32)
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))
    nan = oracle.round_f32(np.array([float("nan")]))
    assert np.isnan(nan[0])


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = synth.Rng(8, 1)
    # exact BF16 ties (the 16 bits dropped are 0x8000) below and above an
    # even and an odd kept significand, both signs: nearest-even decides them
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, 3 + 2 ** -7, 3 + 3 * 2 ** -7, 2 ** -100 * (1 + 2 ** -8),
                     2 ** 100 * (1 + 5 * 2 ** -8)])
    x = np.concatenate([_edge_doubles(), ties, -ties,
                        rng.uniform(20000, -1, 1) * 10.0 ** rng.uniform(20000, -30, 30)])
    ours = oracle.round_bf16(x)
    f32 = torch.from_numpy(x.astype(np.float32))
    ref = f32.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)
    back = oracle.bf16_to_f64(ours)
    ref_back = f32.to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(back[np.isfinite(back)], ref_back[np.isfinite(ref_back)])


def test_reduced_storage_conversion_rounds_values():
    A = synth.config_matrix("scattered_4m", scale=1 / 512)
    M64 = oracle.convert(A, 2048, 0.6, "f64")
    for dt in ("f32", "bf16"):
        M = oracle.convert(A, 2048, 0.6, dt)
        assert np.array_equal(M["dia_ptr"], M64["dia_ptr"])
        assert np.array_equal(M["csr_col"], M64["csr_col"])
        assert np.array_equal(oracle.widen(M["dia_val"], dt),
                              oracle.widen(oracle.store(M64["dia_val"], dt), dt))
        assert np.array_equal(oracle.widen(M["csr_val"], dt),
                              oracle.widen(oracle.store(M64["csr_val"], dt), dt))


# ---------------------------------------------------------------- checks, bounds

def test_csr_check_rejects_bad_input():
    A = synth.example_matrix()
    rp, col = A.row_ptr.copy(), A.col.copy()
    assert oracle.csr_check(8, rp, col) == 0
    bad = rp.copy(); bad[0] = 1
    assert oracle.csr_check(8, bad, col) == 1
    bad = rp.copy(); bad[3], bad[4] = bad[4], bad[3]
    assert oracle.csr_check(8, bad, col) == 2
    bad = col.copy(); bad[5] = 8
    assert oracle.csr_check(8, rp, bad) == 3
    bad = col.copy(); bad[5] = -1
    assert oracle.csr_check(8, rp, bad) == 3
    bad = col.copy(); bad[1] = 0          # duplicate column in row 0
    assert oracle.csr_check(8, rp, bad) == 4
    bad = col.copy(); bad[0], bad[1] = bad[1], bad[0]
    assert oracle.csr_check(8, rp, bad) == 4


def test_fp32_dot_products_stay_within_bound():
    # the Higham bound used as the FP32 tolerance holds for sequential FP32
    # sums of rounded operands, and a planted error of 4x the bound fails it
    rng = synth.Rng(3, 3)
    for k in (1, 7, 27, 300):
        a = rng.uniform(k, -1, 1) * 10.0 ** rng.uniform(k, -3, 3)
        x = rng.uniform(k, -1, 1)
        exact = float(np.sum(a * x, dtype=np.float64))
        s = np.float32(0)
        for ai, xi in zip(oracle.round_f32(a), oracle.round_f32(x)):
            s = np.float32(s + np.float32(ai) * np.float32(xi))
        absrow = float(np.sum(np.abs(a * x)))
        b = oracle.bound_vs_exact(absrow, k, "f32")
        assert abs(float(s) - exact) <= b
        assert not abs(float(s) + 4 * b - exact) <= b


def test_stream_kernels():
    n = 1000
    A = np.arange(n, dtype=float)
    B = np.full(n, 2.0)
    Cv = np.ones(n)
    assert oracle.stream_direct(A, B, Cv).tolist() == (1 + 2 * A).tolist()
    I = np.arange(n, dtype=np.int32)
    assert oracle.stream_indirect(A, B, I, Cv).tolist() == (1 + 2 * A).tolist()


def test_spmv_reads_no_x_outside_the_vector():
    # x sits inside a NaN-filled buffer: a read of x[i + off] outside [0, n)
    # (a missing clip of the diagonal loop, Fig. 13) turns the row into NaN.
    A = synth.config_matrix("stencil7_32", scale=0.5)
    pad = 5000
    buf = np.full(A.n + 2 * pad, np.nan)
    buf[pad:pad + A.n] = synth.uniform_vector(A.n, 4)
    x = buf[pad:pad + A.n]
    assert np.all(np.isfinite(oracle.csr_spmv(A, x)))
    for bl, theta in ((1024, 0.6), (100, 0.3), (4096, 0.6)):
        M = oracle.convert(A, bl, theta)
        assert np.all(np.isfinite(oracle.mhdc_spmv(M, x)))


# ---------------------------------------------------------------- selector network

def test_mlp_oracle_gradient_matches_finite_differences():
    from oracle import mlp
    F, H, O = 5, 7, 4
    rng = synth.Rng(21, 1)
    P = H * F + H + H * H + H + O * H + O
    p = rng.uniform(P, -0.6, 0.6)
    X = rng.uniform(6 * F, -1, 1).reshape(6, F)
    T = rng.uniform(6 * O, -1, 1).reshape(6, O)
    M = (rng.unit(6 * O) < 0.7).astype(float).reshape(6, O)
    g = mlp.gradient(p, F, H, O, X, T, M)
    fd = mlp.fd_gradient(p, F, H, O, X, T, M)
    for k, v in fd.items():
        assert abs(g[k] - v) <= 1e-6 * max(1.0, abs(v)), k


def test_mlp_oracle_closed_form_linear_case():
    # with ReLU units all active and a single output, the loss of a one-sample
    # batch is (w3 . relu(W2 relu(W1 x + b1) + b2) + b3 - t)^2
    from oracle import mlp
    F, H, O = 2, 2, 1
    W1 = np.array([[1.0, 0.0], [0.0, 2.0]]); b1 = np.array([0.5, 0.5])
    W2 = np.eye(2); b2 = np.zeros(2)
    W3 = np.array([[1.0, -1.0]]); b3 = np.array([0.25])
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    x = np.array([[1.0, 1.0]])
    Y, _ = mlp.forward(p, F, H, O, x)
    assert Y[0, 0] == 1.5 - 2.5 + 0.25
    assert mlp.loss(p, F, H, O, x, np.array([[0.0]]), np.ones((1, 1))) == (-0.75) ** 2
