"""CPU checks of the performance models (Sec. 5) against what the paper and
plain byte counting fix: the bounds the paper derives, their limits, and the
volumes recounted from the arrays of a real stencil matrix."""
import numpy as np

import synth
from paper_2105_04937_gb300 import model as pm


def test_stencil_bounds_of_sec_5_2():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        nd = int(rng.integers(1, 64))
        gamma = rng.uniform(1 / nd, 1)
        b = rng.uniform(0.05, 1.0)
        s = pm.stencil_speedups(nd, gamma, b)
        # B-DIA over CSR between 1 + b/2 and 1 + b (Sec. 5.2.5)
        assert 1 + b / 2 < s["bdia_over_csr"] < 1 + b
        # DIA never beats CSR when b <= 1 (Sec. 5.2.4), and is below (3 + 2b) / 5
        assert s["dia_over_csr"] <= 1 + 1e-12
        assert s["dia_over_csr"] <= (3 + 2 * b) / 5 + 1e-12
        # B-DIA over DIA: 1 + 2/3 <= ratio < 1 + 3 (Sec. 5.2.6)
        assert 1 + 2 / 3 - 1e-12 <= s["bdia_over_dia"] < 4


def test_paper_stencil_cases():
    # 1D 3-point, gamma = 1/3; 2D 5-point, 1/5; 3D 7-point, 3/7 (Sec. 6.3), FP64 + INT32
    got = [pm.stencil_speedups(nd, g)["bdia_over_csr"] for nd, g in ((3, 1 / 3), (5, 1 / 5), (7, 3 / 7))]
    assert np.allclose(got, [1.4, 1 + 3 / 7, 1 + 4 / 11])
    # val 3 + col_ind 1.5 + row_ptr 0.5 + x 1 + y 1 over val 3 + x 3 + y 7
    assert np.isclose(pm.stencil_speedups(3, 1 / 3)["dia_over_csr"], 7 / 13)


def test_hdc_model_limits_and_bound():
    b = pm.B_FP64_INT32
    # alpha = 1, beta = 0, v_x = 1 and c -> infinity: the bound 1 + b (Sec. 5.3.2)
    assert abs(pm.rp_est(1.0, 0.0, 1e9) - (1 + b)) < 1e-8
    rng = np.random.default_rng(2)
    for _ in range(2000):
        a, be, c = rng.uniform(0.01, 1), rng.uniform(0, 1), rng.uniform(1, 500)
        vx = rng.uniform(1, 5)
        assert pm.rp_est(a, be, c, b, vx) < 1 + b
    # everything in CSR (beta = 1): HDC reads what CSR reads
    assert abs(pm.rp_est(0.7, 1.0, 27.0) - 1.0) < 1e-12
    # the gain needs alpha >= 1 / (b + 1) when beta < 1 (Sec. 5.3.2)
    assert pm.rp_est(1 / (1 + b) + 1e-6, 0.3, 20.0) > 1.0 > pm.rp_est(1 / (1 + b) - 1e-3, 0.3, 20.0)


def test_volumes_match_counted_bytes():
    """The model's volumes times b_fp n equal the bytes of the actual arrays
    (values 8 B, indices 4 B) of a 3D 7-point stencil, up to the nnz = nd n
    approximation of Sec. 5.2, which the clipped edges make inexact."""
    A = synth.paper_stencil(30000, 3)
    n, nnz, nd = A.n, A.nnz, 7
    csr_a = 8 * nnz + 4 * nnz + 4 * n          # val, col_ind, row_ptr
    assert abs(pm.volume_csr(nnz / n, 0.5, 1.0) * 8 * n - (csr_a + 8 * n + 8 * n)) < 1e-6 * csr_a
    model_a = (pm.volume_csr_stencil(nd, 0.0) - 1) * 8 * n
    assert abs(model_a - csr_a) / csr_a < 1e-2
    # B-HDC with every nonzero in a full DIA part equals B-DIA plus the CSR row_ptr
    for g in (1 / 7, 3 / 7, 1.0):
        v_hdc = pm.volume_hdc(1.0, 0.0, nd, 0.5, v_x=g * nd)
        assert abs(v_hdc - (pm.volume_bdia_stencil(nd, g) + 0.5)) < 1e-12
    assert pm.relative_error(0.9, 1.0) < 0 < pm.relative_error(1.1, 1.0)
