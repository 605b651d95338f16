"""The allocation-free conversion (mhdc_build_noalloc) against mhdc_build.

Some callers cannot allocate device memory while they convert a matrix: a
process that takes all its device memory from one pool at start-up, code on a
latency-critical path where an allocation would stall or fail, or a binding
that may only hand over buffers it already owns.  They call
mhdc_build_noalloc with output arrays of their own; its temporaries live in a
fixed device array inside the library.  Its results must equal what
mhdc_build + mhdc_export give for the same input, bit for bit (the tolerance
every conversion test here uses).  Three calls in a row, on different matrices
and dtypes (the last two through the conversion's global-table path), check
that what one call leaves in the shared device array does not leak into the
next.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth
from gpu_util import bits, dev_csr, torch

pytestmark = pytest.mark.gpu

LIMIT = 262144


@pytest.fixture(scope="module")
def mh():
    t = torch()
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2105_04937_gb300 as m
    m.lib()
    return m


def convert_both(mh, A, n_b, theta, dtype):
    t = torch()
    rp, col, val = dev_csr(A)
    ref = mh.mhdc_build(A.n, rp, col, val, n_b, theta, dtype)
    E = mh.mhdc_export(ref)
    P, R = ref.info["P"], ref.info["nnz_rem"]
    ref.destroy()
    nb = (A.n + n_b - 1) // n_b
    vt = {"f64": t.float64, "f32": t.float32, "bf16": t.int16}[dtype]
    # the caller's own output arrays, filled with garbage first
    out = dict(
        dia_ptr=t.full((nb + 1,), -7, dtype=t.int32, device="cuda"),
        dia_offset=t.full((max(1, P),), -7, dtype=t.int32, device="cuda"),
        dia_val=t.full((max(1, P * n_b),), 3, dtype=vt, device="cuda"),
        csr_row_ptr=t.full((A.n + 1,), -7, dtype=t.int32, device="cuda"),
        csr_col=t.full((max(1, A.nnz),), -7, dtype=t.int32, device="cuda"),
        csr_val=t.full((max(1, A.nnz),), 3, dtype=vt, device="cuda"),
    )
    got_P, got_R = mh.mhdc_build_noalloc(A.n, rp, col, val, n_b, theta, dtype, out["dia_ptr"],
                                         out["dia_offset"], out["dia_val"], out["csr_row_ptr"],
                                         out["csr_col"], out["csr_val"])
    assert (got_P, got_R) == (P, R)
    G = {k: v.cpu().numpy() for k, v in out.items()}
    G["dia_offset"] = G["dia_offset"][:P]
    G["dia_val"] = G["dia_val"][:P * n_b]
    G["csr_col"] = G["csr_col"][:R]
    G["csr_val"] = G["csr_val"][:R]
    for k in ("dia_ptr", "dia_offset", "csr_row_ptr", "csr_col"):
        assert np.array_equal(G[k], E[k]), k
    for k in ("dia_val", "csr_val"):
        assert G[k].size == E[k].size, k
        assert np.array_equal(bits(G[k]), bits(E[k])), k
    return P, R


def distinct_offsets_per_block(A, n_b):
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    off = A.col.astype(np.int64) - rows
    blk = rows // n_b
    return [np.unique(off[blk == b]).size for b in range((A.n + n_b - 1) // n_b)]


# a row block with more distinct offsets than this overflows the largest
# shared-memory table and is counted in a table inside the device array
SHARED_TABLE_LIMIT = 12288


def test_noalloc_matches_mhdc_build_on_calls_in_a_row(mh):
    # call 1: 7-point stencil on 32^3 (223,232 entries), FP64
    A = synth.config_matrix("stencil7_32")
    P1, R1 = convert_both(mh, A, 1024, 0.6, "f64")
    assert P1 == 222 and R1 == 0
    # call 2: scattered diagonals (232,355 entries, rows with random entries;
    # both 8192-row blocks take the global-table path), BF16
    B = synth.config_matrix("scattered_4m", scale=1 / 256)
    assert min(distinct_offsets_per_block(B, 8192)) > SHARED_TABLE_LIMIT
    P2, R2 = convert_both(mh, B, 8192, 0.6, "bf16")
    assert P2 > 0 and R2 > 0
    # call 3: another scattered matrix (14,980 rows, a ragged last block) whose
    # first block also takes the global-table path, FP32: the tables,
    # overflow list and remainder flags that call 2 left behind must not leak
    C_ = synth.config_matrix("scattered_4m", scale=1 / 280)
    assert C_.n == 14980 and C_.nnz <= LIMIT
    assert distinct_offsets_per_block(C_, 8192)[0] > SHARED_TABLE_LIMIT
    P3, R3 = convert_both(mh, C_, 8192, 0.6, "f32")
    assert P3 > 0 and R3 > 0 and (P3, R3) != (P2, R2)


def test_noalloc_rejects_sizes_beyond_its_limit(mh):
    t = torch()
    A = synth.config_matrix("stencil27_128", scale=0.25)     # 32^3 rows, ~0.75M entries
    assert A.n <= LIMIT < A.nnz
    rp, col, val = dev_csr(A)
    nb = (A.n + 4095) // 4096
    z32 = t.zeros(nb + 1, dtype=t.int32, device="cuda")
    zrow = t.zeros(A.n + 1, dtype=t.int32, device="cuda")
    small32 = t.zeros(16, dtype=t.int32, device="cuda")
    small64 = t.zeros(16 * 4096, dtype=t.float64, device="cuda")
    with pytest.raises(mh.MhdcError, match="no-allocation limit") as e:
        mh.mhdc_build_noalloc(A.n, rp, col, val, 4096, 0.6, "f64", z32, small32, small64, zrow,
                              small32, small64[:16])
    assert e.value.code == -1
