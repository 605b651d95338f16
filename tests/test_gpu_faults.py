"""Allocation failures injected on the host, for every entry point that
allocates device memory.

For each call the test first counts the device allocations one clean call
makes (mhdc_debug_alloc_stats), then makes each of them fail in turn
(mhdc_debug_fail_alloc): the call must report MHDC_ERR_OOM and leave no
allocation of the library live once its objects are released, and a clean
call afterwards must still work.  The failure is made by the library's
allocation wrapper before it calls CUDA, so no GPU runs out of memory or
faults.
"""
import numpy as np
import pytest

import synth
from gpu_util import dev_csr, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    t = torch()
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2105_04937_gb300 as m
    m.lib()
    yield m
    m.mhdc_debug_fail_alloc(0)


def live(mh):
    torch().cuda.synchronize()
    return mh.mhdc_debug_alloc_stats()[1]


def release(obj):
    if obj is not None and hasattr(obj, "destroy"):
        obj.destroy()


def sweep(mh, call, prepare=None, tolerated=None):
    """Fail each device allocation of call(state) in turn.  prepare() makes a
    fresh state before every trial (with the hook disarmed); the state and
    the call's result are released after it (their destroy())."""
    base = live(mh)

    def trial(k):
        mh.mhdc_debug_fail_alloc(0)
        state = prepare() if prepare else None
        mh.mhdc_debug_fail_alloc(k)
        out, err = None, None
        try:
            out = call(state)
        except mh.MhdcError as e:
            err = e
        attempts, _ = mh.mhdc_debug_alloc_stats()
        mh.mhdc_debug_fail_alloc(0)
        release(out)
        release(state)
        return out, err, attempts

    out, err, attempts = trial(0)
    assert err is None, err
    assert live(mh) == base, "a clean call leaked"
    assert attempts >= 1, "the call made no device allocation"
    for k in range(1, attempts + 1):
        out, err, _ = trial(k)
        if err is not None:
            assert err.code == mh.MHDC_ERR_OOM, (k, err)
        else:
            assert tolerated is not None and tolerated(out), f"allocation {k} failed silently"
        assert live(mh) == base, f"allocation {k} of {attempts} failing leaked device memory"
    out, err, _ = trial(0)     # the library still works
    assert err is None, err
    assert live(mh) == base
    return attempts


@pytest.mark.parametrize("dt", ["f64", "bf16"])
def test_build_paths_release_everything_on_oom(mh, dt):
    # block selection (shared tables; the scattered rows also reach the
    # 16384-slot and the global-table levels), global selection, DIA input
    S = synth.config_matrix("stencil27_128", scale=0.1)
    W = synth.config_matrix("scattered_4m", scale=1 / 256)
    for A, n_b, fn in ((S, 1000, mh.mhdc_build), (W, 8192, mh.mhdc_build), (S, 512, mh.hdc_build)):
        rp, col, val = dev_csr(A)
        assert sweep(mh, lambda _: fn(A.n, rp, col, val, n_b, 0.6, dt)) >= 5
    t = torch()
    offs = t.tensor([-37, -1, 0, 1, 37], dtype=t.int32, device="cuda")
    dv = t.rand(5 * 20000, dtype=t.float64, device="cuda")
    sweep(mh, lambda _: mh.mhdc_build_dia(20000, offs, dv, 1024, 0.6, dt))


def test_buffers_made_on_first_use_release_on_oom(mh):
    t = torch()
    A = synth.config_matrix("stencil7_32", scale=0.5)
    rp, col, val = dev_csr(A)

    def fresh():
        return mh.mhdc_build(A.n, rp, col, val, 512, 0.6, "f64")

    x = t.rand(A.n, dtype=t.float64).pin_memory()
    y = t.empty(A.n, dtype=t.float64).pin_memory()

    # staging buffers of the host-buffer calls
    def host(h):
        mh.mhdc_spmv_host(h, x, y)

    sweep(mh, host, prepare=fresh)

    def pipelined(h):
        mh.mhdc_spmv_host_async(h, x, y)
        mh.mhdc_host_wait(h)

    sweep(mh, pipelined, prepare=fresh)
    # the FP32-pair arrays of the emulated FP64 variants
    sweep(mh, lambda h: mh.mhdc_set_variant(h, mh.FIRST_EMULATED_VARIANT), prepare=fresh)
    xd = t.rand(A.n, dtype=t.float64, device="cuda")
    yd = t.empty_like(xd)

    def tune(h):
        mh.mhdc_tune(h, xd, yd)

    sweep(mh, tune, prepare=fresh)


def test_batch_mlp_sell_and_selector_release_on_oom(mh):
    A = synth.config_matrix("stencil7_32", scale=0.5)
    rp, col, val = dev_csr(A)
    hs = [mh.mhdc_build(A.n, rp, col, val, 512, 0.6, "f64") for _ in range(3)]
    sweep(mh, lambda _: mh.mhdc_batch_create(hs))
    for h in hs:
        h.destroy()
    sweep(mh, lambda _: mh.mhdc_mlp_create(64, 32, 45, seed=1))
    sweep(mh, lambda _: mh.sell_build(A.n, rp, col, val, 32, 64))
    sweep(mh, lambda _: mh.mhdc_features(A.n, rp, col))
    sweep(mh, lambda _: mh.mhdc_select(A.n, rp, col, val, 1e-12, mh.MHDC_SELECT_MODEL))
    # the autotuner skips a candidate it cannot build (time -1) instead of failing
    sweep(mh, lambda _: mh.mhdc_autotune(A.n, rp, col, val, reps=1),
          tolerated=lambda times: bool(np.any(times < 0)))
