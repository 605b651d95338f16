// Device allocations of the library, in one place: every cudaMalloc,
// cudaFree and stream-ordered pool allocation of the library goes through
// these wrappers, which count the allocations made and still live, and can
// make the n-th allocation from a given point fail as if the device were out
// of memory.  The failure is injected on the host only (the CUDA call is not
// made), so the cleanup paths of every entry point can be tested without
// exhausting or faulting a GPU.  Armed by mhdc_debug_fail_alloc or, for a
// whole process, by the environment variable MHDC_FAULT_ALLOC=n read at the
// first allocation.
#include <atomic>
#include <cstdlib>

#include "mhdc_internal.cuh"

namespace mhdc {
namespace {

std::atomic<int64_t> g_fail_at{-1};   // -1: not yet read from the environment; 0: off
std::atomic<int64_t> g_attempts{0};   // allocation attempts since the last arming
std::atomic<int64_t> g_live{0};       // allocations made and not yet freed

// True if this allocation attempt must fail.
bool inject()
{
    int64_t f = g_fail_at.load();
    if (f < 0) {
        const char *e = std::getenv("MHDC_FAULT_ALLOC");
        const int64_t v = e ? std::atoll(e) : 0;
        int64_t expect = -1;
        g_fail_at.compare_exchange_strong(expect, v > 0 ? v : 0);
        f = g_fail_at.load();
    }
    const int64_t k = ++g_attempts;
    return f > 0 && k == f;
}

}  // namespace

cudaError_t dmalloc(void **p, size_t bytes)
{
    if (inject()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_live++;
    return e;
}

void dfree(void *p)
{
    if (!p) return;
    cudaFree(p);
    g_live--;
}

cudaError_t dmalloc_pool(void **p, size_t bytes, cudaMemPool_t pool, cudaStream_t st)
{
    if (inject()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, st);
    if (e == cudaSuccess) g_live++;
    return e;
}

void dfree_async(void *p, cudaStream_t st)
{
    if (!p) return;
    cudaFreeAsync(p, st);
    g_live--;
}

}  // namespace mhdc

extern "C" {

int mhdc_debug_fail_alloc(int64_t n)
{
    if (n < 0) {
        mhdc::set_error_msg("mhdc_debug_fail_alloc: n must be >= 0");
        return MHDC_ERR_INVALID_ARG;
    }
    mhdc::g_fail_at = n;
    mhdc::g_attempts = 0;
    return MHDC_OK;
}

int mhdc_debug_alloc_stats(int64_t *attempts, int64_t *live)
{
    if (attempts) *attempts = mhdc::g_attempts.load();
    if (live) *live = mhdc::g_live.load();
    return MHDC_OK;
}

}  // extern "C"
