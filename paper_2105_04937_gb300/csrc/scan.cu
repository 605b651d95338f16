// Device-wide exclusive prefix sum of int32 values (reduce, scan the tile
// sums, scan the tiles).  No inter-CTA waits: three launches per level.
#include "mhdc_internal.cuh"

namespace mhdc {
namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Exclusive scan of one value per thread across the CTA; returns the CTA total.
__device__ int32_t cta_exclusive_scan(int32_t v, int32_t &excl)
{
    constexpr int NW = SCAN_THREADS / 32;
    __shared__ int32_t warp_base[NW + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) warp_base[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int32_t w = lane < NW ? warp_base[lane] : 0;
        int32_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int32_t t = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += t;
        }
        if (lane < NW) warp_base[lane] = wi - w;
        if (lane == NW - 1) warp_base[NW] = wi;
    }
    __syncthreads();
    excl = warp_base[wid] + incl - v;
    const int32_t total = warp_base[NW];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(SCAN_THREADS)
k_tile_sums(const int32_t *__restrict__ in, int64_t m, int32_t *__restrict__ sums)
{
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int32_t s = 0;
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; it++) {
        int64_t k = base + (int64_t)it * SCAN_THREADS + threadIdx.x;
        if (k < m) s += in[k];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    __shared__ int32_t ws[SCAN_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; w++) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// Scan one tile; add `bases[blockIdx.x]` (or 0); write out[0..len) and, for
// the last tile, out[m] = total.
__global__ void __launch_bounds__(SCAN_THREADS)
k_tile_scan(const int32_t *__restrict__ in, int64_t m, const int32_t *__restrict__ bases,
            int32_t *__restrict__ out)
{
    __shared__ int32_t tile[SCAN_TILE];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int it = 0; it < SCAN_ITEMS; it++) {
        int idx = it * SCAN_THREADS + threadIdx.x;
        int64_t k = base + idx;
        tile[idx] = k < m ? in[k] : 0;
    }
    __syncthreads();
    int32_t loc[SCAN_ITEMS];
    int32_t tsum = 0;
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; it++) {
        loc[it] = tsum;
        tsum += tile[threadIdx.x * SCAN_ITEMS + it];
    }
    int32_t excl;
    int32_t total = cta_exclusive_scan(tsum, excl);
    const int32_t b = bases ? bases[blockIdx.x] : 0;
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; it++) tile[threadIdx.x * SCAN_ITEMS + it] = b + excl + loc[it];
    __syncthreads();
    for (int it = 0; it < SCAN_ITEMS; it++) {
        int idx = it * SCAN_THREADS + threadIdx.x;
        int64_t k = base + idx;
        if (k < m) out[k] = tile[idx];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[m] = b + total;
}

}  // namespace

int64_t scan_scratch_elems(int64_t m)
{
    if (m <= SCAN_TILE) return 0;
    int64_t nt = (m + SCAN_TILE - 1) / SCAN_TILE;
    return nt + (nt + 1) + scan_scratch_elems(nt);
}

int exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t m, int32_t *scratch,
                       cudaStream_t stream)
{
    if (m <= 0) {
        MHDC_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int32_t), stream));
        return MHDC_OK;
    }
    if (m <= SCAN_TILE) {
        k_tile_scan<<<1, SCAN_THREADS, 0, stream>>>(in, m, nullptr, out);
        MHDC_LAUNCH_CHECK("k_tile_scan");
        return MHDC_OK;
    }
    int64_t nt = (m + SCAN_TILE - 1) / SCAN_TILE;
    int32_t *sums = scratch;
    int32_t *bases = scratch + nt;
    k_tile_sums<<<(unsigned)nt, SCAN_THREADS, 0, stream>>>(in, m, sums);
    MHDC_LAUNCH_CHECK("k_tile_sums");
    int rc = exclusive_scan_i32(sums, bases, nt, scratch + nt + (nt + 1), stream);
    if (rc != MHDC_OK) return rc;
    k_tile_scan<<<(unsigned)nt, SCAN_THREADS, 0, stream>>>(in, m, bases, out);
    MHDC_LAUNCH_CHECK("k_tile_scan");
    return MHDC_OK;
}

}  // namespace mhdc
