// CSR -> M-HDC / blocked HDC conversion on the device (Sec. 3.4, 4.3; Fig. 12).
//
// Steps (one stream; the host only reads sizes back to allocate):
//   1. k_validate       CSR checks (row_ptr bounds, columns in range, strictly
//                       increasing inside a row).
//   2. k_count_select   M-HDC: one CTA per row block counts N(d, ib) for every
//                       offset d = j - i in a hash table (shared memory; a
//                       block with too many distinct offsets is redone with a
//                       table in global memory), keeps d iff N >= 1 and
//                       N >= theta * rows(ib), and sorts the kept offsets.
//      k_count_all      HDC: N(d) over the whole matrix in a dense array, kept
//                       iff N >= 1 and N >= theta * n, compacted in order.
//      Both walk 32 rows per warp with one lane per row, so lanes holding the
//      same offset (rows of one stencil pattern) add their count with one
//      atomic (warp match) instead of one each.
//   3. scan             dia_ptr = exclusive prefix sum of the kept counts.
//   4. k_scatter        dia_val assembled per (block, 256-row chunk) in a
//                       shared-memory tile and written once, coalesced; the
//                       entries left out are counted per row.
//   5. scan + k_rem_fill csr_row_ptr = exclusive prefix sum of those counts;
//                       the rows holding remainder entries copy them in input
//                       order.
// Temporaries are stream-ordered allocations from a pool of the library.
#include <climits>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "mhdc_internal.cuh"

namespace mhdc {
namespace {

constexpr int32_t EMPTY_KEY = INT32_MIN;  // no offset d = j - i equals it (|d| < 2^31 - 1)
constexpr int HCAP = 16384;               // shared-memory hash slots
constexpr int HLIMIT = 12288;             // distinct offsets a shared table accepts
constexpr int CS_THREADS = 512;
constexpr int CS_WARPS = CS_THREADS / 32;

// 32-bit finaliser of MurmurHash3 (Appleby): spreads offsets that differ only
// in high bits (stencil offsets like -16384, 0, 16384) over the table.
__device__ __forceinline__ uint32_t mix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__global__ void k_validate(int64_t n, const int32_t *__restrict__ rp,
                           const int32_t *__restrict__ col, int32_t nnz, int *err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t a = rp[i], b = rp[i + 1];
    if (i == 0 && a != 0) atomicOr(err, 1);
    if (a < 0 || b < a || b > nnz) {
        atomicOr(err, 2);
        return;
    }
    int64_t prev = -1;
    for (int32_t k = a; k < b; k++) {
        const int32_t c = col[k];
        if (c < 0 || (int64_t)c >= n) {
            atomicOr(err, 4);
            return;
        }
        if ((int64_t)c <= prev) {
            atomicOr(err, 8);
            return;
        }
        prev = c;
    }
}

// Add c occurrences of `off`.  With limit > 0 a new key first reserves room
// (used < limit < capacity, so an empty slot always exists); the probe loop
// is bounded by the capacity in any case.  Returns false on overflow.
__device__ __forceinline__ bool table_insert(volatile int32_t *keys, int32_t *cnt, uint32_t mask,
                                             int32_t off, int32_t c, int *used, int limit)
{
    uint32_t h = mix32((uint32_t)off) & mask;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const int32_t k = keys[h];
        if (k == off) {
            atomicAdd(&cnt[h], c);
            return true;
        }
        if (k == EMPTY_KEY) {
            if (limit > 0 && atomicAdd(used, 1) >= limit) return false;
            const int32_t prev = atomicCAS((int32_t *)&keys[h], EMPTY_KEY, off);
            if (prev == EMPTY_KEY) {
                atomicAdd(&cnt[h], c);
                return true;
            }
            if (limit > 0) atomicSub(used, 1);
            if (prev == off) {
                atomicAdd(&cnt[h], c);
                return true;
            }
        }
        h = (h + 1) & mask;
    }
    return false;
}

// Offset counting over 32 consecutive rows [g0, min(g0 + 32, end)), one lane
// per row.  A first walk (entry k of every row at step k) compares each row's
// offsets d = j - i with those of the row before it (the lane before): rows
// with the same length and offsets form a run, and only the first row of a
// run adds its offsets, each with the run's length as count.  Rows of one
// stencil pattern thus cost one addition per offset per run instead of one
// per entry; the counts are exact (no hashing).  The first walk is
// warp-uniform; the second runs on the run-start lanes only.  add(off, c)
// adds c to offset off's count and returns false when the table is full.
// SHARED: the columns come from a shared-memory copy holding entries
// [base, ...) instead of global memory.
template <bool SHARED = false, typename F>
__device__ __forceinline__ void runs_by_lane(int64_t g0, int64_t end, const int32_t *__restrict__ rp,
                                             const int32_t *__restrict__ col, int32_t base, F add)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = g0 + lane;
    const bool live = i < end;
    const int32_t a = live ? rp[i] : 0;
    const int32_t len = live ? rp[i + 1] - a : 0;
    const int32_t maxlen = __reduce_max_sync(0xffffffffu, len);
    auto off_at = [&](int32_t k) -> int32_t {
        if (k >= len) return EMPTY_KEY;
        const int32_t c = SHARED ? col[a + k - base] : __ldg(col + a + k);
        return c - (int32_t)i;
    };
    // every lane takes part in each shuffle (no short-circuit around them)
    const int32_t prev_len = __shfl_up_sync(0xffffffffu, len, 1);
    bool same = lane > 0 && prev_len == len;
    for (int32_t k = 0; k < maxlen; k++) {
        const int32_t off = off_at(k);
        const int32_t prev_off = __shfl_up_sync(0xffffffffu, off, 1);
        same = same && prev_off == off;
    }
    const unsigned live_mask = __ballot_sync(0xffffffffu, live);
    const bool start = live && !same;
    const unsigned starts = __ballot_sync(0xffffffffu, start);
    if (!start) return;
    const unsigned later = starts & ~((2u << lane) - 1u);  // run starts after this lane
    const int32_t next = later ? __ffs(later) - 1 : __popc(live_mask);
    const int32_t run = next - lane;
    for (int32_t k = 0; k < len; k++)
        if (!add(off_at(k), run)) return;
}

// Ascending bitonic sort of a[0..P2) (P2 a power of two) by the whole CTA.
__device__ void cta_bitonic_sort(int32_t *a, int64_t P2)
{
    for (int64_t k = 2; k <= P2; k <<= 1) {
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            for (int64_t i = threadIdx.x; i < P2; i += blockDim.x) {
                const int64_t l = i ^ j;
                if (l > i) {
                    const int32_t x = a[i], y = a[l];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// M-HDC selection for one row block per CTA (block ids[blockIdx.x] when ids
// is given, else blockIdx.x), in three table levels:
//   level 1: <false, true>  shared table of at most SMALL_CAP slots, and each
//            warp stages its 32 rows' columns (up to cw) in shared memory
//            (coalesced loads) before walking them one lane per row;
//   level 2: <false, true>  shared table of at most HCAP slots, smaller
//            staging, for the blocks level 1 could not hold;
//   level 3: <true, false>  a table of 2^tab_log2[c] slots at tab_base[c] in
//            global memory (at least twice the block's entries: cannot fill).
// A shared table accepting no more distinct offsets sets overflow[ib] and the
// CTA stops; the host then runs the next level for those blocks.
constexpr int SMALL_CAP = 2048;
constexpr int CW = 1024;    // staged columns per warp at level 1
constexpr int CW_L2 = 512;  // and at level 2 (with the largest table)
constexpr size_t CS_SMEM_SMALL = (3 * SMALL_CAP + CS_WARPS * CW) * sizeof(int32_t);
constexpr size_t CS_SMEM_L2 = (3 * HCAP + CS_WARPS * CW_L2) * sizeof(int32_t);

template <bool GLOBAL_TABLE, bool STAGE>
__global__ void __launch_bounds__(CS_THREADS)
k_count_select(int64_t n, int32_t n_b, const int32_t *__restrict__ rp,
               const int32_t *__restrict__ col, double theta, const int32_t *__restrict__ ids,
               int32_t cap_max, int32_t cw, int32_t *gkeys, int32_t *gcnt,
               const int64_t *__restrict__ tab_base, const int32_t *__restrict__ tab_log2,
               int32_t *sel_out, int32_t *sel_cnt, int32_t *overflow)
{
    extern __shared__ int32_t smem[];
    __shared__ int used, nsel;
    __shared__ volatile int ovf;
    const int64_t ib = ids ? (int64_t)ids[blockIdx.x] : (int64_t)blockIdx.x;
    const int64_t r0 = ib * (int64_t)n_b;
    const int64_t rows = (n - r0 < n_b) ? (n - r0) : n_b;
    int32_t *keys, *cnt;
    int64_t cap;
    int limit;
    if (GLOBAL_TABLE) {
        keys = gkeys + tab_base[blockIdx.x];
        cnt = gcnt + tab_base[blockIdx.x];
        cap = (int64_t)1 << tab_log2[blockIdx.x];
        limit = 0;
    } else {
        // distinct offsets <= entries m of the block: a table of 2m slots
        // (at least 64, at most cap_max) never fills unless m is large
        const int64_t m = (int64_t)rp[r0 + rows] - rp[r0];
        cap = 64;
        while (cap < 2 * m && cap < cap_max) cap <<= 1;
        keys = smem;
        cnt = smem + cap_max;
        limit = cap == cap_max ? cap_max / 4 * 3 : (int)cap - 1;
    }
    const uint32_t mask = (uint32_t)(cap - 1);
    for (int64_t s = threadIdx.x; s < cap; s += blockDim.x) {
        keys[s] = EMPTY_KEY;
        cnt[s] = 0;
    }
    if (threadIdx.x == 0) {
        used = 0;
        nsel = 0;
        ovf = 0;
    }
    __syncthreads();

    // lanes holding the same offset in a step add their count once (leader lane)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *stage = smem + 3 * cap_max + warp * cw;
    for (int64_t g0 = r0 + 32 * warp; g0 < r0 + rows; g0 += 32 * CS_WARPS) {
        if (__any_sync(0xffffffffu, ovf != 0)) break;  // warp-uniform exit
        auto count = [&](int32_t off, int32_t c) {
            if (table_insert(keys, cnt, mask, off, c, &used, limit)) return true;
            ovf = 1;
            return false;
        };
        const int64_t g1 = (g0 + 32 < r0 + rows) ? g0 + 32 : r0 + rows;
        const int32_t e0 = rp[g0], e1 = rp[g1];
        if (STAGE && e1 - e0 <= cw) {
            for (int32_t e = e0 + lane; e < e1; e += 32) stage[e - e0] = __ldg(col + e);
            __syncwarp();
            runs_by_lane<true>(g0, g1, rp, stage, e0, count);
            __syncwarp();
        } else {
            runs_by_lane(g0, g1, rp, col, 0, count);
        }
    }
    __syncthreads();
    if (ovf) {        if (threadIdx.x == 0) {
            overflow[ib] = 1;
            sel_cnt[ib] = 0;
        }
        return;
    }

    // keep d iff N(d, ib) >= 1 and N >= theta * rows(ib)
    const double thr = theta * (double)rows;
    int32_t *sel = GLOBAL_TABLE ? (sel_out + rp[r0]) : (smem + 2 * cap_max);
    for (int64_t s = threadIdx.x; s < cap; s += blockDim.x) {
        const int32_t k = ((volatile int32_t *)keys)[s];
        if (k != EMPTY_KEY) {
            const int32_t c = ((volatile int32_t *)cnt)[s];
            if (c >= 1 && (double)c >= thr) sel[atomicAdd(&nsel, 1)] = k;
        }
    }
    __syncthreads();
    const int64_t S = nsel;
    int64_t P2 = 1;
    while (P2 < S) P2 <<= 1;
    int32_t *buf = GLOBAL_TABLE ? keys : sel;  // the table is no longer needed
    if (GLOBAL_TABLE) {
        for (int64_t s = threadIdx.x; s < S; s += blockDim.x) buf[s] = sel[s];
    }
    for (int64_t s = S + threadIdx.x; s < P2; s += blockDim.x) buf[s] = INT32_MAX;
    __syncthreads();
    cta_bitonic_sort(buf, P2);
    int32_t *dst = sel_out + rp[r0];
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) dst[s] = buf[s];
    if (threadIdx.x == 0) {
        sel_cnt[ib] = (int32_t)S;
        overflow[ib] = 0;
    }
}

// Selector features: for one block size, histogram the partial diagonals by
// filling rate f = N(d, ib) / rows(ib) in 10 bins ([0, 0.1), ..., [0.9, 1]):
// ent[bin] += N (stored entries) and dia[bin] += 1.  A block whose distinct
// offsets overflow the shared table counts the entries it could not insert
// as single-entry diagonals (bin 0): such offsets are almost all singletons.
__global__ void __launch_bounds__(CS_THREADS)
k_count_hist(int64_t n, int32_t n_b, const int32_t *__restrict__ rp,
             const int32_t *__restrict__ col, unsigned long long *ent, unsigned long long *dia)
{
    extern __shared__ int32_t smem[];
    __shared__ int used;
    __shared__ unsigned long long lost;
    __shared__ unsigned long long h_ent[10], h_dia[10];
    const int64_t ib = blockIdx.x;
    const int64_t r0 = ib * (int64_t)n_b;
    const int64_t rows = (n - r0 < n_b) ? (n - r0) : n_b;
    const int64_t m = (int64_t)rp[r0 + rows] - rp[r0];
    int64_t cap = 64;
    while (cap < 2 * m && cap < HCAP) cap <<= 1;
    const int limit = cap == HCAP ? HLIMIT : (int)cap - 1;
    int32_t *keys = smem, *cnt = smem + HCAP;
    const uint32_t mask = (uint32_t)(cap - 1);
    for (int64_t s = threadIdx.x; s < cap; s += blockDim.x) {
        keys[s] = EMPTY_KEY;
        cnt[s] = 0;
    }
    if (threadIdx.x < 10) h_ent[threadIdx.x] = h_dia[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        used = 0;
        lost = 0;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    for (int64_t g0 = r0 + 32 * warp; g0 < r0 + rows; g0 += 32 * CS_WARPS) {
        runs_by_lane(g0, r0 + rows, rp, col, 0, [&](int32_t off, int32_t c) {
            if (!table_insert(keys, cnt, mask, off, c, &used, limit))
                atomicAdd(&lost, (unsigned long long)c);
            return true;  // keep going: the rest counts as single-entry diagonals
        });
    }
    __syncthreads();
    for (int64_t s = threadIdx.x; s < cap; s += blockDim.x) {
        if (((volatile int32_t *)keys)[s] == EMPTY_KEY) continue;
        const int32_t c = ((volatile int32_t *)cnt)[s];
        int bin = (int)(10.0 * (double)c / (double)rows);
        bin = bin > 9 ? 9 : bin;
        atomicAdd(&h_ent[bin], (unsigned long long)c);
        atomicAdd(&h_dia[bin], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        unsigned long long e = h_ent[threadIdx.x], d = h_dia[threadIdx.x];
        if (threadIdx.x == 0) {
            e += lost;
            d += lost;
        }
        if (e) atomicAdd(&ent[threadIdx.x], e);
        if (d) atomicAdd(&dia[threadIdx.x], d);
    }
}

// HDC: N(d) for d in [-(n-1), n-1] at cnt[d + n - 1].
// Each warp stages its 32 rows' columns in shared memory (CW per warp) when
// they fit, as level 1 of k_count_select does.
constexpr int CA_THREADS = 256;
constexpr size_t CA_SMEM = (CA_THREADS / 32) * CW * sizeof(int32_t);

__global__ void __launch_bounds__(CA_THREADS)
k_count_all(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t *cnt)
{
    extern __shared__ int32_t ca_smem[];
    const int lane = threadIdx.x & 31;
    int32_t *stage = ca_smem + (threadIdx.x >> 5) * CW;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    auto count = [&](int32_t off, int32_t c) {
        atomicAdd(&cnt[(int64_t)off + n - 1], c);
        return true;
    };
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); 32 * g < n;
         g += nw) {
        const int64_t g0 = 32 * g, g1 = (g0 + 32 < n) ? g0 + 32 : n;
        const int32_t e0 = rp[g0], e1 = rp[g1];
        if (e1 - e0 <= CW) {
            for (int32_t e = e0 + lane; e < e1; e += 32) stage[e - e0] = __ldg(col + e);
            __syncwarp();
            runs_by_lane<true>(g0, g1, rp, stage, e0, count);
            __syncwarp();
        } else {
            runs_by_lane(g0, g1, rp, col, 0, count);
        }
    }
}

__global__ void k_flag_global(int64_t m, const int32_t *__restrict__ cnt, double thr,
                              int32_t *flags)
{
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= m) return;
    const int32_t c = cnt[d];
    flags[d] = (c >= 1 && (double)c >= thr) ? 1 : 0;
}

__global__ void k_compact_global(int64_t m, int64_t n, const int32_t *__restrict__ flags,
                                 const int32_t *__restrict__ pos, int32_t *sel)
{
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= m) return;
    if (flags[d]) sel[pos[d]] = (int32_t)(d - (n - 1));
}

__global__ void k_uniform_ptr(int64_t n_blocks, int32_t S, int32_t *dia_ptr)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b <= n_blocks) dia_ptr[b] = (int32_t)(b * S);
}

template <typename VT>
__device__ __forceinline__ VT round_store(double v);
template <>
__device__ __forceinline__ double round_store<double>(double v) { return v; }
template <>
__device__ __forceinline__ float round_store<float>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 round_store<__nv_bfloat16>(double v)
{
    return __float2bfloat16_rn(__double2float_rn(v));
}

// Position of d in the ascending list s[0..m), or -1.
__device__ __forceinline__ int64_t find_sorted(const int32_t *__restrict__ s, int64_t m, int32_t d)
{
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (s[mid] < d) lo = mid + 1;
        else hi = mid;
    }
    return (lo < m && s[lo] == d) ? lo : -1;
}

// Scatter (Fig. 12 layout).  CTA c of row block ib handles the block's rows
// [c * SC_ROWS, (c + 1) * SC_ROWS), in sub-chunks of RC rows whose dia_val
// slots fit a shared-memory tile (S diagonals x RC rows, row stride RC + 1
// against bank conflicts).  Threads take the sub-chunk's entries in order
// (coalesced loads of col and val), find each entry's row by binary search
// in the staged row pointers and its diagonal by binary search in the
// block's sorted offsets, and either place the value in the tile or count
// the entry in its row's remainder count and set its bit in rem_flag.  The tile, zero-filled first, is
// written out one contiguous run per diagonal, so each dia_val element is
// written once.  When even 32 rows of S diagonals exceed the tile, the CTA
// zero-fills its slots in global memory and writes the entries in place.  The
// CTA of the block's last rows also zero-fills the slots past the matrix end,
// and CTA 0 writes the block's dia_offset.
constexpr int SC_THREADS = 256;
constexpr int SC_ROWS = 256;
constexpr int SC_SEL_MAX = 2048;                 // offsets staged in shared memory
constexpr int SC_TILE_BYTES = 48 * 1024;
constexpr int SC_RID_MAX = 8192;                 // entries whose row index is tabulated
constexpr int SC_UNROLL = 4;                     // entries in flight per thread
// offsets | row pointers | remainder counts | row index per entry (uint8),
// then the tile at a 16-byte boundary
constexpr size_t SC_HDR_BYTES =
    ((SC_SEL_MAX + (SC_ROWS + 1) + SC_ROWS) * sizeof(int32_t) + SC_RID_MAX + 15) / 16 * 16;
constexpr size_t SC_SMEM = SC_HDR_BYTES + SC_TILE_BYTES;

// Largest r in [0, m) with a[r] <= e (a ascending, a[0] <= e).
__device__ __forceinline__ int32_t row_of(const int32_t *a, int32_t m, int32_t e)
{
    int32_t lo = 0, hi = m - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (a[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename VT>
__global__ void __launch_bounds__(SC_THREADS)
k_scatter(int64_t n, int32_t n_b, int32_t cpb, const int32_t *__restrict__ rp,
          const int32_t *__restrict__ col, const double *__restrict__ val,
          const int32_t *__restrict__ dia_ptr, const int32_t *__restrict__ sel_list,
          const int32_t *__restrict__ sel_base_rp, int32_t *__restrict__ dia_offset,
          VT *__restrict__ dia_val, int32_t *__restrict__ rem_cnt, uint32_t *__restrict__ rem_flag)
{
    extern __shared__ __align__(16) unsigned char sc_smem[];
    int32_t *sel_s = reinterpret_cast<int32_t *>(sc_smem);
    int32_t *rp_s = sel_s + SC_SEL_MAX;            // SC_ROWS + 1 row pointers
    int32_t *rem_s = rp_s + SC_ROWS + 1;           // SC_ROWS counts
    uint8_t *rid_s = reinterpret_cast<uint8_t *>(rem_s + SC_ROWS);  // row of each entry
    VT *tile = reinterpret_cast<VT *>(sc_smem + SC_HDR_BYTES);
    const int64_t ib = blockIdx.x / cpb;
    const int64_t c = blockIdx.x - ib * cpb;
    const int64_t r0 = ib * (int64_t)n_b;
    const int64_t rows = (n - r0 < n_b) ? (n - r0) : n_b;
    const int64_t t0 = c * SC_ROWS;
    if (t0 >= rows) return;  // CTA-uniform
    const int64_t tn = (rows - t0 < SC_ROWS) ? (rows - t0) : SC_ROWS;
    const int64_t p0 = dia_ptr[ib];
    const int64_t S = dia_ptr[ib + 1] - p0;
    // M-HDC: the block's sorted list sits at sel_list + row_ptr[r0]; HDC: one shared list
    const int32_t *selg = sel_list + (sel_base_rp ? (int64_t)sel_base_rp[r0] : 0);
    if (c == 0)
        for (int64_t q = threadIdx.x; q < S; q += SC_THREADS) dia_offset[p0 + q] = selg[q];
    const bool sel_shared = S <= SC_SEL_MAX;
    if (sel_shared)
        for (int64_t q = threadIdx.x; q < S; q += SC_THREADS) sel_s[q] = selg[q];
    const int32_t *sel = sel_shared ? sel_s : selg;
    VT *dv = dia_val + p0 * (int64_t)n_b;
    const VT zero = round_store<VT>(0.0);
    // padding slots past the end of the matrix (last block only)
    if (t0 + tn == rows && rows < n_b) {
        const int64_t pad = n_b - rows;
        for (int64_t q = threadIdx.x; q < S * pad; q += SC_THREADS) {
            const int64_t p = q / pad;
            dv[p * n_b + rows + (q - p * pad)] = zero;
        }
    }
    // rows per sub-chunk: a multiple of 32 with S * (RC + 1) values in the tile
    int64_t RC = SC_ROWS;
    if (S > 0) {
        RC = ((int64_t)(SC_TILE_BYTES / sizeof(VT)) / S - 1) / 32 * 32;
        if (RC > SC_ROWS) RC = SC_ROWS;
    }
    const bool tiled = RC >= 32;
    if (!tiled) RC = SC_ROWS;  // one sub-chunk, written in place
    const int64_t ld = RC + 1;

    for (int64_t u0 = 0; u0 < tn; u0 += RC) {
        const int64_t un = (tn - u0 < RC) ? (tn - u0) : RC;
        const int64_t rb = r0 + t0 + u0;  // first row of this sub-chunk
        for (int64_t q = threadIdx.x; q <= un; q += SC_THREADS) rp_s[q] = rp[rb + q];
        for (int64_t q = threadIdx.x; q < un; q += SC_THREADS) rem_s[q] = 0;
        if (tiled) {
            for (int64_t q = threadIdx.x; q < S * ld; q += SC_THREADS) tile[q] = zero;
        } else {
            for (int64_t p = 0; p < S; p++)
                for (int64_t t = threadIdx.x; t < un; t += SC_THREADS) dv[p * n_b + (rb - r0) + t] = zero;
        }
        __syncthreads();
        const int32_t e0 = rp_s[0], e1 = rp_s[un];
        // row index of every entry, tabulated by its row's thread when they fit
        const bool rid = e1 - e0 <= SC_RID_MAX;
        if (rid) {
            for (int64_t q = threadIdx.x; q < un; q += SC_THREADS)
                for (int32_t e = rp_s[q]; e < rp_s[q + 1]; e++) rid_s[e - e0] = (uint8_t)q;
            __syncthreads();
        }
        // the loop bound is the warp's first entry, so whole warps iterate
        // together (the ballot below needs every lane)
        const int32_t lane_off = (int32_t)(threadIdx.x & 31);
        for (int32_t wb = e0 + (int32_t)(threadIdx.x - lane_off); wb < e1;
             wb += SC_UNROLL * SC_THREADS) {
            const int32_t eb = wb + lane_off;
            int32_t cc[SC_UNROLL];
            double vv[SC_UNROLL];
#pragma unroll
            for (int u = 0; u < SC_UNROLL; u++) {  // loads of SC_UNROLL entries in flight
                const int32_t e = eb + u * SC_THREADS;
                if (e < e1) {
                    cc[u] = __ldg(col + e);
                    vv[u] = __ldg(val + e);
                }
            }
#pragma unroll
            for (int u = 0; u < SC_UNROLL; u++) {
                const int32_t e = eb + u * SC_THREADS;  // consecutive across the warp
                bool rem = false;
                if (e < e1) {
                    const int32_t r = rid ? (int32_t)rid_s[e - e0] : row_of(rp_s, (int32_t)un, e);
                    const int64_t p = find_sorted(sel, S, cc[u] - (int32_t)(rb + r));
                    if (p < 0) {
                        rem = true;
                        atomicAdd(&rem_s[r], 1);
                    } else if (tiled) {
                        tile[p * ld + r] = round_store<VT>(vv[u]);
                    } else {
                        dv[p * n_b + (rb - r0) + r] = round_store<VT>(vv[u]);
                    }
                }
                // one bit per entry: the warp's 32 bits span at most two words
                const unsigned b = __ballot_sync(0xffffffffu, rem);
                if ((threadIdx.x & 31) == 0 && b) {
                    const int32_t w0 = e >> 5, sh = e & 31;
                    atomicOr(&rem_flag[w0], b << sh);
                    if (sh && (b >> (32 - sh))) atomicOr(&rem_flag[w0 + 1], b >> (32 - sh));
                }
            }
        }
        __syncthreads();
        for (int64_t q = threadIdx.x; q < un; q += SC_THREADS) rem_cnt[rb + q] = rem_s[q];
        if (tiled)
            for (int64_t p = 0; p < S; p++)
                for (int64_t t = threadIdx.x; t < un; t += SC_THREADS)
                    dv[p * n_b + (rb - r0) + t] = tile[p * ld + t];
        __syncthreads();
    }
}

// Remainder (Fig. 12, CSR part), per (block, chunk) as the scatter: the
// chunk's entries are walked in order, 256 at a time, and those whose
// rem_flag bit is set are written in input order from csr_row_ptr of the
// chunk's first row on (block-wide prefix count of the bits).
template <typename VT>
__global__ void __launch_bounds__(SC_THREADS)
k_rem_fill(int64_t n, int32_t n_b, int32_t cpb, const int32_t *__restrict__ rp,
           const int32_t *__restrict__ col, const double *__restrict__ val,
           const uint32_t *__restrict__ rem_flag, const int32_t *__restrict__ csr_row_ptr,
           int32_t *__restrict__ csr_col, VT *__restrict__ csr_val)
{
    __shared__ int32_t wsum[SC_THREADS / 32];
    const int64_t ib = blockIdx.x / cpb;
    const int64_t c = blockIdx.x - ib * cpb;
    const int64_t r0 = ib * (int64_t)n_b;
    const int64_t rows = (n - r0 < n_b) ? (n - r0) : n_b;
    const int64_t t0 = c * SC_ROWS;
    if (t0 >= rows) return;  // CTA-uniform
    const int64_t tn = (rows - t0 < SC_ROWS) ? (rows - t0) : SC_ROWS;
    const int64_t rb = r0 + t0;
    int32_t q = csr_row_ptr[rb];
    if (q == csr_row_ptr[rb + tn]) return;  // no remainder in this chunk (CTA-uniform)
    const int32_t E0 = rp[rb], E1 = rp[rb + tn];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int32_t eb = E0; eb < E1; eb += SC_THREADS) {
        const int32_t e = eb + (int32_t)threadIdx.x;
        const bool f = e < E1 && ((rem_flag[e >> 5] >> (e & 31)) & 1u);
        if (!__syncthreads_or(f)) continue;  // no remainder entry in these 256 (CTA-uniform)
        const unsigned b = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wsum[warp] = __popc(b);
        __syncthreads();
        int32_t before = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < SC_THREADS / 32; w++) {
            const int32_t v = wsum[w];
            before += w < warp ? v : 0;
            tot += v;
        }
        if (f) {
            const int32_t pos = q + before + __popc(b & ((1u << lane) - 1u));
            csr_col[pos] = col[e];
            csr_val[pos] = round_store<VT>(val[e]);
        }
        q += tot;
        __syncthreads();
    }
}

__global__ void k_block_bounds(int64_t n, int32_t n_b, int64_t n_blocks,
                               const int32_t *__restrict__ rowptr, int32_t *__restrict__ out)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > n_blocks) return;
    int64_t r = b * (int64_t)n_b;
    if (r > n) r = n;
    out[b] = rowptr[r];
}

inline unsigned grid_for(int64_t m, int threads) { return (unsigned)((m + threads - 1) / threads); }

// Temporaries come from a stream-ordered pool owned by the library (one per
// device, up to 4 GB kept mapped between builds): allocation and release are
// queued on the build's stream instead of synchronising the device.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

int build_pool(cudaMemPool_t *out)
{
    int dev = 0;
    MHDC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error_msg("mhdc_build: device index out of range");
        return MHDC_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        MHDC_CUDA_TRY(cudaMemPoolCreate(&pool, &props));
        unsigned long long keep = 4ull << 30;
        MHDC_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return MHDC_OK;
}

// Device temporary released (stream-ordered) on scope exit.
struct Buf {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    ~Buf()
    {
        if (p) dfree_async(p, st);
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

int dalloc(Buf &b, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) bytes = 16;
    cudaMemPool_t pool;
    int rc = build_pool(&pool);
    if (rc != MHDC_OK) return rc;
    cudaError_t e = dmalloc_pool(&b.p, bytes, pool, st);
    if (e != cudaSuccess) {
        b.p = nullptr;
        set_error("cudaMallocFromPoolAsync", e);
        return cuda_status(e);
    }
    b.st = st;
    return MHDC_OK;
}

int dalloc_raw(void **p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = dmalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMalloc", e);
        return cuda_status(e);
    }
    return MHDC_OK;
}

#define RC(expr)                          \
    do {                                  \
        int rc_ = (expr);                 \
        if (rc_ != MHDC_OK) return rc_;   \
    } while (0)

// rem_flag: (nnz + 31) / 32 words, zeroed here.
template <typename VT>
int launch_scatter(int64_t n, int32_t n_b, int64_t nb, int64_t nnz, const int32_t *rp,
                   const int32_t *col, const double *val, const int32_t *dia_ptr,
                   const int32_t *sel_list, const int32_t *sel_base_rp, int32_t *dia_offset,
                   VT *dia_val, int32_t *rem_cnt, uint32_t *rem_flag, cudaStream_t st)
{
    if (nb == 0) return MHDC_OK;
    MHDC_CUDA_TRY(cudaMemsetAsync(rem_flag, 0, sizeof(uint32_t) * (size_t)((nnz + 31) / 32), st));
    const int64_t cpb = ((int64_t)n_b + SC_ROWS - 1) / SC_ROWS;
    MHDC_CUDA_TRY(cudaFuncSetAttribute(k_scatter<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SC_SMEM));
    k_scatter<VT><<<(unsigned)(nb * cpb), SC_THREADS, SC_SMEM, st>>>(
        n, n_b, (int32_t)cpb, rp, col, val, dia_ptr, sel_list, sel_base_rp, dia_offset, dia_val,
        rem_cnt, rem_flag);
    MHDC_LAUNCH_CHECK("k_scatter");
    return MHDC_OK;
}

template <typename VT>
int launch_rem_fill(int64_t n, int32_t n_b, int64_t nb, const int32_t *rp, const int32_t *col,
                    const double *val, const uint32_t *rem_flag, const int32_t *csr_row_ptr,
                    int32_t *csr_col, VT *csr_val, cudaStream_t st)
{
    const int64_t cpb = ((int64_t)n_b + SC_ROWS - 1) / SC_ROWS;
    k_rem_fill<VT><<<(unsigned)(nb * cpb), SC_THREADS, 0, st>>>(
        n, n_b, (int32_t)cpb, rp, col, val, rem_flag, csr_row_ptr, csr_col, csr_val);
    MHDC_LAUNCH_CHECK("k_rem_fill");
    return MHDC_OK;
}

template <typename VT>
int scatter_all(mhdc_matrix *A, const int32_t *rp, const int32_t *col, const double *val,
                const int32_t *sel_list, const int32_t *sel_base_rp, cudaStream_t st)
{
    const int64_t n = A->n;
    Buf rem, scr, flag;
    RC(dalloc(rem, sizeof(int32_t) * (size_t)n, st));
    RC(dalloc(scr, sizeof(int32_t) * (size_t)scan_scratch_elems(n), st));
    RC(dalloc(flag, sizeof(uint32_t) * (size_t)((A->nnz + 31) / 32), st));
    RC(launch_scatter<VT>(n, A->n_b, A->n_blocks, A->nnz, rp, col, val, A->dia_ptr, sel_list,
                          sel_base_rp, A->dia_offset, static_cast<VT *>(A->dia_val),
                          rem.as<int32_t>(), flag.as<uint32_t>(), st));
    RC(dalloc_raw((void **)&A->csr_row_ptr, sizeof(int32_t) * (size_t)(n + 1)));
    RC(exclusive_scan_i32(rem.as<int32_t>(), A->csr_row_ptr, n, scr.as<int32_t>(), st));
    int32_t nr = 0;
    MHDC_CUDA_TRY(cudaMemcpyAsync(&nr, A->csr_row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    A->nnz_rem = nr;
    RC(dalloc_raw((void **)&A->csr_col, sizeof(int32_t) * (size_t)nr));
    RC(dalloc_raw(&A->csr_val, sizeof(VT) * (size_t)nr));
    if (nr > 0)
        RC(launch_rem_fill<VT>(n, A->n_b, A->n_blocks, rp, col, val, flag.as<uint32_t>(),
                               A->csr_row_ptr, A->csr_col, static_cast<VT *>(A->csr_val), st));
    return MHDC_OK;
}

// Blocks whose overflow flag is set, with their entry counts (host lists).
int overflowed_blocks(const int32_t *d_ovf, const int32_t *d_bounds, int64_t nb,
                      std::vector<int32_t> &ids, std::vector<int64_t> &entries, cudaStream_t st)
{
    std::vector<int32_t> h_ovf((size_t)nb), h_bounds((size_t)nb + 1);
    MHDC_CUDA_TRY(cudaMemcpyAsync(h_ovf.data(), d_ovf, sizeof(int32_t) * nb,
                                  cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaMemcpyAsync(h_bounds.data(), d_bounds, sizeof(int32_t) * (nb + 1),
                                  cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    ids.clear();
    entries.clear();
    for (int64_t b = 0; b < nb; b++) {
        if (!h_ovf[b]) continue;
        ids.push_back((int32_t)b);
        entries.push_back((int64_t)h_bounds[b + 1] - h_bounds[b]);
    }
    return MHDC_OK;
}

int select_block_mode(mhdc_matrix *A, const int32_t *rp, const int32_t *col, Buf &sel_out,
                      cudaStream_t st)
{
    const int64_t n = A->n, nnz = A->nnz, nb = A->n_blocks;
    Buf sel_cnt, ovf, scr, bounds;
    RC(dalloc(sel_out, sizeof(int32_t) * (size_t)nnz, st));
    RC(dalloc(sel_cnt, sizeof(int32_t) * (size_t)nb, st));
    RC(dalloc(ovf, sizeof(int32_t) * (size_t)nb, st));
    RC(dalloc(bounds, sizeof(int32_t) * (size_t)(nb + 1), st));
    // level 1: small shared tables, staged columns
    MHDC_CUDA_TRY(cudaFuncSetAttribute(k_count_select<false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)CS_SMEM_SMALL));
    k_count_select<false, true><<<(unsigned)nb, CS_THREADS, CS_SMEM_SMALL, st>>>(
        n, A->n_b, rp, col, A->theta, nullptr, SMALL_CAP, CW, nullptr, nullptr, nullptr, nullptr,
        sel_out.as<int32_t>(), sel_cnt.as<int32_t>(), ovf.as<int32_t>());
    MHDC_LAUNCH_CHECK("k_count_select<level 1>");
    k_block_bounds<<<grid_for(nb + 1, 256), 256, 0, st>>>(n, A->n_b, nb, rp, bounds.as<int32_t>());
    MHDC_LAUNCH_CHECK("k_block_bounds");
    std::vector<int32_t> ids;
    std::vector<int64_t> entries;
    RC(overflowed_blocks(ovf.as<int32_t>(), bounds.as<int32_t>(), nb, ids, entries, st));
    if (!ids.empty()) {
        // level 2: the largest shared tables for the blocks level 1 could not hold
        Buf d_ids;
        RC(dalloc(d_ids, sizeof(int32_t) * ids.size(), st));
        MHDC_CUDA_TRY(cudaMemcpyAsync(d_ids.p, ids.data(), sizeof(int32_t) * ids.size(),
                                      cudaMemcpyHostToDevice, st));
        MHDC_CUDA_TRY(cudaFuncSetAttribute(k_count_select<false, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)CS_SMEM_L2));
        k_count_select<false, true><<<(unsigned)ids.size(), CS_THREADS, CS_SMEM_L2, st>>>(
            n, A->n_b, rp, col, A->theta, d_ids.as<int32_t>(), HCAP, CW_L2, nullptr, nullptr,
            nullptr, nullptr, sel_out.as<int32_t>(), sel_cnt.as<int32_t>(), ovf.as<int32_t>());
        MHDC_LAUNCH_CHECK("k_count_select<level 2>");
        RC(overflowed_blocks(ovf.as<int32_t>(), bounds.as<int32_t>(), nb, ids, entries, st));
    }
    if (!ids.empty()) {
        // level 3: global tables of at least twice the block's entries
        std::vector<int32_t> lg;
        std::vector<int64_t> base;
        int64_t total = 0;
        for (int64_t m : entries) {
            int l = 10;
            while (((int64_t)1 << l) < 2 * m) l++;
            lg.push_back(l);
            base.push_back(total);
            total += (int64_t)1 << l;
        }
        Buf gk, gc, d_ids, d_lg, d_base;
        RC(dalloc(gk, sizeof(int32_t) * (size_t)total, st));
        RC(dalloc(gc, sizeof(int32_t) * (size_t)total, st));
        RC(dalloc(d_ids, sizeof(int32_t) * ids.size(), st));
        RC(dalloc(d_lg, sizeof(int32_t) * lg.size(), st));
        RC(dalloc(d_base, sizeof(int64_t) * base.size(), st));
        MHDC_CUDA_TRY(cudaMemcpyAsync(d_ids.p, ids.data(), sizeof(int32_t) * ids.size(),
                                      cudaMemcpyHostToDevice, st));
        MHDC_CUDA_TRY(cudaMemcpyAsync(d_lg.p, lg.data(), sizeof(int32_t) * lg.size(),
                                      cudaMemcpyHostToDevice, st));
        MHDC_CUDA_TRY(cudaMemcpyAsync(d_base.p, base.data(), sizeof(int64_t) * base.size(),
                                      cudaMemcpyHostToDevice, st));
        k_count_select<true, false><<<(unsigned)ids.size(), CS_THREADS, 0, st>>>(
            n, A->n_b, rp, col, A->theta, d_ids.as<int32_t>(), 0, 0, gk.as<int32_t>(),
            gc.as<int32_t>(), d_base.as<int64_t>(), d_lg.as<int32_t>(), sel_out.as<int32_t>(),
            sel_cnt.as<int32_t>(), ovf.as<int32_t>());
        MHDC_LAUNCH_CHECK("k_count_select<level 3>");
        // a global table cannot overflow (its capacity is at least twice the
        // block's entries); check the flags anyway
        RC(overflowed_blocks(ovf.as<int32_t>(), bounds.as<int32_t>(), nb, ids, entries, st));
        if (!ids.empty()) {
            set_error_msg("k_count_select: global table overflow");
            return MHDC_ERR_DEVICE_CHECK;
        }
    }
    RC(dalloc_raw((void **)&A->dia_ptr, sizeof(int32_t) * (size_t)(nb + 1)));
    RC(dalloc(scr, sizeof(int32_t) * (size_t)scan_scratch_elems(nb), st));
    RC(exclusive_scan_i32(sel_cnt.as<int32_t>(), A->dia_ptr, nb, scr.as<int32_t>(), st));
    int32_t P = 0;
    MHDC_CUDA_TRY(cudaMemcpyAsync(&P, A->dia_ptr + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    A->P = P;
    return MHDC_OK;
}

int select_global_mode(mhdc_matrix *A, const int32_t *rp, const int32_t *col, Buf &sel_out,
                       cudaStream_t st)
{
    const int64_t n = A->n, nb = A->n_blocks;
    const int64_t m = 2 * n - 1;
    Buf cnt, flags, pos, scr;
    RC(dalloc(cnt, sizeof(int32_t) * (size_t)m, st));
    RC(dalloc(flags, sizeof(int32_t) * (size_t)m, st));
    RC(dalloc(pos, sizeof(int32_t) * (size_t)(m + 1), st));
    RC(dalloc(scr, sizeof(int32_t) * (size_t)scan_scratch_elems(m), st));
    MHDC_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (size_t)m, st));
    // six CTAs per SM (shared memory allows seven), grid-stride over the row groups
    k_count_all<<<(unsigned)(read_bench_grid() / 8 * 6), CA_THREADS, CA_SMEM, st>>>(n, rp, col,
                                                                            cnt.as<int32_t>());
    MHDC_LAUNCH_CHECK("k_count_all");
    k_flag_global<<<grid_for(m, 256), 256, 0, st>>>(m, cnt.as<int32_t>(), A->theta * (double)n,
                                                     flags.as<int32_t>());
    MHDC_LAUNCH_CHECK("k_flag_global");
    RC(exclusive_scan_i32(flags.as<int32_t>(), pos.as<int32_t>(), m, scr.as<int32_t>(), st));
    int32_t S = 0;
    MHDC_CUDA_TRY(cudaMemcpyAsync(&S, pos.as<int32_t>() + m, sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    if ((int64_t)S * nb >= INT32_MAX) {
        set_error_msg("hdc_build: number of partial diagonals exceeds int32");
        return MHDC_ERR_UNSUPPORTED;
    }
    RC(dalloc(sel_out, sizeof(int32_t) * (size_t)S, st));
    k_compact_global<<<grid_for(m, 256), 256, 0, st>>>(m, n, flags.as<int32_t>(),
                                                        pos.as<int32_t>(), sel_out.as<int32_t>());
    MHDC_LAUNCH_CHECK("k_compact_global");
    RC(dalloc_raw((void **)&A->dia_ptr, sizeof(int32_t) * (size_t)(nb + 1)));
    k_uniform_ptr<<<grid_for(nb + 1, 256), 256, 0, st>>>(nb, S, A->dia_ptr);
    MHDC_LAUNCH_CHECK("k_uniform_ptr");
    A->P = (int64_t)S * nb;
    return MHDC_OK;
}

int finish_stats(mhdc_matrix *A, cudaStream_t st)
{
    const int64_t nb = A->n_blocks;
    std::vector<int32_t> h((size_t)nb + 1);
    Buf bounds;
    RC(dalloc(bounds, sizeof(int32_t) * (size_t)(nb + 1), st));
    k_block_bounds<<<grid_for(nb + 1, 256), 256, 0, st>>>(A->n, A->n_b, nb, A->csr_row_ptr,
                                                          bounds.as<int32_t>());
    MHDC_LAUNCH_CHECK("k_block_bounds");
    MHDC_CUDA_TRY(cudaMemcpyAsync(h.data(), bounds.p, sizeof(int32_t) * (nb + 1),
                                  cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    int64_t rr = 0;
    for (int64_t b = 0; b < nb; b++) {
        if (h[b + 1] != h[b]) {
            const int64_t r0 = b * (int64_t)A->n_b;
            rr += (A->n - r0 < A->n_b) ? (A->n - r0) : A->n_b;
        }
    }
    A->rem_block_rows = rr;
    const int64_t sv = (int64_t)value_size(A->dtype), sy = (int64_t)y_size(A->dtype);
    // V = V_A + V_x + V_y (Sec. 5.1; terms of Sec. 5.3.3): dia_val, dia_offset,
    // dia_ptr, csr_val + csr_col_ind, csr_row_ptr (blocks with a remainder,
    // plus the two bounds each block reads), x once, y once.
    A->bytes_model = sv * A->P * A->n_b + 4 * A->P + 4 * (nb + 1) + (sv + 4) * A->nnz_rem +
                     4 * (rr + 2 * nb) + sv * A->n + sy * A->n;
    A->bytes_device = (int64_t)(sv * A->P * A->n_b + 4 * A->P + 4 * (nb + 1) +
                                (sv + 4) * A->nnz_rem + 4 * (A->n + 1));
    return MHDC_OK;
}

}  // namespace

int feature_hist(int64_t n, const int32_t *rp, const int32_t *col, int32_t n_b,
                 cudaStream_t st, unsigned long long *h_ent, unsigned long long *h_dia)
{
    const int64_t nb = (n + n_b - 1) / n_b;
    Buf d;
    RC(dalloc(d, 20 * sizeof(unsigned long long), st));
    MHDC_CUDA_TRY(cudaMemsetAsync(d.p, 0, 20 * sizeof(unsigned long long), st));
    if (nb > 0) {
        MHDC_CUDA_TRY(cudaFuncSetAttribute(k_count_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(2 * HCAP * sizeof(int32_t))));
        k_count_hist<<<(unsigned)nb, CS_THREADS, 2 * HCAP * sizeof(int32_t), st>>>(
            n, n_b, rp, col, d.as<unsigned long long>(), d.as<unsigned long long>() + 10);
        MHDC_LAUNCH_CHECK("k_count_hist");
    }
    unsigned long long h[20];
    MHDC_CUDA_TRY(cudaMemcpyAsync(h, d.p, sizeof h, cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    memcpy(h_ent, h, 10 * sizeof(unsigned long long));
    memcpy(h_dia, h + 10, 10 * sizeof(unsigned long long));
    return MHDC_OK;
}

void free_matrix(mhdc_matrix *A)
{
    if (!A) return;
    dfree(A->dia_ptr);
    dfree(A->dia_offset);
    dfree(A->dia_val);
    dfree(A->csr_row_ptr);
    dfree(A->csr_col);
    dfree(A->csr_val);
    dfree(A->x_stage);
    dfree(A->y_stage);
    for (int k = 0; k < mhdc_matrix::ASYNC_SLOTS; k++) {
        if (A->ae_done[k]) cudaEventSynchronize(A->ae_done[k]);
        dfree(A->ax[k]);
        dfree(A->ay[k]);
        if (A->ae_in[k]) cudaEventDestroy(A->ae_in[k]);
        if (A->ae_comp[k]) cudaEventDestroy(A->ae_comp[k]);
        if (A->ae_done[k]) cudaEventDestroy(A->ae_done[k]);
    }
    if (A->as_in) cudaStreamDestroy(A->as_in);
    if (A->as_comp) cudaStreamDestroy(A->as_comp);
    if (A->as_out) cudaStreamDestroy(A->as_out);
    dfree(A->status);
    dfree(A->sched);
    dfree(A->dia_dw);
    dfree(A->csr_dw);
    dfree(A->x_dw);
    delete A;
}

namespace {

// (hi, lo) = (RN32(v), RN32(v - hi)): the FP32 pair of an FP64 value (build time).
__global__ void k_split_dw(int64_t m, const double *__restrict__ v, float2 *__restrict__ out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const double d = v[k];
    const float h = __double2float_rn(d);
    out[k] = make_float2(h, __double2float_rn(d - (double)h));
}

// flag |= 1 if a nonzero value lies outside [2^DW_EMIN, 2^DW_EMAX] or is not
// finite (exponent field tests, one atomic per warp).
__global__ void k_value_window(int64_t m, const double *__restrict__ v, int *flag)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (k < m) {
        const unsigned long long u =
            (unsigned long long)__double_as_longlong(v[k]) & 0x7FFFFFFFFFFFFFFFull;
        const int E = (int)(u >> 52) - 1023;
        bad = u != 0 && (E < DW_EMIN || E > DW_EMAX ||
                         (E == DW_EMAX && (u & 0xFFFFFFFFFFFFFull) != 0));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// out = max over i of ptr[i + 1] - ptr[i], i < m (one atomic per warp).
__global__ void k_max_diff(int64_t m, const int32_t *__restrict__ ptr, int *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = __reduce_max_sync(0xffffffffu, i < m ? ptr[i + 1] - ptr[i] : 0);
    if ((threadIdx.x & 31) == 0) atomicMax(out, d);
}

}  // namespace

// Split an FP64 handle's values into FP32 pairs and decide whether the
// emulated product may be used.  Lack of memory only disables emulation.
static void free_dw(mhdc_matrix *A)
{
    dfree(A->dia_dw);
    dfree(A->csr_dw);
    dfree(A->x_dw);
    A->dia_dw = A->csr_dw = A->x_dw = nullptr;
}

// The FP32-pair arrays of the emulated FP64 variants.  On any failure they
// are released again (the handle keeps its native variants) and the error is
// returned.
static int prepare_dw_arrays(mhdc_matrix *A, cudaStream_t st)
{
    const int64_t nd = A->P * (int64_t)A->n_b;
    MHDC_CUDA_TRY(dmalloc((void **)&A->dia_dw, sizeof(float2) * (size_t)(nd ? nd : 1)));
    MHDC_CUDA_TRY(dmalloc((void **)&A->csr_dw, sizeof(float2) * (size_t)(A->nnz_rem ? A->nnz_rem : 1)));
    MHDC_CUDA_TRY(dmalloc((void **)&A->x_dw, sizeof(float2) * (size_t)A->n));
    Buf w;
    RC(dalloc(w, 2 * sizeof(int), st));
    MHDC_CUDA_TRY(cudaMemsetAsync(w.p, 0, 2 * sizeof(int), st));
    if (nd > 0) {
        k_split_dw<<<grid_for(nd, 256), 256, 0, st>>>(nd, (const double *)A->dia_val, A->dia_dw);
        k_value_window<<<grid_for(nd, 256), 256, 0, st>>>(nd, (const double *)A->dia_val, w.as<int>());
    }
    if (A->nnz_rem > 0) {
        k_split_dw<<<grid_for(A->nnz_rem, 256), 256, 0, st>>>(A->nnz_rem, (const double *)A->csr_val,
                                                              A->csr_dw);
        k_value_window<<<grid_for(A->nnz_rem, 256), 256, 0, st>>>(
            A->nnz_rem, (const double *)A->csr_val, w.as<int>());
    }
    MHDC_LAUNCH_CHECK("k_split_dw");
    int h[3] = {0, 0, 0};
    Buf mx;
    RC(dalloc(mx, 2 * sizeof(int), st));
    MHDC_CUDA_TRY(cudaMemsetAsync(mx.p, 0, 2 * sizeof(int), st));
    k_max_diff<<<grid_for(A->n_blocks, 256), 256, 0, st>>>(A->n_blocks, A->dia_ptr, mx.as<int>());
    k_max_diff<<<grid_for(A->n, 256), 256, 0, st>>>(A->n, A->csr_row_ptr, mx.as<int>() + 1);
    MHDC_LAUNCH_CHECK("k_max_diff");
    MHDC_CUDA_TRY(cudaMemcpyAsync(h, w.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaMemcpyAsync(h + 1, mx.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    A->dw_ok = h[0] == 0 && (h[1] + h[2]) <= DW_MAX_TERMS;
    A->bytes_device += (int64_t)sizeof(float2) * (nd + A->nnz_rem + A->n);
    return MHDC_OK;
}

int prepare_dw(mhdc_matrix *A, cudaStream_t st)
{
    A->dw_ok = false;
    if (A->dtype != MHDC_F64 || A->n == 0) return MHDC_OK;
    const int rc = prepare_dw_arrays(A, st);
    if (rc != MHDC_OK) {
        cudaStreamSynchronize(st);  // kernels that write the arrays are done
        free_dw(A);
        A->dw_ok = false;
    }
    return rc;
}

int ensure_dw(mhdc_matrix *A, cudaStream_t st)
{
    if (A->dw_prepared) return MHDC_OK;
    const int rc = prepare_dw(A, st);
    A->dw_prepared = rc == MHDC_OK;
    return rc;
}

static int build_into(mhdc_matrix *A, const int32_t *rp, const int32_t *col, const double *val,
                      cudaStream_t st)
{
    const int64_t n = A->n;
    RC(dalloc_raw((void **)&A->status, sizeof(int)));
    MHDC_CUDA_TRY(cudaMemsetAsync(A->status, 0, sizeof(int), st));
    RC(dalloc_raw((void **)&A->sched, 2 * sizeof(unsigned long long)));
    MHDC_CUDA_TRY(cudaMemsetAsync(A->sched, 0, 2 * sizeof(unsigned long long), st));
    if (n == 0) {
        RC(dalloc_raw((void **)&A->dia_ptr, sizeof(int32_t)));
        RC(dalloc_raw((void **)&A->csr_row_ptr, sizeof(int32_t)));
        RC(dalloc_raw((void **)&A->dia_offset, 0));
        RC(dalloc_raw(&A->dia_val, 0));
        RC(dalloc_raw((void **)&A->csr_col, 0));
        RC(dalloc_raw(&A->csr_val, 0));
        MHDC_CUDA_TRY(cudaMemsetAsync(A->dia_ptr, 0, sizeof(int32_t), st));
        MHDC_CUDA_TRY(cudaMemsetAsync(A->csr_row_ptr, 0, sizeof(int32_t), st));
        MHDC_CUDA_TRY(cudaStreamSynchronize(st));
        return MHDC_OK;
    }
    int32_t nnz = 0;
    MHDC_CUDA_TRY(cudaMemcpyAsync(&nnz, rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    if (nnz < 0) {
        set_error_msg("mhdc_build: row_ptr[n] < 0");
        return MHDC_ERR_BAD_CSR;
    }
    A->nnz = nnz;
    if (nnz > 0 && (!col || !val)) {
        set_error_msg("mhdc_build: null column or value array with nnz > 0");
        return MHDC_ERR_INVALID_ARG;
    }
    {
        Buf err;
        RC(dalloc(err, sizeof(int), st));
        MHDC_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(int), st));
        if (n > 0) {
            k_validate<<<grid_for(n, 256), 256, 0, st>>>(n, rp, col, nnz, err.as<int>());
            MHDC_LAUNCH_CHECK("k_validate");
        }
        int h = 0;
        MHDC_CUDA_TRY(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        MHDC_CUDA_TRY(cudaStreamSynchronize(st));
        if (h) {
            char msg[128];
            snprintf(msg, sizeof msg, "mhdc_build: invalid CSR (flags 0x%x: %s%s%s%s)", h,
                     (h & 1) ? "row_ptr[0]!=0 " : "", (h & 2) ? "row_ptr out of order " : "",
                     (h & 4) ? "column out of range " : "", (h & 8) ? "columns not increasing" : "");
            set_error_msg(msg);
            return MHDC_ERR_BAD_CSR;
        }
    }
    Buf sel_out;
    if (A->mode == MHDC_MODE_BLOCK) {
        RC(select_block_mode(A, rp, col, sel_out, st));
    } else {
        RC(select_global_mode(A, rp, col, sel_out, st));
    }
    const size_t sv = value_size(A->dtype);
    RC(dalloc_raw((void **)&A->dia_offset, sizeof(int32_t) * (size_t)A->P));
    RC(dalloc_raw(&A->dia_val, sv * (size_t)A->P * (size_t)A->n_b));
    const int32_t *base = A->mode == MHDC_MODE_BLOCK ? rp : nullptr;
    switch (A->dtype) {
    case MHDC_F64:
        RC(scatter_all<double>(A, rp, col, val, sel_out.as<int32_t>(), base, st));
        break;
    case MHDC_F32:
        RC(scatter_all<float>(A, rp, col, val, sel_out.as<int32_t>(), base, st));
        break;
    default:
        RC(scatter_all<__nv_bfloat16>(A, rp, col, val, sel_out.as<int32_t>(), base, st));
        break;
    }
    RC(finish_stats(A, st));
    A->spmv_grid = spmv_grid_for(A);
    return MHDC_OK;
}

int build_matrix(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
                 int32_t n_b, double theta, int32_t dtype, int mode, cudaStream_t stream,
                 mhdc_matrix **out)
{
    if (!out || !d_row_ptr || n < 0 || n >= INT32_MAX || n_b < 1 || !std::isfinite(theta) ||
        theta < 0.0 || dtype < MHDC_F64 || dtype > MHDC_BF16) {
        set_error_msg("mhdc_build: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    mhdc_matrix *A = new mhdc_matrix();
    A->n = n;
    A->n_b = n_b;
    A->n_blocks = n == 0 ? 0 : (n + n_b - 1) / n_b;
    A->theta = theta;
    A->dtype = dtype;
    A->mode = mode;
    cudaGetDevice(&A->device);
    int rc = build_into(A, d_row_ptr, d_col, d_val, stream);
    if (rc != MHDC_OK) {
        cudaStreamSynchronize(stream);
        free_matrix(A);
        return rc;
    }
    *out = A;
    return MHDC_OK;
}

// ---------------------------------------------------------------------------
// M-HDC straight from DIA input (Sec. 3.3, Fig. 4 layout: val[d * n + i] =
// a(i, i + offset[d])), as a stencil code holds its matrix: no CSR copy.
// Entries are the in-range positions with a nonzero value, so the result is
// the one mhdc_build gives for the CSR matrix of those entries (the same
// counts, selection, rounding, padding and remainder order).  Every pass is
// an elementwise walk over the DIA array (coalesced).
// ---------------------------------------------------------------------------
namespace {

// err |= 1: an offset outside (-n, n); 2: offsets not strictly increasing
__global__ void k_dia_check(int32_t nd, int64_t n, const int32_t *__restrict__ off, int *err)
{
    const int32_t d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nd) return;
    const int64_t o = off[d];
    if (o <= -n || o >= n) atomicOr(err, 1);
    if (d > 0 && (int64_t)off[d - 1] >= o) atomicOr(err, 2);
}

__device__ __forceinline__ bool dia_entry(const double *__restrict__ val, const int32_t *__restrict__ off,
                                          int64_t n, int32_t d, int64_t i, double *v)
{
    const int64_t j = i + off[d];
    if (j < 0 || j >= n) return false;
    *v = val[(int64_t)d * n + i];
    return *v != 0.0;
}

// cnt[ib * nd + d] = entries of diagonal d = blockIdx.y in row block ib; one
// atomic per warp and block (lanes of one block grouped by a warp match)
__global__ void __launch_bounds__(256)
k_dia_count(int64_t n, int32_t n_b, int32_t nd, const int32_t *__restrict__ off,
            const double *__restrict__ val, int32_t *cnt)
{
    const int32_t d = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; i0 < n; i0 += stride) {
        const int64_t i = i0 + lane;
        double v;
        const bool e = i < n && dia_entry(val, off, n, d, i, &v);
        const int64_t ib = (i < n ? i : n - 1) / n_b;
        const unsigned grp = __match_any_sync(0xffffffffu, (unsigned long long)ib);
        const unsigned hits = __ballot_sync(0xffffffffu, e) & grp;
        if (lane == __ffs(grp) - 1 && hits) atomicAdd(&cnt[ib * nd + d], __popc(hits));
    }
}

// Selection (Sec. 4.3): keep[ib * nd + d] = count >= 1 and >= theta * rows(ib)
__global__ void k_dia_select(int64_t n, int32_t n_b, int64_t nb, int32_t nd, double theta,
                             const int32_t *__restrict__ cnt, int32_t *keep, int32_t *sel_cnt,
                             unsigned long long *total)
{
    const int64_t ib = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ib >= nb) return;
    const int64_t r0 = ib * (int64_t)n_b;
    const double thr = theta * (double)((n - r0 < n_b) ? (n - r0) : n_b);
    int32_t S = 0;
    unsigned long long entries = 0;
    for (int32_t d = 0; d < nd; d++) {
        const int32_t c = cnt[ib * nd + d];
        const int32_t k = (c >= 1 && (double)c >= thr) ? 1 : 0;
        keep[ib * nd + d] = k;
        S += k;
        entries += (unsigned long long)c;
    }
    sel_cnt[ib] = S;
    if (entries) atomicAdd(total, entries);  // one atomic per row block
}

// dia_offset and, per partial diagonal p, its source (block, diagonal);
// keep[] becomes the position p of a kept diagonal, -1 otherwise
__global__ void k_dia_place(int64_t nb, int32_t nd, const int32_t *__restrict__ off,
                            const int32_t *__restrict__ dia_ptr, int32_t *keep,
                            int32_t *dia_offset, int32_t *src_d, int32_t *src_b)
{
    const int64_t ib = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ib >= nb) return;
    int32_t p = dia_ptr[ib];
    for (int32_t d = 0; d < nd; d++) {
        if (keep[ib * nd + d]) {
            dia_offset[p] = off[d];
            src_d[p] = d;
            src_b[p] = (int32_t)ib;
            keep[ib * nd + d] = p++;
        } else {
            keep[ib * nd + d] = -1;
        }
    }
}

// dia_val slot (p, t): the value rounded to the storage type, +0.0 where
// there is no entry (past the matrix end, outside the columns, or zero)
// (grid y walks the partial diagonals, grid x the slots of one)
template <typename VT>
__global__ void k_dia_fill(int64_t n, int32_t n_b, int64_t P, const int32_t *__restrict__ off,
                           const double *__restrict__ val, const int32_t *__restrict__ src_d,
                           const int32_t *__restrict__ src_b, VT *__restrict__ dia_val)
{
    for (int64_t p = blockIdx.y; p < P; p += gridDim.y) {
        const int32_t d = src_d[p];
        const int64_t r0 = (int64_t)src_b[p] * n_b;
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_b;
             t += (int64_t)gridDim.x * blockDim.x) {
            double v = 0.0;
            if (!(r0 + t < n && dia_entry(val, off, n, d, r0 + t, &v))) v = 0.0;
            dia_val[p * n_b + t] = round_store<VT>(v);
        }
    }
}

// per row: entries on the diagonals its block does not keep
__global__ void k_dia_rem_count(int64_t n, int32_t n_b, int32_t nd, const int32_t *__restrict__ off,
                                const double *__restrict__ val, const int32_t *__restrict__ keep,
                                int32_t *rem)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t *kb = keep + (i / n_b) * nd;
    int32_t c = 0;
    for (int32_t d = 0; d < nd; d++) {
        double v;
        if (kb[d] < 0 && dia_entry(val, off, n, d, i, &v)) c++;
    }
    rem[i] = c;
}

// the remainder entries of row i in column order (= ascending offsets)
template <typename VT>
__global__ void k_dia_rem_fill(int64_t n, int32_t n_b, int32_t nd, const int32_t *__restrict__ off,
                               const double *__restrict__ val, const int32_t *__restrict__ keep,
                               const int32_t *__restrict__ csr_row_ptr, int32_t *__restrict__ csr_col,
                               VT *__restrict__ csr_val)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t q = csr_row_ptr[i];
    if (q == csr_row_ptr[i + 1]) return;
    const int32_t *kb = keep + (i / n_b) * nd;
    for (int32_t d = 0; d < nd; d++) {
        double v;
        if (kb[d] < 0 && dia_entry(val, off, n, d, i, &v)) {
            csr_col[q] = (int32_t)(i + off[d]);
            csr_val[q] = round_store<VT>(v);
            q++;
        }
    }
}

template <typename VT>
int dia_fill_all(mhdc_matrix *A, int32_t nd, const int32_t *off, const double *val,
                 const int32_t *keep, const int32_t *src_d, const int32_t *src_b, cudaStream_t st)
{
    const int64_t n = A->n;
    if (A->P > 0) {
        const int64_t gx = ((int64_t)A->n_b + 255) / 256 < 64 ? ((int64_t)A->n_b + 255) / 256 : 64;
        const int64_t gy = A->P < 65535 ? A->P : 65535;
        k_dia_fill<VT><<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(
            n, A->n_b, A->P, off, val, src_d, src_b, static_cast<VT *>(A->dia_val));
        MHDC_LAUNCH_CHECK("k_dia_fill");
    }
    Buf rem, scr;
    RC(dalloc(rem, sizeof(int32_t) * (size_t)n, st));
    RC(dalloc(scr, sizeof(int32_t) * (size_t)scan_scratch_elems(n), st));
    k_dia_rem_count<<<grid_for(n, 256), 256, 0, st>>>(n, A->n_b, nd, off, val, keep, rem.as<int32_t>());
    MHDC_LAUNCH_CHECK("k_dia_rem_count");
    RC(dalloc_raw((void **)&A->csr_row_ptr, sizeof(int32_t) * (size_t)(n + 1)));
    RC(exclusive_scan_i32(rem.as<int32_t>(), A->csr_row_ptr, n, scr.as<int32_t>(), st));
    int32_t nr = 0;
    MHDC_CUDA_TRY(cudaMemcpyAsync(&nr, A->csr_row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    A->nnz_rem = nr;
    RC(dalloc_raw((void **)&A->csr_col, sizeof(int32_t) * (size_t)nr));
    RC(dalloc_raw(&A->csr_val, sizeof(VT) * (size_t)nr));
    if (nr > 0) {
        k_dia_rem_fill<VT><<<grid_for(n, 256), 256, 0, st>>>(n, A->n_b, nd, off, val, keep,
                                                             A->csr_row_ptr, A->csr_col,
                                                             static_cast<VT *>(A->csr_val));
        MHDC_LAUNCH_CHECK("k_dia_rem_fill");
    }
    return MHDC_OK;
}

int build_dia_into(mhdc_matrix *A, int32_t nd, const int32_t *off, const double *val,
                   cudaStream_t st)
{
    const int64_t n = A->n, nb = A->n_blocks;
    RC(dalloc_raw((void **)&A->status, sizeof(int)));
    MHDC_CUDA_TRY(cudaMemsetAsync(A->status, 0, sizeof(int), st));
    RC(dalloc_raw((void **)&A->sched, 2 * sizeof(unsigned long long)));
    MHDC_CUDA_TRY(cudaMemsetAsync(A->sched, 0, 2 * sizeof(unsigned long long), st));
    Buf err, cnt, keep, sel_cnt, scr, total;
    RC(dalloc(err, sizeof(int), st));
    MHDC_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    if (nd > 0) {
        k_dia_check<<<(nd + 255) / 256, 256, 0, st>>>(nd, n, off, err.as<int>());
        MHDC_LAUNCH_CHECK("k_dia_check");
    }
    int h_err = 0;
    MHDC_CUDA_TRY(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err) {
        set_error_msg((h_err & 1) ? "mhdc_build_dia: an offset lies outside (-n, n)"
                                  : "mhdc_build_dia: offsets not strictly increasing");
        return MHDC_ERR_INVALID_ARG;
    }
    const size_t cells = (size_t)nb * (size_t)(nd > 0 ? nd : 1);
    RC(dalloc(cnt, sizeof(int32_t) * cells, st));
    RC(dalloc(keep, sizeof(int32_t) * cells, st));
    RC(dalloc(sel_cnt, sizeof(int32_t) * (size_t)nb, st));
    RC(dalloc(total, sizeof(unsigned long long), st));
    MHDC_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * cells, st));
    MHDC_CUDA_TRY(cudaMemsetAsync(total.p, 0, sizeof(unsigned long long), st));
    if (nd > 0) {
        const int64_t gx = (n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048;
        k_dia_count<<<dim3((unsigned)gx, (unsigned)nd), 256, 0, st>>>(n, A->n_b, nd, off, val,
                                                                      cnt.as<int32_t>());
        MHDC_LAUNCH_CHECK("k_dia_count");
    }
    k_dia_select<<<grid_for(nb, 256), 256, 0, st>>>(n, A->n_b, nb, nd, A->theta, cnt.as<int32_t>(),
                                                     keep.as<int32_t>(), sel_cnt.as<int32_t>(),
                                                     total.as<unsigned long long>());
    MHDC_LAUNCH_CHECK("k_dia_select");
    RC(dalloc_raw((void **)&A->dia_ptr, sizeof(int32_t) * (size_t)(nb + 1)));
    RC(dalloc(scr, sizeof(int32_t) * (size_t)scan_scratch_elems(nb), st));
    RC(exclusive_scan_i32(sel_cnt.as<int32_t>(), A->dia_ptr, nb, scr.as<int32_t>(), st));
    int32_t P = 0;
    unsigned long long nnz = 0;
    MHDC_CUDA_TRY(cudaMemcpyAsync(&P, A->dia_ptr + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaMemcpyAsync(&nnz, total.p, sizeof nnz, cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    if (nnz >= (unsigned long long)INT32_MAX) {
        set_error_msg("mhdc_build_dia: more than 2^31 - 1 entries");
        return MHDC_ERR_UNSUPPORTED;
    }
    A->nnz = (int64_t)nnz;
    A->P = P;
    Buf src_d, src_b;
    RC(dalloc(src_d, sizeof(int32_t) * (size_t)P, st));
    RC(dalloc(src_b, sizeof(int32_t) * (size_t)P, st));
    RC(dalloc_raw((void **)&A->dia_offset, sizeof(int32_t) * (size_t)P));
    RC(dalloc_raw(&A->dia_val, value_size(A->dtype) * (size_t)P * (size_t)A->n_b));
    k_dia_place<<<grid_for(nb, 256), 256, 0, st>>>(nb, nd, off, A->dia_ptr, keep.as<int32_t>(),
                                                    A->dia_offset, src_d.as<int32_t>(),
                                                    src_b.as<int32_t>());
    MHDC_LAUNCH_CHECK("k_dia_place");
    switch (A->dtype) {
    case MHDC_F64:
        RC(dia_fill_all<double>(A, nd, off, val, keep.as<int32_t>(), src_d.as<int32_t>(),
                                src_b.as<int32_t>(), st));
        break;
    case MHDC_F32:
        RC(dia_fill_all<float>(A, nd, off, val, keep.as<int32_t>(), src_d.as<int32_t>(),
                               src_b.as<int32_t>(), st));
        break;
    default:
        RC(dia_fill_all<__nv_bfloat16>(A, nd, off, val, keep.as<int32_t>(), src_d.as<int32_t>(),
                                       src_b.as<int32_t>(), st));
        break;
    }
    RC(finish_stats(A, st));
    A->spmv_grid = spmv_grid_for(A);
    return MHDC_OK;
}

}  // namespace

int tmp_alloc(void **p, size_t bytes, cudaStream_t st)
{
    Buf b;
    RC(dalloc(b, bytes, st));
    *p = b.p;
    b.p = nullptr;  // ownership passes to the caller (tmp_free)
    return MHDC_OK;
}

void tmp_free(void *p, cudaStream_t st)
{
    if (p) dfree_async(p, st);
}

int build_matrix_dia(int64_t n, int32_t nd, const int32_t *d_offset, const double *d_val,
                     int32_t n_b, double theta, int32_t dtype, cudaStream_t stream,
                     mhdc_matrix **out)
{
    if (!out || n < 1 || n >= INT32_MAX || nd < 0 || nd > 65535 || n_b < 1 ||
        !std::isfinite(theta) || theta < 0.0 || dtype < MHDC_F64 || dtype > MHDC_BF16 ||
        (nd > 0 && (!d_offset || !d_val))) {
        set_error_msg("mhdc_build_dia: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    mhdc_matrix *A = new mhdc_matrix();
    A->n = n;
    A->n_b = n_b;
    A->n_blocks = (n + n_b - 1) / n_b;
    A->theta = theta;
    A->dtype = dtype;
    A->mode = MHDC_MODE_BLOCK;
    cudaGetDevice(&A->device);
    int rc = build_dia_into(A, nd, d_offset, d_val, stream);
    if (rc != MHDC_OK) {
        cudaStreamSynchronize(stream);
        free_matrix(A);
        return rc;
    }
    *out = A;
    return MHDC_OK;
}

}  // namespace mhdc

namespace mhdc {

// ---------------------------------------------------------------------------
// Conversion without any device allocation (mhdc_build_noalloc).
//
// For callers that cannot allocate device memory while converting: a process
// whose device memory comes from a fixed pool handed out at start-up, code
// running where an allocation would stall or fail (a latency-critical loop,
// a memory-capped service), or a host language binding that only passes
// buffers it owns.  The caller passes the input CSR and every output array;
// all temporaries live in one file-scope device array of fixed size, which
// every GPU that loads this library keeps until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t NA_MAX_NNZ = 1 << 18;   // stored entries
constexpr int64_t NA_MAX_N = 1 << 18;     // rows (so at most 2^18 row blocks)
constexpr int64_t NA_SCAN = 2 * ((NA_MAX_NNZ + 4095) / 4096) + 8;  // scan tile sums, with room
// int32 words: err | sel_out | sel_cnt | ovf | ovf_pos | rem | rem_flag | scan | keys | cnt | ids | lg | base(i64)
constexpr int64_t NA_ERR = 0;
constexpr int64_t NA_SEL = 64;
constexpr int64_t NA_SELCNT = NA_SEL + NA_MAX_NNZ;
constexpr int64_t NA_OVF = NA_SELCNT + NA_MAX_N;
constexpr int64_t NA_OVFPOS = NA_OVF + NA_MAX_N;
constexpr int64_t NA_REM = NA_OVFPOS + NA_MAX_N + 64;
constexpr int64_t NA_RFLAG = NA_REM + NA_MAX_N + 64;  // one bit per entry
constexpr int64_t NA_SCANS = NA_RFLAG + NA_MAX_NNZ / 32 + 64;
constexpr int64_t NA_KEYS = NA_SCANS + NA_SCAN + 64;
constexpr int64_t NA_CNT = NA_KEYS + 4 * NA_MAX_NNZ;
// a block overflows its shared table only with more than 12288 entries, so at
// most NA_MAX_NNZ / 12288 < NA_MAX_OVF blocks take the global-table path
constexpr int64_t NA_MAX_OVF = 1024;
constexpr int64_t NA_IDS = NA_CNT + 4 * NA_MAX_NNZ;
constexpr int64_t NA_LG = NA_IDS + NA_MAX_OVF;
constexpr int64_t NA_BASE = NA_LG + NA_MAX_OVF;  // int64 entries start here (8-byte aligned)
constexpr int64_t NA_WORDS = NA_BASE + 2 * NA_MAX_OVF;

static __device__ __align__(256) int32_t g_noalloc_scratch[NA_WORDS];

// The device address of g_noalloc_scratch on the current device.  Host code
// cannot use the symbol itself as a pointer (in host code it names a host-side
// stand-in), so every call looks the address up with its device current:
// after a device reset the module, and with it the array, may sit elsewhere.
int noalloc_scratch(int32_t **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_error("cudaGetSymbolAddress(g_noalloc_scratch)", e);
        return MHDC_ERR_CUDA;
    }
    *out = static_cast<int32_t *>(p);
    return MHDC_OK;
}

// List the row blocks whose shared hash table overflowed: ids[pos[b]] = b,
// with the global table of block b at 4 * row_ptr[r0] (2^lg <= 4m slots).
__global__ void k_noalloc_ovf_list(int64_t n, int32_t n_b, int64_t nb, const int32_t *__restrict__ rp,
                                   const int32_t *__restrict__ ovf, const int32_t *__restrict__ pos,
                                   int32_t *ids, int32_t *lg, int64_t *base)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb || !ovf[b]) return;
    const int64_t r0 = b * (int64_t)n_b;
    const int64_t r1 = (n - r0 < n_b) ? n : r0 + n_b;
    const int64_t m = (int64_t)rp[r1] - rp[r0];
    int l = 10;
    while (((int64_t)1 << l) < 2 * m) l++;
    const int32_t q = pos[b];
    ids[q] = (int32_t)b;
    lg[q] = l;
    base[q] = 4 * (int64_t)rp[r0];
}

int read_i32(const int32_t *d, int32_t *h, cudaStream_t st)
{
    MHDC_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    return MHDC_OK;
}

template <typename VT>
int noalloc_fill(int64_t n, int32_t n_b, int64_t nb, int64_t nnz, const int32_t *rp,
                 const int32_t *col, const double *val, int32_t *S, int32_t *dia_ptr,
                 int32_t *dia_offset, void *dia_val, int32_t *csr_row_ptr, int32_t *csr_col,
                 void *csr_val, int64_t cap_rem, int64_t *h_nnz_rem, cudaStream_t st)
{
    int32_t *rem = S + NA_REM;  // per-row remainder counts (n <= NA_MAX_N words)
    uint32_t *flag = reinterpret_cast<uint32_t *>(S + NA_RFLAG);
    RC(launch_scatter<VT>(n, n_b, nb, nnz, rp, col, val, dia_ptr, S + NA_SEL, rp, dia_offset,
                          static_cast<VT *>(dia_val), rem, flag, st));
    RC(exclusive_scan_i32(rem, csr_row_ptr, n, S + NA_SCANS, st));
    int32_t nr = 0;
    RC(read_i32(csr_row_ptr + n, &nr, st));
    *h_nnz_rem = nr;
    if (nr > cap_rem) {
        set_error_msg("mhdc_build_noalloc: csr_col/csr_val capacity too small (needed size in *h_nnz_rem)");
        return MHDC_ERR_INVALID_ARG;
    }
    if (nr > 0)
        RC(launch_rem_fill<VT>(n, n_b, nb, rp, col, val, flag, csr_row_ptr, csr_col,
                               static_cast<VT *>(csr_val), st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    return MHDC_OK;
}

}  // namespace

int build_noalloc(int64_t n, const int32_t *rp, const int32_t *col, const double *val, int32_t n_b,
                  double theta, int32_t dtype, int32_t *dia_ptr, int32_t *dia_offset, void *dia_val,
                  int64_t cap_P, int32_t *csr_row_ptr, int32_t *csr_col, void *csr_val,
                  int64_t cap_rem, int64_t *h_P, int64_t *h_nnz_rem, cudaStream_t st)
{
    if (!rp || !h_P || !h_nnz_rem || n < 1 || n_b < 1 || !std::isfinite(theta) || theta < 0.0 ||
        dtype < MHDC_F64 || dtype > MHDC_BF16 || cap_P < 0 || cap_rem < 0 || !dia_ptr ||
        !csr_row_ptr) {
        set_error_msg("mhdc_build_noalloc: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    if (n > NA_MAX_N) {
        set_error_msg("mhdc_build_noalloc: n exceeds the no-allocation limit of 262144 rows");
        return MHDC_ERR_INVALID_ARG;
    }
    int32_t *S = nullptr;
    RC(noalloc_scratch(&S));
    int32_t nnz = 0;
    RC(read_i32(rp + n, &nnz, st));
    if (nnz < 0) {
        set_error_msg("mhdc_build_noalloc: row_ptr[n] < 0");
        return MHDC_ERR_BAD_CSR;
    }
    if (nnz > NA_MAX_NNZ) {
        set_error_msg("mhdc_build_noalloc: nnz exceeds the no-allocation limit of 262144 entries");
        return MHDC_ERR_INVALID_ARG;
    }
    if (nnz > 0 && (!col || !val)) {
        set_error_msg("mhdc_build_noalloc: null column or value array with nnz > 0");
        return MHDC_ERR_INVALID_ARG;
    }
    const int64_t nb = (n + n_b - 1) / n_b;
    // 1. CSR checks (the error word must start at zero: the array keeps old contents)
    MHDC_CUDA_TRY(cudaMemsetAsync(S + NA_ERR, 0, sizeof(int32_t), st));
    k_validate<<<grid_for(n, 256), 256, 0, st>>>(n, rp, col, nnz, S + NA_ERR);
    MHDC_LAUNCH_CHECK("k_validate");
    int32_t err = 0;
    RC(read_i32(S + NA_ERR, &err, st));
    if (err) {
        set_error_msg("mhdc_build_noalloc: invalid CSR");
        return MHDC_ERR_BAD_CSR;
    }
    // 2. selection per row block (shared-memory tables; overflowing blocks redone
    //    with tables in the scratch array)
    MHDC_CUDA_TRY(cudaFuncSetAttribute(k_count_select<false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)CS_SMEM_L2));
    k_count_select<false, true><<<(unsigned)nb, CS_THREADS, CS_SMEM_L2, st>>>(
        n, n_b, rp, col, theta, nullptr, HCAP, CW_L2, nullptr, nullptr, nullptr, nullptr,
        S + NA_SEL, S + NA_SELCNT, S + NA_OVF);
    MHDC_LAUNCH_CHECK("k_count_select");
    RC(exclusive_scan_i32(S + NA_OVF, S + NA_OVFPOS, nb, S + NA_SCANS, st));
    int32_t novf = 0;
    RC(read_i32(S + NA_OVFPOS + nb, &novf, st));
    if (novf > NA_MAX_OVF) {
        set_error_msg("mhdc_build_noalloc: too many overflowing row blocks");
        return MHDC_ERR_DEVICE_CHECK;
    }
    if (novf > 0) {
        int64_t *base = reinterpret_cast<int64_t *>(S + NA_BASE);
        k_noalloc_ovf_list<<<grid_for(nb, 256), 256, 0, st>>>(n, n_b, nb, rp, S + NA_OVF,
                                                              S + NA_OVFPOS, S + NA_IDS, S + NA_LG,
                                                              base);
        MHDC_LAUNCH_CHECK("k_noalloc_ovf_list");
        k_count_select<true, false><<<(unsigned)novf, CS_THREADS, 0, st>>>(
            n, n_b, rp, col, theta, S + NA_IDS, 0, 0, S + NA_KEYS, S + NA_CNT, base, S + NA_LG,
            S + NA_SEL, S + NA_SELCNT, S + NA_OVF);
        MHDC_LAUNCH_CHECK("k_count_select<global>");
        // a global table holds at least twice its block's entries and cannot
        // overflow; the flags are read back anyway, as mhdc_build does
        RC(exclusive_scan_i32(S + NA_OVF, S + NA_OVFPOS, nb, S + NA_SCANS, st));
        RC(read_i32(S + NA_OVFPOS + nb, &novf, st));
        if (novf != 0) {
            set_error_msg("k_count_select: global table overflow");
            return MHDC_ERR_DEVICE_CHECK;
        }
    }
    // 3. dia_ptr (caller's array) and the number of partial diagonals
    RC(exclusive_scan_i32(S + NA_SELCNT, dia_ptr, nb, S + NA_SCANS, st));
    int32_t P = 0;
    RC(read_i32(dia_ptr + nb, &P, st));
    *h_P = P;
    *h_nnz_rem = 0;
    if (P > cap_P) {
        set_error_msg("mhdc_build_noalloc: dia_offset/dia_val capacity too small (needed P in *h_P)");
        return MHDC_ERR_INVALID_ARG;
    }
    if (P > 0 && (!dia_offset || !dia_val)) {
        set_error_msg("mhdc_build_noalloc: null dia_offset or dia_val with P > 0");
        return MHDC_ERR_INVALID_ARG;
    }
    if (nnz > 0 && cap_rem > 0 && (!csr_col || !csr_val)) {
        set_error_msg("mhdc_build_noalloc: null csr_col or csr_val");
        return MHDC_ERR_INVALID_ARG;
    }
    // 4-5. scatter and remainder compaction
    switch (dtype) {
    case MHDC_F64:
        return noalloc_fill<double>(n, n_b, nb, nnz, rp, col, val, S, dia_ptr, dia_offset, dia_val,
                                    csr_row_ptr, csr_col, csr_val, cap_rem, h_nnz_rem, st);
    case MHDC_F32:
        return noalloc_fill<float>(n, n_b, nb, nnz, rp, col, val, S, dia_ptr, dia_offset, dia_val,
                                   csr_row_ptr, csr_col, csr_val, cap_rem, h_nnz_rem, st);
    default:
        return noalloc_fill<__nv_bfloat16>(n, n_b, nb, nnz, rp, col, val, S, dia_ptr, dia_offset,
                                           dia_val, csr_row_ptr, csr_col, csr_val, cap_rem,
                                           h_nnz_rem, st);
    }
}

}  // namespace mhdc
