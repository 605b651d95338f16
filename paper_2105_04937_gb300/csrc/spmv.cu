// y = A x kernels: M-HDC (Fig. 13), plain CSR (Fig. 2) and the memory
// benchmarks of Sec. 6.2 (Figs. 19-20).
//
// M-HDC work split: a warp owns a tile of RW consecutive rows inside one row
// block (RW = 32 lanes x V rows per 16-byte vector x U vectors per lane).
// For the tile it first adds the CSR remainder rows (skipped with two loads
// when the tile has none), then walks the block's diagonals: each lane loads
// 16 bytes of dia_val per diagonal (coalesced, 512 B per warp, no L1
// allocation since every value is read once) and the matching x values
// (L1/L2-cached: consecutive diagonals of a block hit the same x window), and
// accumulates in registers; y is written once.  One warp per tile, a grid
// of 8-warp CTAs covering every tile.
#include <cstring>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "dw_arith.cuh"
#include "mhdc_internal.cuh"

namespace mhdc {
namespace {

template <typename VT>
struct Tr;
template <>
struct Tr<double> {
    using X = double;
    using Y = double;
    using Acc = double;
    static constexpr int V = 2;
};
template <>
struct Tr<float> {
    using X = float;
    using Y = float;
    using Acc = float;
    static constexpr int V = 4;
};
template <>
struct Tr<__nv_bfloat16> {
    using X = __nv_bfloat16;
    using Y = float;
    using Acc = float;
    static constexpr int V = 8;
};

__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }

// 16-byte load of data read exactly once per product: bypass L1 allocation.
__device__ __forceinline__ uint4 ld_stream16(const void *p)
{
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p));
    return r;
}

template <typename T>
__device__ __forceinline__ T ldg_elem(const T *p)
{
    return __ldg(p);
}

constexpr int SPMV_THREADS = 256;
constexpr int SPMV_WARPS = SPMV_THREADS / 32;
// Resident CTAs per SM the register tiles are compiled for, i.e. their
// register budget (5 CTAs of 256 threads: 48 registers a thread, 4: 64, 2:
// 128).  The kernels wait on memory, so the small tiles keep 40 warps per SM
// (32 for BF16, whose 8 remainder rows per lane need more, and for tiles of
// 4 loads per group); the largest tiles need more registers for their loads
// in flight.
constexpr int spmv_min_blocks(int U, int D, int vsize)
{
    return U * D <= 2 ? (vsize == 2 ? 4 : 5) : U * D <= 4 ? (vsize == 2 && U > 1 ? 3 : 4) : 2;
}

// x[j .. j+V) into xv: one 16-byte load when j is 16-byte aligned, else V
// element loads (all in bounds: the caller checked 0 <= j, j + V <= n).
template <typename X, int V>
__device__ __forceinline__ void load_x(const X *__restrict__ x, int64_t j, bool aligned, X (&xv)[V])
{
    if constexpr (V * sizeof(X) == 16) {
        if (aligned) {
            const uint4 r = __ldg(reinterpret_cast<const uint4 *>(x + j));
            memcpy(xv, &r, 16);
            return;
        }
    }
#pragma unroll
    for (int m = 0; m < V; m++) xv[m] = ldg_elem(x + j + m);
}

// One warp = one tile of RW = 32 * V * U consecutive rows of one row block.
// The block's diagonals are taken D at a time: the D * U 16-byte value loads
// of a group are issued first, then the x loads, then the FMAs, so a warp
// keeps D * U * 512 bytes of dia_val in flight.
//
// CK (mhdc_set_checked): every index into the handle's arrays, x and y is
// compared with the array's extent first; a failed check skips the access
// (0 is used) and marks the status word.  The operations are otherwise those
// of the unchecked tile, so an in-bounds product gives the same y.
template <typename VT, int U, int D, bool VEC, bool PF = false, bool CK = false>
__device__ __forceinline__ void
reg_tile(int64_t w, int64_t n, int32_t n_b, int32_t tpb, const int32_t *__restrict__ dia_ptr,
         const int32_t *__restrict__ dia_offset, const VT *__restrict__ dia_val,
         const int32_t *__restrict__ csr_row_ptr, const int32_t *__restrict__ csr_col,
         const VT *__restrict__ csr_val, const typename Tr<VT>::X *__restrict__ x,
         typename Tr<VT>::Y *__restrict__ y, BoundsCheck ck = BoundsCheck{})
{
    using Acc = typename Tr<VT>::Acc;
    using X = typename Tr<VT>::X;
    constexpr int V = VEC ? Tr<VT>::V : 1;
    constexpr int RW = 32 * V * U;
    const int lane = threadIdx.x & 31;
    const int64_t ib = w / tpb;
    const int32_t tw = (int32_t)(w - ib * tpb) * RW;
    const int64_t r0 = ib * (int64_t)n_b;
    const int32_t rows = (int32_t)((n - r0 < n_b) ? (n - r0) : n_b);
    if (tw >= rows) return;  // warp-uniform
    const bool full = tw + RW <= rows;
    const bool x_al = (reinterpret_cast<uintptr_t>(x) & 15) == 0;

    int32_t tl[U];
#pragma unroll
    for (int u = 0; u < U; u++) tl[u] = tw + (u * 32 + lane) * V;

    // the block's diagonal range, loaded with the remainder bounds below (independent)
    int32_t p0 = 0, p1 = 0;
    if constexpr (CK) {
        if (ck_in(ck, ib, ib + 2, ck.n_blocks + 1)) {
            p0 = dia_ptr[ib];
            p1 = dia_ptr[ib + 1];
            if (!ck_in(ck, p0, p1, ck.P)) p0 = p1 = 0;
        }
    } else {
        p0 = dia_ptr[ib];
        p1 = dia_ptr[ib + 1];
    }
    if constexpr (VEC && PF) {
        // every diagonal's values of this tile into L2 ahead of their loads:
        // one bulk prefetch per diagonal (lane d takes diagonal p0 + d), the
        // tile's slice clipped to the block's n_b slots (16-byte multiples).
        // Used by the batched kernel, whose warps walk several tiles in turn;
        // it slowed the one-tile-per-warp grid down.
        const int32_t nv = (n_b - tw < RW) ? n_b - tw : RW;
        const uint32_t bytes = (uint32_t)(nv * (int32_t)sizeof(VT));
        for (int32_t q = p0 + lane; q < p1; q += 32) {
            const VT *src = dia_val + (int64_t)q * n_b + tw;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes)
                         : "memory");
        }
    }

    Acc acc[U][V];
#pragma unroll
    for (int u = 0; u < U; u++)
#pragma unroll
        for (int m = 0; m < V; m++) acc[u][m] = Acc(0);

    // CSR remainder rows of the tile (Fig. 13, first loop), summed by
    // rem_rows_add: every row from zero in column order, with the next
    // entries of all the lane's rows loaded together.  With V >= 4 rows per
    // lane (FP32, BF16) each lane instead sums whole rows tw + rr (rr = lane,
    // lane + 32, ..., coalesced row bounds), and the sums reach their owners
    // through shared memory: the same operations as summing into acc
    // directly.
    {
        const int32_t tend = full ? tw + RW : rows;
        if constexpr (CK) {
            if (!ck_in(ck, r0 + tw, r0 + tend + 1, n + 1)) return;
        }
        const int32_t q0 = csr_row_ptr[r0 + tw], q1 = csr_row_ptr[r0 + tend];
        if (q0 != q1 && CK) {
            // checked: each lane sums its own rows (tl[u] + m) row by row
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int m = 0; m < V; m++) {
                    const int32_t t = tl[u] + m;
                    if (t < rows)
                        rem_row_add_ck(acc[u][m], csr_row_ptr[r0 + t], csr_row_ptr[r0 + t + 1],
                                       csr_col, csr_val, x, n, ck);
                }
        } else if (q0 != q1 && V < 4) {
            // V rows per vector (FP64: 2), U vectors per lane
            constexpr int R = U * V;
            Acc s[R];
            int32_t a[R], b[R];
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int m = 0; m < V; m++) {
                    const int32_t t = tl[u] + m;
                    s[u * V + m] = Acc(0);
                    a[u * V + m] = t < rows ? csr_row_ptr[r0 + t] : 0;
                    b[u * V + m] = t < rows ? csr_row_ptr[r0 + t + 1] : 0;
                }
            rem_rows_add<R, 1>(s, a, b, csr_col, csr_val, x);
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int m = 0; m < V; m++) acc[u][m] = s[u * V + m];
        } else if (q0 != q1) {
            constexpr int R = RW / 32;
            __shared__ Acc rsum[SPMV_WARPS][RW];
            Acc *rs = rsum[threadIdx.x >> 5];
            Acc s[R];
            int32_t a[R], b[R];
#pragma unroll
            for (int j = 0; j < R; j++) {
                const int32_t t = tw + lane + 32 * j;
                s[j] = Acc(0);
                a[j] = t < rows ? csr_row_ptr[r0 + t] : 0;
                b[j] = t < rows ? csr_row_ptr[r0 + t + 1] : 0;
            }
            if constexpr (sizeof(VT) == 2) {
                // BF16: the tile's remainder entries are gathered by the whole
                // warp, RSG per lane at a time (columns and values coalesced,
                // then the x gathers), into shared memory as (value, x) FP32
                // pairs; each lane then runs its rows' FMA chains from there
                // in column order.  The same operations as rem_rows_add
                // without its registers for 8 rows of loads per lane.
                constexpr int RSG = 4;
                constexpr int CAP = 32 * RSG;
                __shared__ float2 rst[SPMV_WARPS][CAP];
                float2 *st = rst[threadIdx.x >> 5];
                bool lng[R];
#pragma unroll
                for (int j = 0; j < R; j++) lng[j] = sizeof(Acc) < sizeof(double) && b[j] - a[j] > REM_LONG;
                for (int32_t c0 = q0; c0 < q1; c0 += CAP) {
                    const int32_t c1 = (q1 - c0 < CAP) ? q1 : c0 + CAP;
                    int32_t cc[RSG];
                    VT vv[RSG];
                    X xx[RSG];
#pragma unroll
                    for (int m = 0; m < RSG; m++) {
                        const int32_t e = c0 + lane + 32 * m;
                        cc[m] = e < c1 ? csr_col[e] : 0;
                        vv[m] = e < c1 ? csr_val[e] : VT(0);
                    }
#pragma unroll
                    for (int m = 0; m < RSG; m++)
                        xx[m] = c0 + lane + 32 * m < c1 ? __ldg(x + cc[m]) : X(0);
#pragma unroll
                    for (int m = 0; m < RSG; m++)
                        if (c0 + lane + 32 * m < c1)
                            st[lane + 32 * m] = make_float2(rem_in(vv[m]), rem_in(xx[m]));
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < R; j++) {
                        if (lng[j]) continue;
                        const int32_t k0 = a[j] > c0 ? a[j] : c0, k1 = b[j] < c1 ? b[j] : c1;
                        for (int32_t k = k0; k < k1; k++) {
                            const float2 pv = st[k - c0];
                            s[j] = rem_fma(pv.x, pv.y, s[j]);
                        }
                    }
                    __syncwarp();
                }
#pragma unroll
                for (int j = 0; j < R; j++)
                    if (lng[j]) rem_row_add(s[j], a[j], b[j], csr_col, csr_val, x);
            } else {
                rem_rows_add<R, 1>(s, a, b, csr_col, csr_val, x);
            }
#pragma unroll
            for (int j = 0; j < R; j++) rs[lane + 32 * j] = s[j];
            __syncwarp();
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int m = 0; m < V; m++) acc[u][m] = rs[tl[u] - tw + m];
            __syncwarp();
        }
    }

    // the block's partial diagonals (Fig. 13, second loop)
    const int64_t xrow0 = r0 + tw;  // x index of the tile's first row at offset 0
    int32_t p = p0;
    auto group = [&](auto Dc, auto Fc) {
        constexpr int DD = decltype(Dc)::value;
        constexpr bool FAST = decltype(Fc)::value;
        int64_t off[DD];
#pragma unroll
        for (int d = 0; d < DD; d++) off[d] = dia_offset[p + d];
        VT v[DD][U][V];
#pragma unroll
        for (int d = 0; d < DD; d++) {
            const VT *vp = dia_val + (int64_t)(p + d) * n_b;
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t vi = (int64_t)(p + d) * n_b + tl[u];
                if ((full || tl[u] < rows) && (!CK || ck_in(ck, vi, vi + V, ck.dia_slots))) {
                    if constexpr (VEC) {
                        const uint4 r = ld_stream16(vp + tl[u]);
                        memcpy(v[d][u], &r, 16);
                    } else {
                        v[d][u][0] = vp[tl[u]];
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < V; m++) v[d][u][m] = VT(0);
                }
            }
        }
        X xv[DD][U][V];
#pragma unroll
        for (int d = 0; d < DD; d++) {
            const int64_t jw = xrow0 + off[d];
            const int64_t r = ((jw % V) + V) % V;  // warp-uniform misalignment in elements
            // warp-uniform: the whole tile reads x inside [0, n)
            if (FAST || (full && jw >= 0 && jw + RW <= n)) {
                if constexpr (VEC && V * sizeof(X) == 16 && V > 2) {
                    if (x_al && r != 0 && (FAST || jw - r + RW + V <= n)) {
                        // two aligned 16-byte loads and a byte shift per vector
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            const int64_t ja = (jw - r) + (tl[u] - tw);
                            if (CK && !ck_in(ck, ja, ja + 2 * V, n)) {
#pragma unroll
                                for (int m = 0; m < V; m++) xv[d][u][m] = X(0);
                                continue;
                            }
                            const X *a = x + ja;
                            const uint4 lo = __ldg(reinterpret_cast<const uint4 *>(a));
                            const uint4 hi = __ldg(reinterpret_cast<const uint4 *>(a + V));
                            const uint4 q = window16(lo, hi, (int)(r * sizeof(X)));
                            memcpy(xv[d][u], &q, 16);
                        }
                        continue;
                    }
                }
                const bool al = x_al && r == 0;
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int64_t j0 = jw + (tl[u] - tw);
                    if (CK && !ck_in(ck, j0, j0 + V, n)) {
#pragma unroll
                        for (int m = 0; m < V; m++) xv[d][u][m] = X(0);
                        continue;
                    }
                    load_x<X, V>(x, j0, al, xv[d][u]);
                }
            } else {
#pragma unroll
                for (int u = 0; u < U; u++)
#pragma unroll
                    for (int m = 0; m < V; m++) {
                        const int64_t jm = jw + (tl[u] - tw) + m;
                        xv[d][u][m] = (tl[u] + m < rows && jm >= 0 && jm < n) ? ldg_elem(x + jm)
                                                                              : X(0);
                    }
            }
        }
#pragma unroll
        for (int d = 0; d < DD; d++)
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int m = 0; m < V; m++) acc[u][m] += widen(v[d][u][m]) * widen(xv[d][u][m]);
        p += DD;
    };
    // Offsets ascend inside a block, so when the first and the last diagonal
    // keep the whole tile's x window (plus one vector for the shifted loads)
    // inside [0, n), every diagonal does and the groups skip their x checks.
    bool all_in = !CK && full && p1 > p0;
    if (all_in) all_in = xrow0 + dia_offset[p0] >= 0 && xrow0 + dia_offset[p1 - 1] + RW + V <= n;
    if (all_in) {
        for (; p + D <= p1;) group(std::integral_constant<int, D>{}, std::true_type{});
        for (; p < p1;) group(std::integral_constant<int, 1>{}, std::true_type{});
    } else {
        for (; p + D <= p1;) group(std::integral_constant<int, D>{}, std::false_type{});
        for (; p < p1;) group(std::integral_constant<int, 1>{}, std::false_type{});
    }

#pragma unroll
    for (int u = 0; u < U; u++) {
#pragma unroll
        for (int m = 0; m < V; m++)
            if (tl[u] + m < rows && (!CK || ck_in(ck, r0 + tl[u] + m, r0 + tl[u] + m + 1, n)))
                y[r0 + tl[u] + m] = acc[u][m];
    }
}

// Persistent tile scheduling (the DYN kernels): the grid holds only resident
// CTAs; each warp takes its own tile first, then the next free tile from
// sched[0] until none is left, so that tiles of uneven cost (a heavy CSR
// remainder) spread evenly; the last CTA to finish clears both counters for
// the next launch.  One call site of the tile body keeps the registers of
// the one-tile-per-warp kernels unchanged.
template <typename F>
__device__ __forceinline__ void tile_loop_dyn(int64_t n_tiles, unsigned long long *sched, F &&tile)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
         w < n_tiles;) {  // warp-uniform
        tile(w);
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&sched[0], 1ull);
        w = nw + (int64_t)__shfl_sync(0xffffffffu, t, 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&sched[1], 1ull) == (unsigned long long)gridDim.x - 1) {
            sched[0] = 0;
            sched[1] = 0;
            __threadfence();
        }
    }
}

template <typename VT, int U, int D, bool VEC, bool DYN = false>
__global__ void __launch_bounds__(SPMV_THREADS, spmv_min_blocks(U, D, sizeof(VT)))
k_mhdc_spmv(int64_t n, int32_t n_b, int32_t tpb, int64_t n_tiles,
            const int32_t *__restrict__ dia_ptr, const int32_t *__restrict__ dia_offset,
            const VT *__restrict__ dia_val, const int32_t *__restrict__ csr_row_ptr,
            const int32_t *__restrict__ csr_col, const VT *__restrict__ csr_val,
            const typename Tr<VT>::X *__restrict__ x, typename Tr<VT>::Y *__restrict__ y,
            unsigned long long *__restrict__ sched)
{
    if constexpr (DYN) {
        tile_loop_dyn(n_tiles, sched, [&](int64_t w) {
            reg_tile<VT, U, D, VEC>(w, n, n_b, tpb, dia_ptr, dia_offset, dia_val, csr_row_ptr,
                                    csr_col, csr_val, x, y);
        });
    } else {  // one tile a warp; sched unused
        const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (w >= n_tiles) return;
        reg_tile<VT, U, D, VEC>(w, n, n_b, tpb, dia_ptr, dia_offset, dia_val, csr_row_ptr,
                                csr_col, csr_val, x, y);
    }
}

// The bounds-checked product of mhdc_set_checked: the default tile shapes
// (U = 1; D = 2 with 16-byte vectors, D = 4 without), every access checked.
template <typename VT, bool VEC>
__global__ void __launch_bounds__(SPMV_THREADS)
k_mhdc_spmv_ck(int64_t n, int32_t n_b, int32_t tpb, int64_t n_tiles,
               const int32_t *__restrict__ dia_ptr, const int32_t *__restrict__ dia_offset,
               const VT *__restrict__ dia_val, const int32_t *__restrict__ csr_row_ptr,
               const int32_t *__restrict__ csr_col, const VT *__restrict__ csr_val,
               const typename Tr<VT>::X *__restrict__ x, typename Tr<VT>::Y *__restrict__ y,
               BoundsCheck ck)
{
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= n_tiles) return;
    reg_tile<VT, 1, VEC ? 2 : 4, VEC, false, true>(w, n, n_b, tpb, dia_ptr, dia_offset, dia_val,
                                                   csr_row_ptr, csr_col, csr_val, x, y, ck);
}

// ---------------------------------------------------------------------------
// Emulated FP64 product (variants 10-12 of FP64 handles).
//
// GB300 runs FP64 FMAs about 64x slower than FP32 ones, which makes the
// native FP64 M-HDC product bound by the FP64 pipe, not by HBM.  Here every
// value a and x_j is a pair of FP32 numbers (hi, lo) with hi + lo = a to about
// 2^-48 relative error (the split of the values is done once at build, that
// of x by k_split_x with integer operations only), and each row accumulates
//   s += a * x
// as an FP32 pair (dw::dw_fma): the high product enters the high word by
// TwoSum, and the product's exact error, the two cross products and the
// TwoSum error are added into the low word, renormalised by Fast2Sum (15 FP32
// operations a term).  Error per row of k terms, every nonzero |a|, |x| in
// [2^-45, 2^60] and k <= 48: at most (5.2 k + 18) * 2^-48 * sum_j |a_ij x_j|
// including the final rounding to FP64, i.e. below 9.6e-13 (the derivation
// is in dw_arith.cuh).
// A row that reads an x outside the window comes out NaN (the split marks
// such an x) and is recomputed with native FP64 arithmetic (native_row).
// ---------------------------------------------------------------------------
// x_dw[i] = FP32 pair of x[i] (integer operations only): hi = x rounded to 24
// significant bits (half-up on the magnitude), lo = x - hi (exact, at most 29
// bits) rounded to FP32.  Any nonzero |x| outside [2^DW_EMIN, 2^DW_EMAX] or
// non-finite becomes the pair (NaN, 0): every emulated sum that uses it is
// NaN (in-window terms cannot overflow FP32, so nothing else is), and the
// product recomputes exactly those rows natively.
// RN(d) for |d| < 2^29 on the FP32 pipe: d = dh 2^15 + dl with dl in
// [0, 2^15) and |dh| < 2^14, each half exact in FP32 by the magic-number
// construction (1.5 * 2^23 + dh, 2^23 + dl), and one FMA rounds the exact sum
// once.  (On GB300 the int-to-float conversion shares the slow FP64 pipe.)
__device__ __forceinline__ float i29_to_float_rn(int32_t d)
{
    const int32_t dh = d >> 15;  // floor(d / 2^15)
    const int32_t dl = d & 0x7FFF;
    const float fh = __fsub_rn(__int_as_float(0x4B400000 + dh), 12582912.0f);
    const float fl = __fsub_rn(__int_as_float(0x4B000000 + dl), 8388608.0f);
    return __fmaf_rn(fh, 32768.0f, fl);
}

__device__ __forceinline__ bool split_dw(double xd, float2 &o)
{
    // the two 32-bit halves of x: sign, 11 exponent bits and the top 20
    // fraction bits in hw; the low 32 fraction bits in lw
    const uint32_t hw = (uint32_t)__double2hiint(xd), lw = (uint32_t)__double2loint(xd);
    const uint32_t sign = hw & 0x80000000u;
    const uint32_t mh = hw & 0x7FFFFFFFu;
    o = make_float2(0.f, 0.f);
    if ((mh | lw) == 0) return true;
    const int E = (int)(mh >> 20) - 1023;
    if (E < DW_EMIN || E >= DW_EMAX) {  // also inf / nan (E = 1024) and subnormals
        o = make_float2(__int_as_float(0x7FC00000), 0.f);
        return false;
    }
    // magnitude rounded half-up at bit 29 (24 significant bits), low bits cleared
    const uint32_t lr = lw + (1u << 28);
    const uint32_t mhr = mh + (lr < lw ? 1u : 0u);
    const uint32_t lrc = lr & ~((1u << 29) - 1u);
    const int Er = (int)(mhr >> 20) - 1023;
    const uint32_t hb = sign | ((uint32_t)(Er + 127) << 23) | (((mhr << 3) | (lrc >> 29)) & 0x7FFFFFu);
    // x - hi in units of ulp(x): |d| < 2^29, so the low words' difference is exact
    const int32_t d = (int32_t)(lw - lrc);
    float lo = __fmul_rn(i29_to_float_rn(d), __uint_as_float((uint32_t)(E - 52 + 127) << 23));
    if (sign) lo = -lo;
    o = make_float2(__uint_as_float(hb), lo);
    return true;
}

// Pairs of elements (one 16-byte load of x where x is 16-byte aligned, one
// 16-byte store into x_dw), consecutive threads on consecutive pairs.  The
// product launched after it may start its CTAs at once
// (griddepcontrol.launch_dependents); they wait for this grid's completion
// and memory before reading x_dw.
constexpr int SPLIT_THREADS = 256;

constexpr int SPLIT_EPT = 4;  // elements a thread, in pairs (2 and 8 measured slower)

__global__ void __launch_bounds__(SPLIT_THREADS)
k_split_x(int64_t n, const double *__restrict__ x, float2 *__restrict__ x_dw)
{
    asm volatile("griddepcontrol.launch_dependents;");
    // launched as a programmatic dependent of the stream's previous kernel:
    // x (possibly that kernel's output) and x_dw (read by the previous
    // product of this handle) are free after this wait
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t base = (int64_t)blockIdx.x * SPLIT_THREADS * SPLIT_EPT;
    const bool al = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
#pragma unroll
    for (int q = 0; q < SPLIT_EPT / 2; q++) {
        // pair q of the thread: consecutive threads take consecutive pairs
        const int64_t i = base + 2 * ((int64_t)q * SPLIT_THREADS + threadIdx.x);
        if (i >= n) break;
        const bool two = i + 1 < n;
        double a, b = 0.0;
        if (two && al) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(x + i));
            a = v.x;
            b = v.y;
        } else {
            a = __ldg(x + i);
            if (two) b = __ldg(x + i + 1);
        }
        float2 o0, o1;
        split_dw(a, o0);
        if (two) {
            split_dw(b, o1);
            *reinterpret_cast<float4 *>(x_dw + i) = make_float4(o0.x, o0.y, o1.x, o1.y);
        } else {
            x_dw[i] = o0;
        }
    }
}

inline unsigned split_grid(int64_t n)
{
    const int64_t per = (int64_t)SPLIT_THREADS * SPLIT_EPT;
    return (unsigned)((n + per - 1) / per);
}

// One warp tile of the emulated product: the rows and tile geometry of
// reg_tile<double, U, D, true> (RW = 64 U rows), FP32-pair arithmetic.
template <int U, int D>
__device__ __forceinline__ void
dw_tile(int64_t w, int64_t n, int32_t n_b, int32_t tpb, const int32_t *__restrict__ dia_ptr,
        const int32_t *__restrict__ dia_offset, const float2 *__restrict__ dia_dw,
        const int32_t *__restrict__ csr_row_ptr, const int32_t *__restrict__ csr_col,
        const float2 *__restrict__ csr_dw, const float2 *__restrict__ x_dw,
        const double *__restrict__ dia_val, const double *__restrict__ csr_val,
        const double *__restrict__ x, double *__restrict__ y)
{
    constexpr int V = 2;  // float2 slots per 16-byte load
    constexpr int RW = 32 * V * U;
    const int lane = threadIdx.x & 31;
    const int64_t ib = w / tpb;
    const int32_t tw = (int32_t)(w - ib * tpb) * RW;
    const int64_t r0 = ib * (int64_t)n_b;
    const int32_t rows = (int32_t)((n - r0 < n_b) ? (n - r0) : n_b);
    if (tw >= rows) return;
    const bool full = tw + RW <= rows;
    int32_t tl[U];
#pragma unroll
    for (int u = 0; u < U; u++) tl[u] = tw + (u * 32 + lane) * V;
    float sh[U][V], sl[U][V];
#pragma unroll
    for (int u = 0; u < U; u++)
#pragma unroll
        for (int m = 0; m < V; m++) sh[u][m] = sl[u][m] = 0.f;
    const int32_t p0 = dia_ptr[ib], p1 = dia_ptr[ib + 1];

    {
        const int32_t tend = full ? tw + RW : rows;
        if (csr_row_ptr[r0 + tw] != csr_row_ptr[r0 + tend]) {
            // the lane's rows, each in column order; every round loads the
            // next entry of every row (values, then the gathers of x) before
            // its steps, so the rows' loads are in flight together
            constexpr int R = U * V;
            int32_t a[R], b[R];
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int m = 0; m < V; m++) {
                    const int32_t t = tl[u] + m;
                    a[u * V + m] = t < rows ? csr_row_ptr[r0 + t] : 0;
                    b[u * V + m] = t < rows ? csr_row_ptr[r0 + t + 1] : 0;
                }
            for (;;) {
                bool more = false;
#pragma unroll
                for (int r = 0; r < R; r++) more |= a[r] < b[r];
                if (!more) break;
                float2 av[R], xv[R];
                int32_t c[R];
#pragma unroll
                for (int r = 0; r < R; r++) {
                    c[r] = a[r] < b[r] ? __ldg(csr_col + a[r]) : 0;
                    av[r] = a[r] < b[r] ? __ldg(csr_dw + a[r]) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int r = 0; r < R; r++) xv[r] = a[r] < b[r] ? __ldg(x_dw + c[r]) : make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < R; r++)
                    if (a[r] < b[r]) {
                        dw::dw_fma(sh[r / V][r % V], sl[r / V][r % V], av[r], xv[r]);
                        a[r]++;
                    }
            }
        }
    }

    const int64_t xrow0 = r0 + tw;
    int32_t p = p0;
    auto group = [&](auto Dc, auto Fc) {
        constexpr int DD = decltype(Dc)::value;
        constexpr bool FAST = decltype(Fc)::value;
        int64_t off[DD];
#pragma unroll
        for (int d = 0; d < DD; d++) off[d] = dia_offset[p + d];
        float2 v[DD][U][V];
#pragma unroll
        for (int d = 0; d < DD; d++) {
            const float2 *vp = dia_dw + (int64_t)(p + d) * n_b;
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (FAST || full || tl[u] < rows) {
                    const uint4 r = ld_stream16(vp + tl[u]);
                    memcpy(v[d][u], &r, 16);
                } else {
                    v[d][u][0] = v[d][u][1] = make_float2(0.f, 0.f);
                }
            }
        }
        float2 xv[DD][U][V];
#pragma unroll
        for (int d = 0; d < DD; d++) {
            const int64_t jw = xrow0 + off[d];
            if (FAST || (full && jw >= 0 && jw + RW <= n)) {
                const bool al = (jw & 1) == 0;
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int64_t j = jw + (tl[u] - tw);
                    if (al) {
                        const uint4 r = __ldg(reinterpret_cast<const uint4 *>(x_dw + j));
                        memcpy(xv[d][u], &r, 16);
                    } else {
                        xv[d][u][0] = __ldg(x_dw + j);
                        xv[d][u][1] = __ldg(x_dw + j + 1);
                    }
                }
            } else {
#pragma unroll
                for (int u = 0; u < U; u++)
#pragma unroll
                    for (int m = 0; m < V; m++) {
                        const int64_t jm = jw + (tl[u] - tw) + m;
                        xv[d][u][m] = (tl[u] + m < rows && jm >= 0 && jm < n)
                                          ? __ldg(x_dw + jm)
                                          : make_float2(0.f, 0.f);
                    }
            }
        }
#pragma unroll
        for (int d = 0; d < DD; d++)
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int m = 0; m < V; m++) dw::dw_fma(sh[u][m], sl[u][m], v[d][u][m], xv[d][u][m]);
        p += DD;
    };
    // ascending offsets: the first and last diagonal bound every x window
    bool all_in = full && p1 > p0;
    if (all_in) all_in = xrow0 + dia_offset[p0] >= 0 && xrow0 + dia_offset[p1 - 1] + RW <= n;
    if (all_in) {
        for (; p + D <= p1;) group(std::integral_constant<int, D>{}, std::true_type{});
        for (; p < p1;) group(std::integral_constant<int, 1>{}, std::true_type{});
    } else {
        for (; p + D <= p1;) group(std::integral_constant<int, D>{}, std::false_type{});
        for (; p < p1;) group(std::integral_constant<int, 1>{}, std::false_type{});
    }

#pragma unroll
    for (int u = 0; u < U; u++)
#pragma unroll
        for (int m = 0; m < V; m++)
            if (tl[u] + m < rows) {
                const int32_t t = tl[u] + m;
                y[r0 + t] = isnan(sh[u][m])  // read an x outside the window
                                ? native_row(r0 + t, t, ib, n, n_b, dia_ptr, dia_offset, dia_val,
                                             csr_row_ptr, csr_col, csr_val, x)
                                : dw::f32_to_f64(sh[u][m]) + dw::f32_to_f64(sl[u][m]);
            }
}

template <int U, int D, bool DYN = false>
__global__ void __launch_bounds__(SPMV_THREADS, U * D <= 2 ? 5 : 4)
k_mhdc_spmv_dw(int64_t n, int32_t n_b, int32_t tpb, int64_t n_tiles,
               const int32_t *__restrict__ dia_ptr, const int32_t *__restrict__ dia_offset,
               const float2 *__restrict__ dia_dw, const int32_t *__restrict__ csr_row_ptr,
               const int32_t *__restrict__ csr_col, const float2 *__restrict__ csr_dw,
               const float2 *__restrict__ x_dw, const double *__restrict__ dia_val,
               const double *__restrict__ csr_val, const double *__restrict__ x,
               double *__restrict__ y, unsigned long long *__restrict__ sched)
{
    asm volatile("griddepcontrol.launch_dependents;");
    // launched as a programmatic dependent of k_split_x: its x_dw is complete
    // and visible after this wait (a no-op for a plain launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if constexpr (DYN) {
        tile_loop_dyn(n_tiles, sched, [&](int64_t w) {
            dw_tile<U, D>(w, n, n_b, tpb, dia_ptr, dia_offset, dia_dw, csr_row_ptr, csr_col,
                          csr_dw, x_dw, dia_val, csr_val, x, y);
        });
    } else {  // one tile a warp; sched unused
        const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (w >= n_tiles) return;
        dw_tile<U, D>(w, n, n_b, tpb, dia_ptr, dia_offset, dia_dw, csr_row_ptr, csr_col, csr_dw,
                      x_dw, dia_val, csr_val, x, y);
    }
}


// Plain CSR (Fig. 2), one thread per row: s = fma(val[k], x[col_ind[k]], s)
// over the row, four entries per step.  One FP64 FMA per nonzero and no
// cross-lane reduction: on GB300 the FP64 pipe (about 0.6 T FMA/s) rather
// than HBM bounds an FP64 SpMV, so the baseline must not spend extra FP64
// adds.  A warp's 32 rows are contiguous in val / col_ind, so the per-thread
// strided loads are served from L1 lines the warp already fetched.
constexpr int CSR_THREADS = 256;

__global__ void __launch_bounds__(CSR_THREADS)
k_csr_spmv(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
           const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * CSR_THREADS + threadIdx.x;
    if (i >= n) return;
    const int32_t a = rp[i], b = rp[i + 1];
    double s = 0.0;
    int32_t k = a;
    for (; k + 4 <= b; k += 4) {
        const double v0 = __ldg(val + k), v1 = __ldg(val + k + 1), v2 = __ldg(val + k + 2),
                     v3 = __ldg(val + k + 3);
        const int32_t c0 = __ldg(col + k), c1 = __ldg(col + k + 1), c2 = __ldg(col + k + 2),
                      c3 = __ldg(col + k + 3);
        const double x0 = __ldg(x + c0), x1 = __ldg(x + c1), x2 = __ldg(x + c2), x3 = __ldg(x + c3);
        s = fma(v0, x0, s);
        s = fma(v1, x1, s);
        s = fma(v2, x2, s);
        s = fma(v3, x3, s);
    }
    for (; k < b; k++) s = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), s);
    y[i] = s;
}

// Unblocked DIA order (Fig. 5) on a handle built with global selection, where
// every row block holds the same D diagonals (dia_ptr[ib] = ib * D): the
// remainder rows initialise y (the "y = 0" pass plus the remainder's CSR
// terms, in column order), then each diagonal is one pass over all n rows,
// y[i] += dia_val * x[i + off], so y is read and written once per diagonal.
// The operations of each row are those of the blocked kernel in the same
// order, so both give bit-identical y.
constexpr int DIA_THREADS = 256;

template <typename VT>
__global__ void __launch_bounds__(DIA_THREADS)
k_dia_rem(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
          const VT *__restrict__ val, const typename Tr<VT>::X *__restrict__ x,
          typename Tr<VT>::Y *__restrict__ y)
{
    using Acc = typename Tr<VT>::Acc;
    const int64_t i = (int64_t)blockIdx.x * DIA_THREADS + threadIdx.x;
    if (i >= n) return;
    Acc s = Acc(0);
    rem_row_add(s, rp[i], rp[i + 1], col, val, x);
    y[i] = s;
}

// Pass of diagonal k: thread g owns rows [g V, g V + V), all inside one row
// block (n_b % V == 0 when VEC), and reads their V values with one 16-byte
// load; rows whose column falls outside [0, n) add 0 * 0 as the blocked
// kernel does.
template <typename VT, bool VEC>
__global__ void __launch_bounds__(DIA_THREADS)
k_dia_pass(int64_t n, int32_t n_b, int32_t D, int32_t k, const int32_t *__restrict__ dia_offset,
           const VT *__restrict__ dia_val, const typename Tr<VT>::X *__restrict__ x,
           typename Tr<VT>::Y *__restrict__ y)
{
    using X = typename Tr<VT>::X;
    constexpr int V = VEC ? Tr<VT>::V : 1;
    const int64_t i0 = ((int64_t)blockIdx.x * DIA_THREADS + threadIdx.x) * V;
    if (i0 >= n) return;
    const int64_t ib = i0 / n_b;
    const int64_t t = i0 - ib * n_b;
    const VT *vp = dia_val + (ib * D + k) * (int64_t)n_b + t;
    VT v[V];
    if constexpr (VEC) {
        const uint4 r = ld_stream16(vp);
        memcpy(v, &r, 16);
    } else {
        v[0] = vp[0];
    }
    const int64_t off = dia_offset[k];
#pragma unroll
    for (int m = 0; m < V; m++) {
        const int64_t i = i0 + m;
        if (i < n) {
            const int64_t j = i + off;
            const X xv = (j >= 0 && j < n) ? ldg_elem(x + j) : X(0);
            y[i] = y[i] + widen(v[m]) * widen(xv);
        }
    }
}

template <typename VT>
int dia_typed(const mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t st)
{
    using X = typename Tr<VT>::X;
    using Y = typename Tr<VT>::Y;
    const X *x = static_cast<const X *>(d_x);
    Y *y = static_cast<Y *>(d_y);
    const int64_t n = A->n;
    k_dia_rem<VT><<<(unsigned)((n + DIA_THREADS - 1) / DIA_THREADS), DIA_THREADS, 0, st>>>(
        n, A->csr_row_ptr, A->csr_col, static_cast<const VT *>(A->csr_val), x, y);
    MHDC_LAUNCH_CHECK("k_dia_rem");
    const int32_t D = (int32_t)(A->P / A->n_blocks);
    constexpr int VV = Tr<VT>::V;
    const bool vec = (A->n_b % VV) == 0;
    const int64_t groups = vec ? (n + VV - 1) / VV : n;
    const unsigned grid = (unsigned)((groups + DIA_THREADS - 1) / DIA_THREADS);
    for (int32_t k = 0; k < D; k++) {
        if (vec)
            k_dia_pass<VT, true><<<grid, DIA_THREADS, 0, st>>>(
                n, A->n_b, D, k, A->dia_offset, static_cast<const VT *>(A->dia_val), x, y);
        else
            k_dia_pass<VT, false><<<grid, DIA_THREADS, 0, st>>>(
                n, A->n_b, D, k, A->dia_offset, static_cast<const VT *>(A->dia_val), x, y);
        MHDC_LAUNCH_CHECK("k_dia_pass");
    }
    return MHDC_OK;
}

// Read-only member of the memory benchmarks: out[cta] = bitwise XOR of the
// 64-bit words of the CTA's share of A (16-byte loads, 4 in flight per
// thread).  Integer XOR keeps the FP64 pipe, which on GB300 is slower than
// HBM, out of the measurement.
__global__ void __launch_bounds__(256) k_read(int64_t N2, const ulonglong2 *__restrict__ A,
                                              unsigned long long *__restrict__ out)
{
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long s = 0;
    for (; i + 3 * st < N2; i += 4 * st) {
        ulonglong2 v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = __ldg(A + i + u * st);
#pragma unroll
        for (int u = 0; u < 4; u++) s ^= v[u].x ^ v[u].y;
    }
    for (; i < N2; i += st) {
        const ulonglong2 v = __ldg(A + i);
        s ^= v.x ^ v.y;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s ^= __shfl_xor_sync(0xffffffffu, s, d);
    __shared__ unsigned long long ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t ^= ws[w];
        out[blockIdx.x] = t;
    }
}

// FMA-throughput probe: each thread runs `iters` rounds of 8 independent FMA
// chains in FP64 (fp64 != 0) or FP32 and stores a value that depends on them.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T seed, T *__restrict__ out)
{
    T a = seed + (T)threadIdx.x, b = seed * (T)0.5, c[8];
#pragma unroll
    for (int k = 0; k < 8; k++) c[k] = (T)k * (T)0.125 + (T)threadIdx.x;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++) c[k] = fma(a, b, c[k]);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += c[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_stream(int64_t N, const double *__restrict__ A, const double *__restrict__ B,
                         const int32_t *__restrict__ I, double *__restrict__ C, int indirect)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (indirect) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
            C[i] += A[i] * B[I[i]];
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
            C[i] += A[i] * B[i];
    }
}

int num_sms()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// Persistent tile scheduling (the DYN kernels, U = 1 register tiles and the
// two-diagonal emulated tiles, with the handle's counter) pays where
// tiles differ in cost: a CSR remainder of at least 5 % of the nonzeros.  On
// the 4M-row scattered matrix (remainder 21 %) FP32 went 105 -> 103 us and
// BF16 113.5 -> 106.8 us; on the 27-point stencil (remainder 0.1 %) one tile
// per warp was 2 us faster, the hardware's own CTA scheduling being enough.
bool persistent_tiles(const mhdc_matrix *A, int threads)
{
    return A->sched && threads == SPMV_THREADS && A->nnz_rem * 20 >= A->nnz;
}

// CTAs of kernel fn (SPMV_THREADS a CTA, no dynamic shared memory) that the
// GPU holds at once: the grid of a persistent launch.
int64_t resident_ctas(const void *fn)
{
    static std::mutex mu;
    static std::unordered_map<const void *, int> occ;
    std::lock_guard<std::mutex> lock(mu);
    auto it = occ.find(fn);
    if (it == occ.end()) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, SPMV_THREADS, 0) != cudaSuccess ||
            o < 1)
            o = 1;
        it = occ.emplace(fn, o).first;
    }
    return (int64_t)num_sms() * it->second;
}

struct Variant {
    const void *fn;
    int rw;                      // rows per warp tile
    const void *fn_dyn = nullptr;  // the same tile with persistent scheduling, if built
};

// Tile shapes of the 16-byte-vector kernel: (U vectors per lane, D diagonals
// per load group).  Index = the handle's variant id.
template <typename VT>
Variant vec_variant(int id)
{
    constexpr int V = Tr<VT>::V;
    switch (id) {
    case 0: return {(const void *)k_mhdc_spmv<VT, 1, 4, true>, 32 * V,
                    (const void *)k_mhdc_spmv<VT, 1, 4, true, true>};
    case 1: return {(const void *)k_mhdc_spmv<VT, 2, 2, true>, 64 * V};
    case 2: return {(const void *)k_mhdc_spmv<VT, 2, 4, true>, 64 * V};
    case 3: return {(const void *)k_mhdc_spmv<VT, 1, 8, true>, 32 * V};
    case 4: return {(const void *)k_mhdc_spmv<VT, 4, 2, true>, 128 * V};
    default: return {(const void *)k_mhdc_spmv<VT, 1, 2, true>, 32 * V,
                     (const void *)k_mhdc_spmv<VT, 1, 2, true, true>};
    }
}

template <typename VT>
Variant pick_variant(int32_t n_b, int id)
{
    constexpr int V = Tr<VT>::V;
    if ((n_b % V) != 0) {  // dia_val rows not 16-byte aligned: element loads
        if (n_b >= 32 * 4) return {(const void *)k_mhdc_spmv<VT, 4, 2, false>, 32 * 4};
        return {(const void *)k_mhdc_spmv<VT, 1, 4, false>, 32};
    }
    if (id < 0) id = 5;  // U = 1, D = 2: the fastest on every measured workload
    return vec_variant<VT>(id);
}

Variant variant_for(const mhdc_matrix *A, int id)
{
    switch (A->dtype) {
    case MHDC_F64: return pick_variant<double>(A->n_b, id);
    case MHDC_F32: return pick_variant<float>(A->n_b, id);
    default: return pick_variant<__nv_bfloat16>(A->n_b, id);
    }
}

int launch_dw(mhdc_matrix *A, int shape, const void *d_x, void *d_y, cudaStream_t stream)
{
    constexpr int RWs[3] = {64, 128, 64};
    const int rw = RWs[shape];
    int32_t tpb = (int32_t)((A->n_b + rw - 1) / rw);
    int64_t tiles = (int64_t)tpb * A->n_blocks;
    const int threads = tiles < 2 * SPMV_WARPS * (int64_t)num_sms() ? 32 : SPMV_THREADS;
    const int64_t grid = (tiles + threads / 32 - 1) / (threads / 32);
    // programmatic dependent launches: each kernel's CTAs are scheduled while
    // the one before drains and wait in-kernel for its completion
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    {
        cudaLaunchConfig_t sc = {};
        sc.gridDim = dim3(split_grid(A->n));
        sc.blockDim = dim3(SPLIT_THREADS);
        sc.stream = stream;
        sc.attrs = attr;
        sc.numAttrs = 1;
        MHDC_CUDA_TRY(cudaLaunchKernelEx(&sc, k_split_x, A->n, (const double *)d_x, A->x_dw));
    }
    MHDC_LAUNCH_CHECK("k_split_x");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool dyn = persistent_tiles(A, threads) && shape < 2;
    auto args = [&](auto kern) -> int {
        unsigned long long *sched = nullptr;
        if (dyn) {
            sched = A->sched;
            const int64_t cap = resident_ctas((const void *)kern);
            cfg.gridDim = dim3((unsigned)(grid < cap ? grid : cap));
        }
        MHDC_CUDA_TRY(cudaLaunchKernelEx(
            &cfg, kern, A->n, A->n_b, tpb, tiles, (const int32_t *)A->dia_ptr,
            (const int32_t *)A->dia_offset, (const float2 *)A->dia_dw,
            (const int32_t *)A->csr_row_ptr, (const int32_t *)A->csr_col,
            (const float2 *)A->csr_dw, (const float2 *)A->x_dw, (const double *)A->dia_val,
            (const double *)A->csr_val, (const double *)d_x, (double *)d_y, sched));
        return MHDC_OK;
    };
    int rc;
    switch (shape) {
    case 0: rc = dyn ? args(k_mhdc_spmv_dw<1, 2, true>) : args(k_mhdc_spmv_dw<1, 2>); break;
    case 1: rc = dyn ? args(k_mhdc_spmv_dw<2, 2, true>) : args(k_mhdc_spmv_dw<2, 2>); break;
    default: rc = args(k_mhdc_spmv_dw<1, 4>); break;
    }
    if (rc != MHDC_OK) return rc;
    MHDC_LAUNCH_CHECK("k_mhdc_spmv_dw");
    return MHDC_OK;
}


template <typename VT>
int launch_checked_typed(mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t stream)
{
    using X = typename Tr<VT>::X;
    using Y = typename Tr<VT>::Y;
    const bool vec = (A->n_b % Tr<VT>::V) == 0;
    const int rw = vec ? 32 * Tr<VT>::V : 32;
    const int32_t tpb = (int32_t)((A->n_b + rw - 1) / rw);
    const int64_t tiles = (int64_t)tpb * A->n_blocks;
    const int64_t grid = (tiles + SPMV_WARPS - 1) / SPMV_WARPS;
    const BoundsCheck ck{A->n_blocks, A->P, A->P * (int64_t)A->n_b, A->nnz_rem, A->status};
    auto go = [&](auto kern) {
        kern<<<(unsigned)grid, SPMV_THREADS, 0, stream>>>(
            A->n, A->n_b, tpb, tiles, A->dia_ptr, A->dia_offset, static_cast<const VT *>(A->dia_val),
            A->csr_row_ptr, A->csr_col, static_cast<const VT *>(A->csr_val),
            static_cast<const X *>(d_x), static_cast<Y *>(d_y), ck);
    };
    if (vec) go(k_mhdc_spmv_ck<VT, true>);
    else go(k_mhdc_spmv_ck<VT, false>);
    MHDC_LAUNCH_CHECK("k_mhdc_spmv_ck");
    return MHDC_OK;
}

int launch_checked(mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t stream)
{
    switch (A->dtype) {
    case MHDC_F64: return launch_checked_typed<double>(A, d_x, d_y, stream);
    case MHDC_F32: return launch_checked_typed<float>(A, d_x, d_y, stream);
    default: return launch_checked_typed<__nv_bfloat16>(A, d_x, d_y, stream);
    }
}

int launch_variant(mhdc_matrix *A, int id, const void *d_x, void *d_y, cudaStream_t stream)
{
    if (id >= FIRST_XW_VARIANT) {
        if (xw_supported(A, d_x)) return launch_spmv_xw(A, id - FIRST_XW_VARIANT, d_x, d_y, stream);
        id = -1;
    } else if (id >= FIRST_DW_VARIANT) {
        if (emulation_possible(A)) {
            if (id < FIRST_TMA_DW_VARIANT) return launch_dw(A, id - FIRST_DW_VARIANT, d_x, d_y, stream);
            k_split_x<<<split_grid(A->n), SPLIT_THREADS, 0, stream>>>(
                A->n, (const double *)d_x, A->x_dw);
            MHDC_LAUNCH_CHECK("k_split_x");
            return launch_spmv_tma_dw(A, id - FIRST_TMA_DW_VARIANT, d_x, d_y, stream);
        }
        id = -1;
    }
    if (id >= NUM_REG_VARIANTS) {
        if (tma_supported(A)) return launch_spmv_tma(A, id - NUM_REG_VARIANTS, d_x, d_y, stream);
        id = -1;
    }
    Variant v = variant_for(A, id);
    int32_t tpb = (int32_t)((A->n_b + v.rw - 1) / v.rw);
    int64_t tiles = (int64_t)tpb * A->n_blocks;
    // a matrix with fewer tiles than two 8-warp CTAs per SM would leave SMs
    // idle: one-warp CTAs spread its tiles over every SM, and 32-row tiles of
    // one row a lane (element loads, 8 diagonals a load group) give it twice
    // the warps or more whatever the variant -- the same sums in the same
    // order; on the 7-point 32^3 matrix 4.4 -> 2.8 us a product
    const int threads = tiles < 2 * SPMV_WARPS * (int64_t)num_sms() ? 32 : SPMV_THREADS;
    if (threads == 32) {
        switch (A->dtype) {
        case MHDC_F64: v = {(const void *)k_mhdc_spmv<double, 1, 8, false>, 32}; break;
        case MHDC_F32: v = {(const void *)k_mhdc_spmv<float, 1, 8, false>, 32}; break;
        default: v = {(const void *)k_mhdc_spmv<__nv_bfloat16, 1, 8, false>, 32}; break;
        }
        tpb = (int32_t)((A->n_b + 31) / 32);
        tiles = (int64_t)tpb * A->n_blocks;
    }
    int64_t grid = (tiles + threads / 32 - 1) / (threads / 32);
    unsigned long long *sched = nullptr;
    const void *fn = v.fn;
    if (v.fn_dyn && persistent_tiles(A, threads)) {
        fn = v.fn_dyn;
        sched = A->sched;
        const int64_t cap = resident_ctas(fn);
        if (grid > cap) grid = cap;
    }
    int64_t n = A->n;
    int32_t n_b = A->n_b;
    const void *dv = A->dia_val, *cv = A->csr_val;
    const int32_t *dp = A->dia_ptr, *doff = A->dia_offset, *crp = A->csr_row_ptr, *cc = A->csr_col;
    void *args[] = {&n, &n_b, &tpb, &tiles, (void *)&dp, (void *)&doff, (void *)&dv, (void *)&crp,
                    (void *)&cc, (void *)&cv, (void *)&d_x, &d_y, (void *)&sched};
    MHDC_CUDA_TRY(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(threads), args, 0, stream));
    return MHDC_OK;
}

}  // namespace

int spmv_grid_for(const mhdc_matrix *A)
{
    if (A->n == 0) return 0;
    const Variant v = variant_for(A, (A->variant >= 0 && A->variant < NUM_REG_VARIANTS) ? A->variant : -1);
    const int64_t tpb = (A->n_b + v.rw - 1) / v.rw;
    return (int)((tpb * A->n_blocks + SPMV_WARPS - 1) / SPMV_WARPS);
}

int launch_spmv(mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t stream)
{
    if (A->n == 0) return MHDC_OK;
    if (A->checked) return launch_checked(A, d_x, d_y, stream);
    return launch_variant(A, A->variant, d_x, d_y, stream);
}

int tune_spmv(mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t stream, int32_t *best,
              float *times_us)
{
    if (A->n == 0) {
        if (best) *best = -1;
        return MHDC_OK;
    }
    cudaEvent_t e0, e1;
    MHDC_CUDA_TRY(cudaEventCreate(&e0));
    MHDC_CUDA_TRY(cudaEventCreate(&e1));
    int best_id = -1;
    float best_t = 0.f;
    const int reps = 20;
    auto time_id = [&](int id, float *us_out) -> int {
        int rc = MHDC_OK;
        for (int r = 0; r < 3 && rc == MHDC_OK; r++) rc = launch_variant(A, id, d_x, d_y, stream);
        cudaEventRecord(e0, stream);
        for (int r = 0; r < reps && rc == MHDC_OK; r++) rc = launch_variant(A, id, d_x, d_y, stream);
        cudaEventRecord(e1, stream);
        if (rc != MHDC_OK) return rc;
        MHDC_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *us_out = ms * 1e3f / reps;
        return MHDC_OK;
    };
    for (int id = 0; id < MHDC_NUM_VARIANTS; id++) {
        float us = 0.f;
        const int rc = time_id(id, &us);
        if (rc != MHDC_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rc;
        }
        if (times_us) times_us[id] = us;
        if (best_id < 0 || us < best_t) {
            best_id = id;
            best_t = us;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    A->variant = best_id;
    if (best) *best = best_id;
    return MHDC_OK;
}

int launch_csr(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
               const double *x, double *y, cudaStream_t stream)
{
    if (n == 0) return MHDC_OK;
    const int64_t grid = (n + CSR_THREADS - 1) / CSR_THREADS;
    k_csr_spmv<<<(unsigned)grid, CSR_THREADS, 0, stream>>>(n, rp, col, val, x, y);
    MHDC_LAUNCH_CHECK("k_csr_spmv");
    return MHDC_OK;
}

int launch_dia(const mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t stream)
{
    if (A->n == 0) return MHDC_OK;
    switch (A->dtype) {
    case MHDC_F64: return dia_typed<double>(A, d_x, d_y, stream);
    case MHDC_F32: return dia_typed<float>(A, d_x, d_y, stream);
    default: return dia_typed<__nv_bfloat16>(A, d_x, d_y, stream);
    }
}

int launch_read_bench(int64_t N, const double *A, double *out, int grid, cudaStream_t stream)
{
    if (N <= 0) return MHDC_OK;
    k_read<<<grid, 256, 0, stream>>>(N / 2, reinterpret_cast<const ulonglong2 *>(A),
                                     reinterpret_cast<unsigned long long *>(out));
    MHDC_LAUNCH_CHECK("k_read");
    return MHDC_OK;
}

int read_bench_grid() { return num_sms() * 8; }

int launch_fma_probe(int fp64, int iters, void *out, cudaStream_t stream)
{
    if (fp64) k_fma_probe<double><<<num_sms() * 8, 256, 0, stream>>>(iters, 1.0, (double *)out);
    else k_fma_probe<float><<<num_sms() * 8, 256, 0, stream>>>(iters, 1.0f, (float *)out);
    MHDC_LAUNCH_CHECK("k_fma_probe");
    return MHDC_OK;
}

int launch_stream_bench(int64_t N, const double *A, const double *B, const int32_t *I, double *C,
                        int indirect, cudaStream_t stream)
{
    if (N <= 0) return MHDC_OK;
    int64_t need = (N + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    k_stream<<<(unsigned)(need < cap ? need : cap), 256, 0, stream>>>(N, A, B, I, C, indirect);
    MHDC_LAUNCH_CHECK("k_stream");
    return MHDC_OK;
}

}  // namespace mhdc

// ---------------------------------------------------------------------------
// Batched product: y_i = A_i x_i for m matrices in one persistent launch.
// The warp tiles of all matrices form one list (matrix i's tiles start at
// tile0[i]); warps take chunks of BATCH_CHUNK tiles from a global counter, so
// matrices of uneven size share the GPU without a launch per matrix.  Each
// tile runs the register kernel's code (reg_tile, U = 1, D = 2).  The last CTA
// to finish resets the counters for the next launch (no waits between CTAs).
// ---------------------------------------------------------------------------
namespace mhdc {
namespace {

constexpr int BATCH_CHUNK = 4;

// Last matrix whose first tile is <= g (tile0 ascending, mats[0].tile0 = 0).
__device__ __forceinline__ int batch_find(const BatchMat *__restrict__ mats, int32_t m, int64_t g)
{
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mats[mid].tile0 <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename VT>
__global__ void __launch_bounds__(SPMV_THREADS, 4)
k_batch_spmv(int32_t m, const BatchMat *__restrict__ mats, int64_t total_tiles,
             const void *const *__restrict__ xs, void *const *__restrict__ ys,
             unsigned long long *__restrict__ ctr)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctr[0], (unsigned long long)BATCH_CHUNK);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= (unsigned long long)total_tiles) break;
        for (int c = 0; c < BATCH_CHUNK; c++) {
            const int64_t g = (int64_t)base + c;
            if (g >= total_tiles) break;
            const int lo = batch_find(mats, m, g);
            const BatchMat &M = mats[lo];
            const int64_t w = g - M.tile0;
            using X = typename Tr<VT>::X;
            using Y = typename Tr<VT>::Y;
            if (M.vec)
                reg_tile<VT, 1, 2, true, true>(w, M.n, M.n_b, M.tpb, M.dia_ptr, M.dia_offset,
                                         static_cast<const VT *>(M.dia_val), M.csr_row_ptr,
                                         M.csr_col, static_cast<const VT *>(M.csr_val),
                                         static_cast<const X *>(xs[lo]), static_cast<Y *>(ys[lo]));
            else
                reg_tile<VT, 1, 2, false>(w, M.n, M.n_b, M.tpb, M.dia_ptr, M.dia_offset,
                                          static_cast<const VT *>(M.dia_val), M.csr_row_ptr,
                                          M.csr_col, static_cast<const VT *>(M.csr_val),
                                          static_cast<const X *>(xs[lo]), static_cast<Y *>(ys[lo]));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctr[1], 1ull) == (unsigned long long)gridDim.x - 1) {
            ctr[0] = 0;
            ctr[1] = 0;
            __threadfence();
        }
    }
}

template <typename VT>
const void *batch_kernel() { return (const void *)k_batch_spmv<VT>; }

}  // namespace

int batch_prepare(mhdc_batch *B)
{
    const void *fn = B->dtype == MHDC_F64 ? batch_kernel<double>()
                     : B->dtype == MHDC_F32 ? batch_kernel<float>() : batch_kernel<__nv_bfloat16>();
    int occ = 0;
    MHDC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, SPMV_THREADS, 0));
    if (occ < 1) occ = 1;
    const int64_t need = (B->total_tiles + (int64_t)SPMV_WARPS * BATCH_CHUNK - 1) /
                         ((int64_t)SPMV_WARPS * BATCH_CHUNK);
    const int64_t cap = (int64_t)num_sms() * occ;
    B->grid = (int)(need < cap ? (need > 0 ? need : 1) : cap);
    return MHDC_OK;
}

int batch_tile_rows(int dtype, int n_b, int *vec)
{
    const int V = dtype == MHDC_F64 ? 2 : dtype == MHDC_F32 ? 4 : 8;
    *vec = (n_b % V) == 0;
    return *vec ? 32 * V : 32;
}

int launch_batch(mhdc_batch *B, const void *const *d_xs, void *const *d_ys, cudaStream_t st)
{
    if (B->total_tiles == 0) return MHDC_OK;
    const void *fn = B->dtype == MHDC_F64 ? batch_kernel<double>()
                     : B->dtype == MHDC_F32 ? batch_kernel<float>() : batch_kernel<__nv_bfloat16>();
    int32_t m = B->m;
    const BatchMat *mats = B->d_mats;
    int64_t tiles = B->total_tiles;
    unsigned long long *ctr = B->d_ctr;
    void *args[] = {&m, (void *)&mats, &tiles, (void *)&d_xs, (void *)&d_ys, (void *)&ctr};
    MHDC_CUDA_TRY(cudaLaunchKernel(fn, dim3(B->grid), dim3(SPMV_THREADS), args, 0, st));
    return MHDC_OK;
}

}  // namespace mhdc
