// M-HDC y = A x (Fig. 13) with the diagonal values streamed by TMA.
//
// A persistent CTA = NCW consumer warps + 1 producer warp.  Work unit = R
// consecutive rows of one row block (R = NCW * 32 lanes * U vectors * 16 B).
// For every diagonal of the unit's block, the producer's elected lane issues
// one 1-D bulk copy (cp.async.bulk) of the unit's R values (contiguous in
// dia_val) into a ring of STAGES shared-memory buffers, completing on the
// stage's "full" mbarrier.  Consumers first issue the x loads of the next D
// diagonals (their addresses depend only on the offsets), then wait for the
// stages, read their rows' values from shared memory (16 B per lane,
// conflict-free), accumulate in registers and release the stages on the
// "empty" mbarriers.  The CSR remainder rows of a unit are added by the
// consumers from global memory before the diagonals; y is written once.
//
// Every mbarrier wait is bounded: a wait that gives up sets bit 0 of
// *status, the waiting warp stops, and the producer drains the copies it
// still has in flight (again bounded) before the CTA exits.
#include <cstring>
#include <type_traits>

#include "dw_arith.cuh"
#include "mhdc_internal.cuh"

namespace mhdc {
namespace {

template <typename VT>
struct TrT;
template <>
struct TrT<double> {
    using X = double;
    using Y = double;
    using Acc = double;
};
template <>
struct TrT<float> {
    using X = float;
    using Y = float;
    using Acc = float;
};
template <>
struct TrT<__nv_bfloat16> {
    using X = __nv_bfloat16;
    using Y = float;
    using Acc = float;
};

__device__ __forceinline__ double wide(double v) { return v; }
__device__ __forceinline__ float wide(float v) { return v; }
__device__ __forceinline__ float wide(__nv_bfloat16 v) { return __bfloat162float(v); }

// A wait gives up after WAIT_LIMIT_NS of global-timer time (or SPIN_LIMIT
// polls, whichever comes first); a correct pipeline never gets near either.
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;
constexpr uint32_t SPIN_LIMIT = 1u << 30;

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with the given parity to complete; false if
// the bounded spin gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1; i < SPIN_LIMIT; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0 && global_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
    return false;
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size % 16 == 0),
// completing `bytes` of transaction count on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

template <typename X, int V>
__device__ __forceinline__ void load_xv(const X *__restrict__ x, int64_t j, bool aligned, X (&xv)[V])
{
    if (aligned) {
        const uint4 r = __ldg(reinterpret_cast<const uint4 *>(x + j));
        memcpy(xv, &r, 16);
        return;
    }
#pragma unroll
    for (int m = 0; m < V; m++) xv[m] = __ldg(x + j + m);
}

template <typename VT, int NCW, int U, int D, int STAGES>
struct TmaCfg {
    static constexpr int V = 16 / sizeof(VT);
    static constexpr int NT = NCW * 32;          // consumer threads
    static constexpr int R = NT * U * V;         // rows per unit
    static constexpr int STAGE_BYTES = R * (int)sizeof(VT);
    static constexpr int THREADS = NT + 32;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES;
};

template <typename VT, int NCW, int U, int D, int STAGES>
__global__ void __launch_bounds__(TmaCfg<VT, NCW, U, D, STAGES>::THREADS)
k_mhdc_spmv_tma(int64_t n, int32_t n_b, int32_t upb, int64_t n_units,
                const int32_t *__restrict__ dia_ptr, const int32_t *__restrict__ dia_offset,
                const VT *__restrict__ dia_val, const int32_t *__restrict__ csr_row_ptr,
                const int32_t *__restrict__ csr_col, const VT *__restrict__ csr_val,
                const typename TrT<VT>::X *__restrict__ x, typename TrT<VT>::Y *__restrict__ y,
                int *__restrict__ status)
{
    using C = TmaCfg<VT, NCW, U, D, STAGES>;
    using Acc = typename TrT<VT>::Acc;
    using X = typename TrT<VT>::X;
    constexpr int V = C::V, NT = C::NT, R = C::R;
    extern __shared__ __align__(128) uint8_t ring[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == NCW) {
        // ---------------- producer (one elected lane)
        if (lane != 0) return;
        int stage = 0;
        uint32_t phase = 0;
        int64_t issued = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
            const int64_t ib = u / upb;
            const int32_t t0 = (int32_t)(u - ib * upb) * R;
            const int64_t r0 = ib * (int64_t)n_b;
            const int32_t rows = (int32_t)((n - r0 < n_b) ? (n - r0) : n_b);
            if (t0 >= rows) continue;
            const int32_t ru = (rows - t0 < R) ? rows - t0 : R;
            const uint32_t bytes = (uint32_t)(((int64_t)ru * sizeof(VT) + 15) & ~(int64_t)15);
            const int32_t p0 = dia_ptr[ib], p1 = dia_ptr[ib + 1];
            for (int32_t p = p0; p < p1; p++) {
                if (!mbar_wait(&empty[stage], phase ^ 1)) {
                    atomicOr(status, 1);
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&full[stage], bytes);
                bulk_load(ring + (size_t)stage * C::STAGE_BYTES,
                          dia_val + (int64_t)p * n_b + t0, bytes, &full[stage]);
                issued++;
                if (++stage == STAGES) {
                    stage = 0;
                    phase ^= 1;
                }
            }
        }
        if (!ok) {
            // drain: wait (bounded) for the copies still in flight
            const int64_t k = issued < STAGES ? issued : STAGES;
            for (int64_t q = 1; q <= k; q++) {
                int s = stage - (int)q;
                uint32_t ph = phase;
                if (s < 0) {
                    s += STAGES;
                    ph ^= 1;
                }
                mbar_wait(&full[s], ph);
            }
        }
        return;
    }

    // ---------------- consumers
    int stage = 0;
    uint32_t phase = 0;
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int64_t ib = u / upb;
        const int32_t t0 = (int32_t)(u - ib * upb) * R;
        const int64_t r0 = ib * (int64_t)n_b;
        const int32_t rows = (int32_t)((n - r0 < n_b) ? (n - r0) : n_b);
        if (t0 >= rows) continue;
        const int32_t ru = (rows - t0 < R) ? rows - t0 : R;
        const bool full_unit = ru == R;

        int32_t tl[U];  // first row (within the unit) of each of this lane's vectors
#pragma unroll
        for (int k = 0; k < U; k++) tl[k] = (k * NT + tid) * V;

        Acc acc[U][V];
#pragma unroll
        for (int k = 0; k < U; k++)
#pragma unroll
            for (int m = 0; m < V; m++) acc[k][m] = Acc(0);

        // CSR remainder rows of the unit (Fig. 13, first loop)
        if (csr_row_ptr[r0 + t0] != csr_row_ptr[r0 + t0 + ru]) {
#pragma unroll
            for (int k = 0; k < U; k++)
#pragma unroll
                for (int m = 0; m < V; m++) {
                    const int32_t t = tl[k] + m;
                    if (t < ru) {
                        const int64_t i = r0 + t0 + t;
                        rem_row_add(acc[k][m], csr_row_ptr[i], csr_row_ptr[i + 1], csr_col,
                                    csr_val, x);
                    }
                }
        }

        // the block's diagonals, D stages at a time (Fig. 13, second loop)
        const int32_t p0 = dia_ptr[ib], p1 = dia_ptr[ib + 1];
        const int64_t xw = r0 + t0 + (int64_t)warp * 32 * V;  // this warp's first row, k = 0
        bool ok = true;
        int32_t p = p0;
        auto group = [&](auto Dc) {
            constexpr int DD = decltype(Dc)::value;
            X xv[DD][U][V];
#pragma unroll
            for (int d = 0; d < DD; d++) {
                const int64_t off = dia_offset[p + d];
#pragma unroll
                for (int k = 0; k < U; k++) {
                    const int64_t jw = xw + (int64_t)k * NT * V + off;  // warp-uniform
                    if (full_unit && jw >= 0 && jw + 32 * V <= n) {
                        const int64_t j = jw + lane * V;
                        load_xv<X, V>(x, j, ((reinterpret_cast<uintptr_t>(x + jw)) & 15) == 0,
                                      xv[d][k]);
                    } else {
#pragma unroll
                        for (int m = 0; m < V; m++) {
                            const int64_t jm = jw + lane * V + m;
                            xv[d][k][m] = (tl[k] + m < ru && jm >= 0 && jm < n) ? __ldg(x + jm)
                                                                                 : X(0);
                        }
                    }
                }
            }
#pragma unroll
            for (int d = 0; d < DD; d++) {
                int s = stage + d;
                uint32_t ph = phase;
                if (s >= STAGES) {
                    s -= STAGES;
                    ph ^= 1;
                }
                if (!mbar_wait(&full[s], ph)) ok = false;
            }
            if (!ok) return;
#pragma unroll
            for (int d = 0; d < DD; d++) {
                int s = stage + d;
                if (s >= STAGES) s -= STAGES;
                const VT *sv = reinterpret_cast<const VT *>(ring + (size_t)s * C::STAGE_BYTES);
#pragma unroll
                for (int k = 0; k < U; k++) {
                    VT v[V];
                    const uint4 r = *reinterpret_cast<const uint4 *>(sv + tl[k]);
                    memcpy(v, &r, 16);
#pragma unroll
                    for (int m = 0; m < V; m++) acc[k][m] += wide(v[m]) * wide(xv[d][k][m]);
                }
            }
            __syncwarp();
#pragma unroll
            for (int d = 0; d < DD; d++) {
                int s = stage + d;
                if (s >= STAGES) s -= STAGES;
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            stage += DD;
            if (stage >= STAGES) {
                stage -= STAGES;
                phase ^= 1;
            }
            p += DD;
        };
        while (ok && p + D <= p1) group(std::integral_constant<int, D>{});
        while (ok && p < p1) group(std::integral_constant<int, 1>{});
        if (!ok) {
            if (lane == 0) atomicOr(status, 1);
            return;
        }
#pragma unroll
        for (int k = 0; k < U; k++)
#pragma unroll
            for (int m = 0; m < V; m++)
                if (tl[k] + m < ru) y[r0 + t0 + tl[k] + m] = acc[k][m];
    }
}

// ---------------------------------------------------------------------------
// Both operands in shared memory (variants 16-19).
//
// As k_mhdc_spmv_tma, and x too is staged by TMA.  For a unit whose rows
// start at a0 = r0 + t0, diagonal p reads x[a0 + off_p, a0 + off_p + R).
// Consecutive diagonals of a block share one x window of XCAP elements: it
// starts at base = (a0 + off of its first diagonal) rounded down to 16 bytes,
// and diagonal p joins it while (a0 + off_p + R) rounded up to 16 bytes stays
// within base + XW (XW = XCAP - V: one vector of slack, so that a misaligned
// 16-byte read stays inside the window).  Per window the producer issues one
// bulk copy of its in-range part [max(base, 0), min(end, n rounded down to 16
// bytes)) into a ring of XSTAGES windows (completing on the window's "xfull"
// mbarrier), then the copies of its diagonals' values into the value ring.
// The consumers apply the same rule to the same offsets, wait for a window
// once, read x from shared memory for each of its diagonals and release it
// ("xempty") when they move on.  Warps whose x range is not wholly inside
// [0, n rounded down to 16 bytes) take an element-wise path: 0 outside
// [0, n), global memory for the last n mod V elements.  The remainder rows
// are read from global memory first, as in k_mhdc_spmv_tma.  For a stencil
// the windows turn the block's nd diagonals into a few x copies (3 for the
// 27-point stencil), and the consumers' only waits are the mbarriers.
// ---------------------------------------------------------------------------
// Written by the producer for each value stage before its copy is issued
// (the stage's mbarrier arrive releases it to the consumers).
struct __align__(16) XwMeta {
    int64_t a;      // x index of the unit's first row on this diagonal
    int32_t e0;     // a - (first element of the x window), >= 0
    int32_t first;  // the diagonal opens a new x window
};

// The producer's position in its sequence of windows: unit u (rows from t0
// of its row block, x index a0 of the unit's first row, value copy size
// `bytes`: the unit's rows of one diagonal rounded up to 16 bytes) and its
// next diagonal p of [p, p1).  Units without diagonals are
// skipped (their consumers only add the remainder); u >= n_units: done.
struct XwCursor {
    int64_t u, a0;
    int32_t t0, p, p1;
    uint32_t bytes;

    template <int R, int ES>
    __device__ void seek(int64_t from, int64_t step, int64_t n_units, int32_t upb, int64_t n,
                         int32_t n_b, const int32_t *__restrict__ dia_ptr)
    {
        for (u = from; u < n_units; u += step) {
            const int64_t ib = u / upb;
            t0 = (int32_t)(u - ib * upb) * R;
            const int64_t r0 = ib * (int64_t)n_b;
            const int32_t rows = (int32_t)((n - r0 < n_b) ? (n - r0) : n_b);
            if (t0 >= rows) continue;
            p = dia_ptr[ib];
            p1 = dia_ptr[ib + 1];
            if (p == p1) continue;
            a0 = r0 + t0;
            const int32_t ru = (rows - t0 < R) ? rows - t0 : R;
            bytes = (uint32_t)(((int64_t)ru * ES + 15) & ~(int64_t)15);
            return;
        }
    }

    // One past the last diagonal of the window that starts at p.
    template <int R, int V, int XW>
    __device__ int32_t window_end(const int32_t *__restrict__ dia_offset) const
    {
        const int64_t base = (a0 + dia_offset[p]) & -(int64_t)V;
        int32_t q = p + 1;
        while (q < p1 && ((a0 + dia_offset[q] + R + V - 1) & -(int64_t)V) - base <= XW) q++;
        return q;
    }
};

template <typename VT, int NCW, int U, int DSTAGES, int XSTAGES>
struct XwCfg {
    static constexpr int V = 16 / sizeof(VT);
    static constexpr int NT = NCW * 32;          // consumer threads
    static constexpr int R = NT * U * V;         // rows per unit
    static constexpr int STAGE_BYTES = R * (int)sizeof(VT);
    static constexpr int XCAP = R + 512;         // elements per x window
    static constexpr int XW = XCAP - V;
    static constexpr int XBYTES = XCAP * (int)sizeof(VT);
    static constexpr int THREADS = NT + 32;
    static constexpr size_t SMEM = (size_t)DSTAGES * STAGE_BYTES + (size_t)XSTAGES * XBYTES;
    static_assert(STAGE_BYTES % 16 == 0 && XBYTES % 16 == 0, "stages must be 16-byte multiples");
};

template <typename VT, int NCW, int U, int DSTAGES, int XSTAGES>
__global__ void __launch_bounds__(XwCfg<VT, NCW, U, DSTAGES, XSTAGES>::THREADS)
k_mhdc_spmv_xw(int64_t n, int32_t n_b, int32_t upb, int64_t n_units,
               const int32_t *__restrict__ dia_ptr, const int32_t *__restrict__ dia_offset,
               const VT *__restrict__ dia_val, const int32_t *__restrict__ csr_row_ptr,
               const int32_t *__restrict__ csr_col, const VT *__restrict__ csr_val,
               const typename TrT<VT>::X *__restrict__ x, typename TrT<VT>::Y *__restrict__ y,
               int *__restrict__ status)
{
    using C = XwCfg<VT, NCW, U, DSTAGES, XSTAGES>;
    using Acc = typename TrT<VT>::Acc;
    using X = typename TrT<VT>::X;
    static_assert(sizeof(X) == sizeof(VT), "x and values have one element size");
    constexpr int V = C::V, NT = C::NT, R = C::R;
    constexpr int64_t VM = -(int64_t)V;  // mask: round down to a multiple of V
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *const dring = smem;
    uint8_t *const xring = smem + (size_t)DSTAGES * C::STAGE_BYTES;
    __shared__ __align__(8) uint64_t dfull[DSTAGES], dempty[DSTAGES], xfull[XSTAGES],
        xempty[XSTAGES];
    __shared__ XwMeta meta[DSTAGES];  // per value stage: its diagonal's x position

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < DSTAGES; s++) {
            mbar_init(&dfull[s], 1);
            mbar_init(&dempty[s], NCW);
        }
        for (int s = 0; s < XSTAGES; s++) {
            mbar_init(&xfull[s], 1);
            mbar_init(&xempty[s], NCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int64_t nV = n & VM;  // x[0, nV) can be bulk-copied

    if (warp == NCW) {
        // ---------------- producer (one elected lane)
        // Two cursors walk the same windows: x copies run XLOOK windows ahead
        // of the value copies, so a window's x is in flight while the values
        // of the windows before it stream.  Deadlock-free: x window g reuses
        // the slot of window g - XSTAGES <= (window of the values being
        // issued) - 2, which the consumers release on entering the window
        // after it, whose values are already issued.
        if (lane != 0) return;
        constexpr int XLOOK = XSTAGES - 2;
        XwCursor xc, dc;
        xc.seek<R, (int)sizeof(VT)>(blockIdx.x, gridDim.x, n_units, upb, n, n_b, dia_ptr);
        dc = xc;
        int ds = 0, xs = 0;
        uint32_t dph = 0, xph = 0;
        int64_t dissued = 0, xissued = 0, xg = 0, dg = 0;
        bool ok = true;
        while (ok && dc.u < n_units) {
            while (xc.u < n_units && xg <= dg + XLOOK) {
                const int32_t q = xc.window_end<R, V, C::XW>(dia_offset);
                const int64_t base = (xc.a0 + dia_offset[xc.p]) & VM;
                const int64_t wend = (xc.a0 + dia_offset[q - 1] + R + V - 1) & VM;
                const int64_t lo = base > 0 ? base : 0;
                const int64_t hi = wend < nV ? wend : nV;
                const uint32_t xbytes = hi > lo ? (uint32_t)((hi - lo) * sizeof(X)) : 0u;
                if (!mbar_wait(&xempty[xs], xph ^ 1)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&xfull[xs], xbytes);
                if (xbytes)
                    bulk_load(xring + (size_t)xs * C::XBYTES + (size_t)(lo - base) * sizeof(X),
                              x + lo, xbytes, &xfull[xs]);
                xissued++;
                if (++xs == XSTAGES) {
                    xs = 0;
                    xph ^= 1;
                }
                xg++;
                xc.p = q;
                if (xc.p == xc.p1) xc.seek<R, (int)sizeof(VT)>(xc.u + gridDim.x, gridDim.x, n_units, upb, n, n_b, dia_ptr);
            }
            if (!ok) break;
            const int32_t q = dc.window_end<R, V, C::XW>(dia_offset);
            const int64_t dbase = (dc.a0 + dia_offset[dc.p]) & VM;
            for (int32_t pw = dc.p; dc.p < q; dc.p++) {
                if (!mbar_wait(&dempty[ds], dph ^ 1)) {
                    ok = false;
                    break;
                }
                const int64_t a = dc.a0 + dia_offset[dc.p];
                meta[ds].a = a;
                meta[ds].e0 = (int32_t)(a - dbase);
                meta[ds].first = dc.p == pw;
                mbar_arrive_expect_tx(&dfull[ds], dc.bytes);  // releases the metadata too
                bulk_load(dring + (size_t)ds * C::STAGE_BYTES,
                          dia_val + (int64_t)dc.p * n_b + dc.t0, dc.bytes, &dfull[ds]);
                dissued++;
                if (++ds == DSTAGES) {
                    ds = 0;
                    dph ^= 1;
                }
            }
            dg++;
            if (ok && dc.p == dc.p1) dc.seek<R, (int)sizeof(VT)>(dc.u + gridDim.x, gridDim.x, n_units, upb, n, n_b, dia_ptr);
        }
        if (!ok) {
            atomicOr(status, 1);
            // drain: wait (bounded) for the copies still in flight
            const int64_t kd = dissued < DSTAGES ? dissued : DSTAGES;
            for (int64_t j = 1; j <= kd; j++) {
                int s = ds - (int)j;
                uint32_t ph = dph;
                if (s < 0) {
                    s += DSTAGES;
                    ph ^= 1;
                }
                mbar_wait(&dfull[s], ph);
            }
            const int64_t kx = xissued < XSTAGES ? xissued : XSTAGES;
            for (int64_t j = 1; j <= kx; j++) {
                int s = xs - (int)j;
                uint32_t ph = xph;
                if (s < 0) {
                    s += XSTAGES;
                    ph ^= 1;
                }
                mbar_wait(&xfull[s], ph);
            }
        }
        return;
    }

    // ---------------- consumers
    int ds = 0, xs = 0;
    uint32_t dph = 0, xph = 0;
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int64_t ib = u / upb;
        const int32_t t0 = (int32_t)(u - ib * upb) * R;
        const int64_t r0 = ib * (int64_t)n_b;
        const int32_t rows = (int32_t)((n - r0 < n_b) ? (n - r0) : n_b);
        if (t0 >= rows) continue;
        const int32_t ru = (rows - t0 < R) ? rows - t0 : R;

        int32_t tl[U];  // first row (within the unit) of each of this lane's vectors
#pragma unroll
        for (int k = 0; k < U; k++) tl[k] = (k * NT + tid) * V;

        Acc acc[U][V];
#pragma unroll
        for (int k = 0; k < U; k++)
#pragma unroll
            for (int m = 0; m < V; m++) acc[k][m] = Acc(0);

        // CSR remainder rows of the unit (Fig. 13, first loop)
        if (csr_row_ptr[r0 + t0] != csr_row_ptr[r0 + t0 + ru]) {
#pragma unroll
            for (int k = 0; k < U; k++)
#pragma unroll
                for (int m = 0; m < V; m++) {
                    const int32_t t = tl[k] + m;
                    if (t < ru) {
                        const int64_t i = r0 + t0 + t;
                        rem_row_add(acc[k][m], csr_row_ptr[i], csr_row_ptr[i + 1], csr_col,
                                    csr_val, x);
                    }
                }
        }

        // the block's diagonals (Fig. 13, second loop), one at a time; the
        // producer's metadata of each value stage gives the diagonal's x
        // index a and its position e0 in the current x window
        const int32_t p1 = dia_ptr[ib + 1];
        bool held = false, ok = true;
        for (int32_t p = dia_ptr[ib]; p < p1; p++) {
            if (!__all_sync(0xffffffffu, mbar_wait(&dfull[ds], dph))) {
                ok = false;
                break;
            }
            const XwMeta mt = meta[ds];
            if (mt.first) {  // warp-uniform: the diagonal opens the next x window
                if (held) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&xempty[xs]);
                    if (++xs == XSTAGES) {
                        xs = 0;
                        xph ^= 1;
                    }
                }
                held = true;
                if (!__all_sync(0xffffffffu, mbar_wait(&xfull[xs], xph))) {
                    ok = false;
                    break;
                }
            }
            const int64_t a = mt.a;  // x index of the unit's first row
            const VT *sv = reinterpret_cast<const VT *>(dring + (size_t)ds * C::STAGE_BYTES);
            const X *sx = reinterpret_cast<const X *>(xring + (size_t)xs * C::XBYTES);  // x[base]
            const int32_t e0 = mt.e0;      // window index of the unit's first row, >= 0
            const int64_t base = a - e0;
            const int r = e0 & (V - 1);    // misalignment in elements (warp-uniform)
#pragma unroll
            for (int k = 0; k < U; k++) {
                VT v[V];
                const uint4 rv = *reinterpret_cast<const uint4 *>(sv + tl[k]);
                memcpy(v, &rv, 16);
                X xv[V];
                const int64_t jw = a + (int64_t)(k * NT + warp * 32) * V;  // warp-uniform
                if (jw >= 0 && jw + 32 * V <= nV) {
                    const X *xp = sx + e0 + tl[k];
                    if (r == 0) {
                        const uint4 q = *reinterpret_cast<const uint4 *>(xp);
                        memcpy(xv, &q, 16);
                    } else if constexpr (V == 2) {
                        xv[0] = xp[0];
                        xv[1] = xp[1];
                    } else {
                        const uint4 lo = *reinterpret_cast<const uint4 *>(xp - r);
                        const uint4 hi = *reinterpret_cast<const uint4 *>(xp - r + V);
                        const uint4 q = window16(lo, hi, r * (int)sizeof(X));
                        memcpy(xv, &q, 16);
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < V; m++) {
                        const int64_t j = a + tl[k] + m;
                        xv[m] = (j < 0 || j >= n) ? X(0) : (j < nV ? sx[j - base] : __ldg(x + j));
                    }
                }
#pragma unroll
                for (int m = 0; m < V; m++) acc[k][m] += wide(v[m]) * wide(xv[m]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[ds]);
            if (++ds == DSTAGES) {
                ds = 0;
                dph ^= 1;
            }
        }
        if (!ok) {
            if (lane == 0) atomicOr(status, 1);
            return;
        }
        if (held) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&xempty[xs]);
            if (++xs == XSTAGES) {
                xs = 0;
                xph ^= 1;
            }
        }
#pragma unroll
        for (int k = 0; k < U; k++)
#pragma unroll
            for (int m = 0; m < V; m++)
                if (tl[k] + m < ru) y[r0 + t0 + tl[k] + m] = acc[k][m];
    }
}

int num_sms_tma();

// ---------------------------------------------------------------------------
// FP64 handles, emulated product (variants 13-15): the same pipeline over
// 8-byte slots.  The producer streams the FP32 pairs dia_dw and consumers run
// the double-word arithmetic of dw_arith.cuh on x_dw; a row whose sum comes
// out NaN read an x outside the window (marked by the split) and is
// recomputed with native FP64 arithmetic (native_row).
// ---------------------------------------------------------------------------
template <int NCW, int U, int D, int STAGES>
__device__ __forceinline__ void tma_dw_consumer(
    int64_t n, int32_t n_b, int32_t upb, int64_t n_units, const int32_t *__restrict__ dia_ptr,
    const int32_t *__restrict__ dia_offset, const double *__restrict__ dia_val,
    const int32_t *__restrict__ csr_row_ptr, const int32_t *__restrict__ csr_col,
    const double *__restrict__ csr_val, const float2 *__restrict__ csr_dw,
    const double *__restrict__ x, const float2 *__restrict__ x_dw, double *__restrict__ y,
    uint8_t *ring, uint64_t *full, uint64_t *empty, int *__restrict__ status)
{
    constexpr int V = 2, NT = NCW * 32, R = NT * U * V, STAGE_BYTES = R * 8;
    using XT = float2;
    const XT *xs = x_dw;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int stage = 0;
    uint32_t phase = 0;
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int64_t ib = u / upb;
        const int32_t t0 = (int32_t)(u - ib * upb) * R;
        const int64_t r0 = ib * (int64_t)n_b;
        const int32_t rows = (int32_t)((n - r0 < n_b) ? (n - r0) : n_b);
        if (t0 >= rows) continue;
        const int32_t ru = (rows - t0 < R) ? rows - t0 : R;
        const bool full_unit = ru == R;
        int32_t tl[U];
#pragma unroll
        for (int k = 0; k < U; k++) tl[k] = (k * NT + tid) * V;
        float sh[U][V], sl[U][V];
#pragma unroll
        for (int k = 0; k < U; k++)
#pragma unroll
            for (int m = 0; m < V; m++) sh[k][m] = sl[k][m] = 0.f;
        if (csr_row_ptr[r0 + t0] != csr_row_ptr[r0 + t0 + ru]) {
#pragma unroll
            for (int k = 0; k < U; k++)
#pragma unroll
                for (int m = 0; m < V; m++) {
                    const int32_t t = tl[k] + m;
                    if (t < ru) {
                        const int64_t i = r0 + t0 + t;
                        const int32_t a = csr_row_ptr[i], b = csr_row_ptr[i + 1];
                        for (int32_t q = a; q < b; q++)
                            dw::dw_fma(sh[k][m], sl[k][m], __ldg(csr_dw + q),
                                       __ldg(x_dw + __ldg(csr_col + q)));
                    }
                }
        }
        const int32_t p0 = dia_ptr[ib], p1 = dia_ptr[ib + 1];
        const int64_t xw = r0 + t0 + (int64_t)warp * 32 * V;
        bool ok = true;
        int32_t p = p0;
        auto group = [&](auto Dc) {
            constexpr int DD = decltype(Dc)::value;
            XT xv[DD][U][V];
#pragma unroll
            for (int d = 0; d < DD; d++) {
                const int64_t off = dia_offset[p + d];
#pragma unroll
                for (int k = 0; k < U; k++) {
                    const int64_t jw = xw + (int64_t)k * NT * V + off;
                    if (full_unit && jw >= 0 && jw + 32 * V <= n) {
                        const int64_t j = jw + lane * V;
                        if ((reinterpret_cast<uintptr_t>(xs + jw) & 15) == 0) {
                            const uint4 r = __ldg(reinterpret_cast<const uint4 *>(xs + j));
                            memcpy(xv[d][k], &r, 16);
                        } else {
                            xv[d][k][0] = __ldg(xs + j);
                            xv[d][k][1] = __ldg(xs + j + 1);
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < V; m++) {
                            const int64_t jm = jw + lane * V + m;
                            if (tl[k] + m < ru && jm >= 0 && jm < n) xv[d][k][m] = __ldg(xs + jm);
                            else memset(&xv[d][k][m], 0, sizeof(XT));
                        }
                    }
                }
            }
#pragma unroll
            for (int d = 0; d < DD; d++) {
                int st = stage + d;
                uint32_t ph = phase;
                if (st >= STAGES) {
                    st -= STAGES;
                    ph ^= 1;
                }
                if (!mbar_wait(&full[st], ph)) ok = false;
            }
            if (!ok) return;
#pragma unroll
            for (int d = 0; d < DD; d++) {
                int st = stage + d;
                if (st >= STAGES) st -= STAGES;
                const uint8_t *sv = ring + (size_t)st * STAGE_BYTES;
#pragma unroll
                for (int k = 0; k < U; k++) {
                    const uint4 r = *reinterpret_cast<const uint4 *>(sv + (size_t)tl[k] * 8);
                    float2 v[V];
                    memcpy(v, &r, 16);
#pragma unroll
                    for (int m = 0; m < V; m++) dw::dw_fma(sh[k][m], sl[k][m], v[m], xv[d][k][m]);
                }
            }
            __syncwarp();
#pragma unroll
            for (int d = 0; d < DD; d++) {
                int st = stage + d;
                if (st >= STAGES) st -= STAGES;
                if (lane == 0) mbar_arrive(&empty[st]);
            }
            stage += DD;
            if (stage >= STAGES) {
                stage -= STAGES;
                phase ^= 1;
            }
            p += DD;
        };
        while (ok && p + D <= p1) group(std::integral_constant<int, D>{});
        while (ok && p < p1) group(std::integral_constant<int, 1>{});
        if (!ok) {
            if (lane == 0) atomicOr(status, 1);
            return;
        }
#pragma unroll
        for (int k = 0; k < U; k++)
#pragma unroll
            for (int m = 0; m < V; m++)
                if (tl[k] + m < ru) {
                    const int32_t t = t0 + tl[k] + m;
                    y[r0 + t] = isnan(sh[k][m])  // read an x outside the window
                                    ? native_row(r0 + t, t, ib, n, n_b, dia_ptr, dia_offset,
                                                 dia_val, csr_row_ptr, csr_col, csr_val, x)
                                    : dw::f32_to_f64(sh[k][m]) + dw::f32_to_f64(sl[k][m]);
                }
    }
}

template <int NCW, int U, int D, int STAGES>
__global__ void __launch_bounds__(NCW * 32 + 32)
k_mhdc_spmv_tma_dw(int64_t n, int32_t n_b, int32_t upb, int64_t n_units,
                   const int32_t *__restrict__ dia_ptr, const int32_t *__restrict__ dia_offset,
                   const double *__restrict__ dia_val, const float2 *__restrict__ dia_dw,
                   const int32_t *__restrict__ csr_row_ptr, const int32_t *__restrict__ csr_col,
                   const double *__restrict__ csr_val, const float2 *__restrict__ csr_dw,
                   const double *__restrict__ x, const float2 *__restrict__ x_dw,
                   double *__restrict__ y, int *__restrict__ status)
{
    constexpr int V = 2, NT = NCW * 32, R = NT * U * V, STAGE_BYTES = R * 8;
    extern __shared__ __align__(128) uint8_t ring[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == NCW) {
        if (lane != 0) return;
        const uint8_t *src = reinterpret_cast<const uint8_t *>(dia_dw);
        int stage = 0;
        uint32_t phase = 0;
        int64_t issued = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
            const int64_t ib = u / upb;
            const int32_t t0 = (int32_t)(u - ib * upb) * R;
            const int64_t r0 = ib * (int64_t)n_b;
            const int32_t rows = (int32_t)((n - r0 < n_b) ? (n - r0) : n_b);
            if (t0 >= rows) continue;
            const int32_t ru = (rows - t0 < R) ? rows - t0 : R;
            const uint32_t bytes = (uint32_t)(((int64_t)ru * 8 + 15) & ~(int64_t)15);
            const int32_t p0 = dia_ptr[ib], p1 = dia_ptr[ib + 1];
            for (int32_t p = p0; p < p1; p++) {
                if (!mbar_wait(&empty[stage], phase ^ 1)) {
                    atomicOr(status, 1);
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&full[stage], bytes);
                bulk_load(ring + (size_t)stage * STAGE_BYTES,
                          src + ((int64_t)p * n_b + t0) * 8, bytes, &full[stage]);
                issued++;
                if (++stage == STAGES) {
                    stage = 0;
                    phase ^= 1;
                }
            }
        }
        if (!ok) {
            const int64_t k = issued < STAGES ? issued : STAGES;
            for (int64_t q = 1; q <= k; q++) {
                int st = stage - (int)q;
                uint32_t ph = phase;
                if (st < 0) {
                    st += STAGES;
                    ph ^= 1;
                }
                mbar_wait(&full[st], ph);
            }
        }
        return;
    }
    tma_dw_consumer<NCW, U, D, STAGES>(n, n_b, upb, n_units, dia_ptr, dia_offset, dia_val,
                                       csr_row_ptr, csr_col, csr_val, csr_dw, x, x_dw, y, ring,
                                       full, empty, status);
}

template <int NCW, int U, int D, int STAGES>
int launch_tma_dw_cfg(mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t st)
{
    constexpr int R = NCW * 32 * U * 2, THREADS = NCW * 32 + 32;
    constexpr size_t SMEM = (size_t)STAGES * R * 8;
    auto kern = k_mhdc_spmv_tma_dw<NCW, U, D, STAGES>;
    static int occ = -1;
    if (occ < 0) {
        MHDC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)SMEM));
        int o = 0;
        MHDC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, THREADS, SMEM));
        occ = o > 0 ? o : 1;
    }
    const int32_t upb = (int32_t)((A->n_b + R - 1) / R);
    const int64_t units = (int64_t)upb * A->n_blocks;
    int64_t grid = (int64_t)num_sms_tma() * occ;
    if (grid > units) grid = units;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, THREADS, SMEM, st>>>(
        A->n, A->n_b, upb, units, A->dia_ptr, A->dia_offset, (const double *)A->dia_val,
        A->dia_dw, A->csr_row_ptr, A->csr_col, (const double *)A->csr_val, A->csr_dw,
        (const double *)d_x, A->x_dw, (double *)d_y, A->status);
    MHDC_LAUNCH_CHECK("k_mhdc_spmv_tma_dw");
    return MHDC_OK;
}

int num_sms_tma()
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

template <typename VT, int NCW, int U, int D, int STAGES>
int launch_tma_cfg(const mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t st)
{
    using Cf = TmaCfg<VT, NCW, U, D, STAGES>;
    auto kern = k_mhdc_spmv_tma<VT, NCW, U, D, STAGES>;
    static int occ = -1;
    if (occ < 0) {
        MHDC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)Cf::SMEM));
        int o = 0;
        MHDC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, Cf::THREADS, Cf::SMEM));
        occ = o > 0 ? o : 1;
    }
    const int32_t upb = (int32_t)((A->n_b + Cf::R - 1) / Cf::R);
    const int64_t units = (int64_t)upb * A->n_blocks;
    int64_t grid = (int64_t)num_sms_tma() * occ;
    if (grid > units) grid = units;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, Cf::THREADS, Cf::SMEM, st>>>(
        A->n, A->n_b, upb, units, A->dia_ptr, A->dia_offset, static_cast<const VT *>(A->dia_val),
        A->csr_row_ptr, A->csr_col, static_cast<const VT *>(A->csr_val),
        static_cast<const typename TrT<VT>::X *>(d_x), static_cast<typename TrT<VT>::Y *>(d_y),
        A->status);
    MHDC_LAUNCH_CHECK("k_mhdc_spmv_tma");
    return MHDC_OK;
}

template <typename VT>
int launch_tma_typed(const mhdc_matrix *A, int shape, const void *d_x, void *d_y, cudaStream_t st)
{
    switch (shape) {
    case 0: return launch_tma_cfg<VT, 4, 2, 1, 16>(A, d_x, d_y, st);
    case 1: return launch_tma_cfg<VT, 4, 2, 2, 16>(A, d_x, d_y, st);
    case 2: return launch_tma_cfg<VT, 8, 1, 2, 16>(A, d_x, d_y, st);
    default: return launch_tma_cfg<VT, 4, 1, 2, 24>(A, d_x, d_y, st);
    }
}

template <typename VT, int NCW, int U, int DSTAGES, int XSTAGES>
int launch_xw_cfg(const mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t st)
{
    using Cf = XwCfg<VT, NCW, U, DSTAGES, XSTAGES>;
    auto kern = k_mhdc_spmv_xw<VT, NCW, U, DSTAGES, XSTAGES>;
    static int occ = -1;
    if (occ < 0) {
        MHDC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)Cf::SMEM));
        int o = 0;
        MHDC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, Cf::THREADS, Cf::SMEM));
        occ = o > 0 ? o : 1;
    }
    const int32_t upb = (int32_t)((A->n_b + Cf::R - 1) / Cf::R);
    const int64_t units = (int64_t)upb * A->n_blocks;
    int64_t grid = (int64_t)num_sms_tma() * occ;
    if (grid > units) grid = units;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, Cf::THREADS, Cf::SMEM, st>>>(
        A->n, A->n_b, upb, units, A->dia_ptr, A->dia_offset, static_cast<const VT *>(A->dia_val),
        A->csr_row_ptr, A->csr_col, static_cast<const VT *>(A->csr_val),
        static_cast<const typename TrT<VT>::X *>(d_x), static_cast<typename TrT<VT>::Y *>(d_y),
        A->status);
    MHDC_LAUNCH_CHECK("k_mhdc_spmv_xw");
    return MHDC_OK;
}

// (consumer warps, vectors per lane, value stages, x windows)
template <typename VT>
int launch_xw_typed(const mhdc_matrix *A, int shape, const void *d_x, void *d_y, cudaStream_t st)
{
    switch (shape) {
    case 0: return launch_xw_cfg<VT, 4, 2, 8, 4>(A, d_x, d_y, st);
    case 1: return launch_xw_cfg<VT, 8, 1, 8, 4>(A, d_x, d_y, st);
    case 2: return launch_xw_cfg<VT, 4, 1, 12, 6>(A, d_x, d_y, st);
    default: return launch_xw_cfg<VT, 8, 2, 6, 3>(A, d_x, d_y, st);
    }
}

}  // namespace

int launch_spmv_tma_dw(mhdc_matrix *A, int shape, const void *d_x, void *d_y,
                       cudaStream_t stream)
{
    switch (shape) {
    case 0: return launch_tma_dw_cfg<8, 1, 2, 16>(A, d_x, d_y, stream);
    case 1: return launch_tma_dw_cfg<4, 2, 2, 16>(A, d_x, d_y, stream);
    default: return launch_tma_dw_cfg<8, 1, 1, 24>(A, d_x, d_y, stream);
    }
}

bool tma_supported(const mhdc_matrix *A)
{
    return (A->n_b * (int64_t)value_size(A->dtype)) % 16 == 0;
}

bool xw_supported(const mhdc_matrix *A, const void *d_x)
{
    return tma_supported(A) && (reinterpret_cast<uintptr_t>(d_x) & 15) == 0;
}

int launch_spmv_xw(const mhdc_matrix *A, int shape, const void *d_x, void *d_y,
                   cudaStream_t stream)
{
    switch (A->dtype) {
    case MHDC_F64: return launch_xw_typed<double>(A, shape, d_x, d_y, stream);
    case MHDC_F32: return launch_xw_typed<float>(A, shape, d_x, d_y, stream);
    default: return launch_xw_typed<__nv_bfloat16>(A, shape, d_x, d_y, stream);
    }
}

int launch_spmv_tma(const mhdc_matrix *A, int shape, const void *d_x, void *d_y,
                    cudaStream_t stream)
{
    switch (A->dtype) {
    case MHDC_F64: return launch_tma_typed<double>(A, shape, d_x, d_y, stream);
    case MHDC_F32: return launch_tma_typed<float>(A, shape, d_x, d_y, stream);
    default: return launch_tma_typed<__nv_bfloat16>(A, shape, d_x, d_y, stream);
    }
}

}  // namespace mhdc
