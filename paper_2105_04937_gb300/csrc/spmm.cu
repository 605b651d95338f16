// SpMM: Y = A X for k right-hand sides (row-major X, Y), the M-HDC kernel of
// Fig. 13 with each scalar x_j replaced by row j of X.
//
// Work split.  A pass covers KC consecutive columns of X and Y.  The KC
// entries of one row of X are QV * L elements: L lanes each load one slice of
// QV elements (16 bytes when KC is wide enough), so G = 32 / L consecutive
// rows of X form one contiguous run of G * KC elements per warp load -- every
// byte a warp fetches through L1 is used (a lane-per-row layout instead reads
// 16 bytes out of every KC-element row per load and wastes most of each
// line).  A warp tile is RW = G * U rows of one row block; lane (g, c) owns
// columns [c * QV, c * QV + QV) of the pass and U rows of the tile, either
// strided (tw + g + G u: per diagonal one value and one X slice per row, D
// diagonals loaded before their FMAs) or consecutive (tw + g U + u: a run of
// consecutive offsets shares X rows between its diagonals, see the run
// tiles below).  Each (row, column) accumulates the CSR remainder first, in
// column order, then the diagonals in ascending order: the operations of the
// SpMV kernel, whatever the tile.
#include <cstring>
#include <type_traits>

#include "mhdc_internal.cuh"

namespace mhdc {
namespace {

template <typename VT>
struct MmTr;
template <>
struct MmTr<double> {
    using X = double;
    using Y = double;
    using Acc = double;
};
template <>
struct MmTr<float> {
    using X = float;
    using Y = float;
    using Acc = float;
};
template <>
struct MmTr<__nv_bfloat16> {
    using X = __nv_bfloat16;
    using Y = float;
    using Acc = float;
};

__device__ __forceinline__ double wd(double v) { return v; }
__device__ __forceinline__ float wd(float v) { return v; }
__device__ __forceinline__ float wd(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double mm_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mm_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// N contiguous elements at p: one load of N * sizeof(T) bytes (16, 8, 4 or 2,
// aligned to that size) when vec, else element loads of the first lim ones
// (0 for the rest).
template <typename T, int N>
__device__ __forceinline__ void ld_slice(const T *__restrict__ p, bool vec, int lim, T (&v)[N])
{
    constexpr int B = N * (int)sizeof(T);
    if (vec) {
        if constexpr (B == 16) {
            const uint4 r = __ldg(reinterpret_cast<const uint4 *>(p));
            memcpy(v, &r, 16);
            return;
        } else if constexpr (B == 8) {
            const uint2 r = __ldg(reinterpret_cast<const uint2 *>(p));
            memcpy(v, &r, 8);
            return;
        } else if constexpr (B == 4) {
            const unsigned r = __ldg(reinterpret_cast<const unsigned *>(p));
            memcpy(v, &r, 4);
            return;
        } else if constexpr (B == 2) {
            const unsigned short r = __ldg(reinterpret_cast<const unsigned short *>(p));
            memcpy(v, &r, 2);
            return;
        }
    }
#pragma unroll
    for (int m = 0; m < N; m++) v[m] = m < lim ? __ldg(p + m) : T(0);
}

// N contiguous results to p: 16-byte stores (or one store of N * sizeof(T)
// bytes below 16) when vec, else element stores of the first lim ones.
template <typename T, int N>
__device__ __forceinline__ void st_slice(T *__restrict__ p, bool vec, int lim, const T (&v)[N])
{
    constexpr int B = N * (int)sizeof(T);
    if (vec) {
        if constexpr (B >= 16) {
#pragma unroll
            for (int q = 0; q < B / 16; q++) {
                uint4 r;
                memcpy(&r, reinterpret_cast<const char *>(v) + 16 * q, 16);
                reinterpret_cast<uint4 *>(p)[q] = r;
            }
            return;
        } else if constexpr (B == 8) {
            uint2 r;
            memcpy(&r, v, 8);
            *reinterpret_cast<uint2 *>(p) = r;
            return;
        } else if constexpr (B == 4) {
            unsigned r;
            memcpy(&r, v, 4);
            *reinterpret_cast<unsigned *>(p) = r;
            return;
        }
    }
#pragma unroll
    for (int m = 0; m < N; m++)
        if (m < lim) p[m] = v[m];
}

constexpr int MM_THREADS = 256;
constexpr int MM_WARPS = MM_THREADS / 32;
// Resident CTAs per SM the tile shapes are compiled for (4: 64 registers a
// thread); latency-bound, so occupancy first, more registers for larger tiles.
constexpr int mm_min_blocks(int U, int D) { return U * D <= 4 ? 4 : 3; }

template <typename X, int KC>
struct Slice {
    static constexpr int QV = (KC * (int)sizeof(X) >= 16) ? 16 / (int)sizeof(X) : KC;
    static constexpr int L = KC / QV;  // lanes per row of X
    static constexpr int G = 32 / L;   // rows of X per warp load
};

// CSR remainder rows (Fig. 13, first loop) of the lane's rows t[u] into
// acc: each row in column order from zero; a row longer than REM_LONG under
// FP32 accumulation is summed per column in FP64 and rounded once, as
// rem_row_add does for one column.
template <typename VT, int KC, int U>
__device__ __forceinline__ void
mm_remainder(const int32_t (&t)[U], int32_t tw, int32_t tend, int32_t rows, int64_t r0,
             const int32_t *__restrict__ csr_row_ptr, const int32_t *__restrict__ csr_col,
             const VT *__restrict__ csr_val, const typename MmTr<VT>::X *__restrict__ xs,
             int64_t ldx, bool xvec, int lim,
             typename MmTr<VT>::Acc (&acc)[U][Slice<typename MmTr<VT>::X, KC>::QV])
{
    using X = typename MmTr<VT>::X;
    using Acc = typename MmTr<VT>::Acc;
    constexpr int QV = Slice<X, KC>::QV;
    if (csr_row_ptr[r0 + tw] == csr_row_ptr[r0 + tend]) return;  // warp-uniform
#pragma unroll
    for (int u = 0; u < U; u++) {
        if (t[u] >= rows) continue;
        const int64_t i = r0 + t[u];
        const int32_t a = csr_row_ptr[i], b = csr_row_ptr[i + 1];
        if constexpr (sizeof(Acc) < sizeof(double)) {
            if (b - a > REM_LONG) {
#pragma unroll
                for (int m = 0; m < QV; m++) {
                    if (m >= lim) continue;
                    double s = 0.0;
                    for (int32_t q = a; q < b; q++)
                        s = fma((double)wd(csr_val[q]),
                                (double)wd(__ldg(xs + (int64_t)csr_col[q] * ldx + m)), s);
                    acc[u][m] = (Acc)s;
                }
                continue;
            }
        }
        for (int32_t q = a; q < b; q++) {
            const Acc av = wd(csr_val[q]);
            X xv[QV];
            ld_slice<X, QV>(xs + (int64_t)csr_col[q] * ldx, xvec, lim, xv);
#pragma unroll
            for (int m = 0; m < QV; m++) acc[u][m] = mm_fma(av, wd(xv[m]), acc[u][m]);
        }
    }
}

// Y rows t[u] of the lane's slice from acc.
template <typename VT, int KC, int U>
__device__ __forceinline__ void
mm_store(const int32_t (&t)[U], int32_t rows, int64_t r0, typename MmTr<VT>::Y *__restrict__ ys,
         int64_t ldy, bool yvec, int lim,
         const typename MmTr<VT>::Acc (&acc)[U][Slice<typename MmTr<VT>::X, KC>::QV])
{
    using Y = typename MmTr<VT>::Y;
    constexpr int QV = Slice<typename MmTr<VT>::X, KC>::QV;
    if (lim <= 0) return;
#pragma unroll
    for (int u = 0; u < U; u++) {
        if (t[u] >= rows) continue;
        Y out[QV];
#pragma unroll
        for (int m = 0; m < QV; m++) out[m] = (Y)acc[u][m];
        st_slice<Y, QV>(ys + (r0 + t[u]) * ldy, yvec, lim, out);
    }
}

template <typename VT, int KC, int U, int D>
__global__ void __launch_bounds__(MM_THREADS, mm_min_blocks(U, D))
k_mhdc_spmm(int64_t n, int32_t n_b, int32_t tpb, int64_t n_tiles, int32_t c0, int32_t k,
            const int32_t *__restrict__ dia_ptr, const int32_t *__restrict__ dia_offset,
            const VT *__restrict__ dia_val, const int32_t *__restrict__ csr_row_ptr,
            const int32_t *__restrict__ csr_col, const VT *__restrict__ csr_val,
            const typename MmTr<VT>::X *__restrict__ Xm, int64_t ldx,
            typename MmTr<VT>::Y *__restrict__ Ym, int64_t ldy)
{
    using X = typename MmTr<VT>::X;
    using Y = typename MmTr<VT>::Y;
    using Acc = typename MmTr<VT>::Acc;
    constexpr int QV = Slice<X, KC>::QV, L = Slice<X, KC>::L, G = Slice<X, KC>::G;
    constexpr int RW = G * U;
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * MM_WARPS + (threadIdx.x >> 5);
    if (w >= n_tiles) return;
    const int64_t ib = w / tpb;
    const int32_t tw = (int32_t)(w - ib * tpb) * RW;
    const int64_t r0 = ib * (int64_t)n_b;
    const int32_t rows = (int32_t)((n - r0 < n_b) ? (n - r0) : n_b);
    if (tw >= rows) return;  // warp-uniform
    const int g = lane / L;
    const int cq = (lane % L) * QV;  // first column of this lane's slice in the pass
    const int kc = (k - c0 < KC) ? k - c0 : KC;
    const int lim = kc - cq;  // columns of the slice inside the pass (<= 0: none)
    constexpr int BX = QV * (int)sizeof(X);
    constexpr int BY = (QV * (int)sizeof(Y) >= 16) ? 16 : QV * (int)sizeof(Y);
    const bool xvec = kc == KC && (reinterpret_cast<uintptr_t>(Xm + c0) % BX) == 0 &&
                      ((ldx * (int64_t)sizeof(X)) % BX) == 0;
    const bool yvec = kc == KC && (reinterpret_cast<uintptr_t>(Ym + c0) % BY) == 0 &&
                      ((ldy * (int64_t)sizeof(Y)) % BY) == 0;
    const X *__restrict__ xs = Xm + c0 + cq;

    int32_t t[U];
#pragma unroll
    for (int u = 0; u < U; u++) t[u] = tw + g + G * u;
    Acc acc[U][QV];
#pragma unroll
    for (int u = 0; u < U; u++)
#pragma unroll
        for (int m = 0; m < QV; m++) acc[u][m] = Acc(0);

    const int32_t p0 = dia_ptr[ib], p1 = dia_ptr[ib + 1];

    mm_remainder<VT, KC, U>(t, tw, (tw + RW < rows) ? tw + RW : rows, rows, r0, csr_row_ptr, csr_col,
                            csr_val, xs, ldx, xvec, lim, acc);

    // the block's partial diagonals (Fig. 13, second loop), D at a time.
    // Addresses: the lane's X row pointers are set once; per diagonal only
    // off * ldx (warp-uniform) is added.  Tiles at the matrix edge (a row of
    // the tile outside the matrix, or an X row outside [0, n) for some
    // diagonal) check every row of every group.
    const X *__restrict__ xr[U];
#pragma unroll
    for (int u = 0; u < U; u++) xr[u] = xs + (r0 + t[u]) * ldx;
    const bool full = tw + RW <= rows;
    const int64_t jlo = r0 + tw, jhi = r0 + tw + RW;  // the tile's rows, [jlo, jhi)
    int32_t p = p0;
    auto group = [&](auto Dc) {
        constexpr int DD = decltype(Dc)::value;
        int64_t off[DD];
#pragma unroll
        for (int d = 0; d < DD; d++) off[d] = dia_offset[p + d];
        Acc v[DD][U];
        X xv[DD][U][QV];
#pragma unroll
        for (int d = 0; d < DD; d++)
#pragma unroll
            for (int u = 0; u < U; u++)
                v[d][u] = t[u] < rows ? wd(dia_val[(int64_t)(p + d) * n_b + t[u]]) : Acc(0);
#pragma unroll
        for (int d = 0; d < DD; d++)
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t j = r0 + t[u] + off[d];
                if (t[u] < rows && j >= 0 && j < n) {
                    ld_slice<X, QV>(xs + j * ldx, xvec, lim, xv[d][u]);
                } else {
#pragma unroll
                    for (int m = 0; m < QV; m++) xv[d][u][m] = X(0);
                }
            }
#pragma unroll
        for (int d = 0; d < DD; d++)
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int m = 0; m < QV; m++) acc[u][m] = mm_fma(v[d][u], wd(xv[d][u][m]), acc[u][m]);
        p += DD;
    };
    // the block's offsets ascend, so its first and last diagonal bound the
    // X rows of the whole tile: a tile inside [0, n) for all of them runs a
    // loop without per-group checks, the value pointer advanced per group
    bool all_in = full && xvec && p1 > p0;
    if (all_in) {
        const int64_t omin = dia_offset[p0], omax = dia_offset[p1 - 1];
        all_in = jlo + omin >= 0 && jhi + omax <= n;
    }
    if (all_in) {
        const VT *vp = dia_val + (int64_t)p0 * n_b + tw + g;
        auto fgroup = [&](auto Dc) {
            constexpr int DD = decltype(Dc)::value;
            int64_t xo[DD];
#pragma unroll
            for (int d = 0; d < DD; d++) xo[d] = (int64_t)dia_offset[p + d] * ldx;
            Acc v[DD][U];
            X xv[DD][U][QV];
#pragma unroll
            for (int d = 0; d < DD; d++)
#pragma unroll
                for (int u = 0; u < U; u++) v[d][u] = wd(vp[(int64_t)d * n_b + G * u]);
#pragma unroll
            for (int d = 0; d < DD; d++)
#pragma unroll
                for (int u = 0; u < U; u++) ld_slice<X, QV>(xr[u] + xo[d], true, QV, xv[d][u]);
#pragma unroll
            for (int d = 0; d < DD; d++)
#pragma unroll
                for (int u = 0; u < U; u++)
#pragma unroll
                    for (int m = 0; m < QV; m++)
                        acc[u][m] = mm_fma(v[d][u], wd(xv[d][u][m]), acc[u][m]);
            p += DD;
            vp += (int64_t)DD * n_b;
        };
        for (; p + D <= p1;) fgroup(std::integral_constant<int, D>{});
        for (; p < p1;) fgroup(std::integral_constant<int, 1>{});
    } else {
        for (; p + D <= p1;) group(std::integral_constant<int, D>{});
        for (; p < p1;) group(std::integral_constant<int, 1>{});
    }

    mm_store<VT, KC, U>(t, rows, r0, Ym + c0 + cq, ldy, yvec, lim, acc);
}

// Run tiles: lane (g, c) owns the U consecutive rows tw + g U + u (u < U).
// For a run of MM consecutive offsets off, off + 1, ..., the lane's rows need
// X rows off .. off + U + MM - 2 past its first row, so U + MM - 1 slice loads
// serve MM U (row, diagonal) pairs -- a stencil's runs of three offsets
// (off - 1, off, off + 1) load each X row once instead of three times.  Runs
// are found from dia_offset as the tile walks its diagonals (at most three
// a run).  Every accumulator still adds its diagonals in ascending order:
// the same Y as the other shapes.
// Resident CTAs per SM: four (64 registers) where the run's values, X rows
// and accumulators fit without spilling (FP32 up to U = 4, FP64 up to U = 3),
// else three (80 registers; BF16 slices widen to eight FP32 values).
constexpr int mm_run_min_blocks(int U, int vt_bytes)
{
    return (vt_bytes == 4 && U <= 4) || (vt_bytes == 8 && U <= 3) ? 4 : 3;
}

template <typename VT, int KC, int U>
__global__ void __launch_bounds__(MM_THREADS, mm_run_min_blocks(U, (int)sizeof(VT)))
k_mhdc_spmm_run(int64_t n, int32_t n_b, int32_t tpb, int64_t n_tiles, int32_t c0, int32_t k,
                const int32_t *__restrict__ dia_ptr, const int32_t *__restrict__ dia_offset,
                const VT *__restrict__ dia_val, const int32_t *__restrict__ csr_row_ptr,
                const int32_t *__restrict__ csr_col, const VT *__restrict__ csr_val,
                const typename MmTr<VT>::X *__restrict__ Xm, int64_t ldx,
                typename MmTr<VT>::Y *__restrict__ Ym, int64_t ldy)
{
    using X = typename MmTr<VT>::X;
    using Y = typename MmTr<VT>::Y;
    using Acc = typename MmTr<VT>::Acc;
    constexpr int QV = Slice<X, KC>::QV, L = Slice<X, KC>::L, G = Slice<X, KC>::G;
    constexpr int RW = G * U;
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * MM_WARPS + (threadIdx.x >> 5);
    if (w >= n_tiles) return;
    const int64_t ib = w / tpb;
    const int32_t tw = (int32_t)(w - ib * tpb) * RW;
    const int64_t r0 = ib * (int64_t)n_b;
    const int32_t rows = (int32_t)((n - r0 < n_b) ? (n - r0) : n_b);
    if (tw >= rows) return;  // warp-uniform
    const int g = lane / L;
    const int cq = (lane % L) * QV;
    const int kc = (k - c0 < KC) ? k - c0 : KC;
    const int lim = kc - cq;
    constexpr int BX = QV * (int)sizeof(X);
    constexpr int BY = (QV * (int)sizeof(Y) >= 16) ? 16 : QV * (int)sizeof(Y);
    const bool xvec = kc == KC && (reinterpret_cast<uintptr_t>(Xm + c0) % BX) == 0 &&
                      ((ldx * (int64_t)sizeof(X)) % BX) == 0;
    const bool yvec = kc == KC && (reinterpret_cast<uintptr_t>(Ym + c0) % BY) == 0 &&
                      ((ldy * (int64_t)sizeof(Y)) % BY) == 0;
    const X *__restrict__ xs = Xm + c0 + cq;

    int32_t t[U];
#pragma unroll
    for (int u = 0; u < U; u++) t[u] = tw + g * U + u;
    Acc acc[U][QV];
#pragma unroll
    for (int u = 0; u < U; u++)
#pragma unroll
        for (int m = 0; m < QV; m++) acc[u][m] = Acc(0);
    const int32_t p0 = dia_ptr[ib], p1 = dia_ptr[ib + 1];
    mm_remainder<VT, KC, U>(t, tw, (tw + RW < rows) ? tw + RW : rows, rows, r0, csr_row_ptr, csr_col,
                            csr_val, xs, ldx, xvec, lim, acc);

    const bool full = tw + RW <= rows;
    const int64_t jlo = r0 + tw, jhi = r0 + tw + RW;  // the tile's rows, [jlo, jhi)
    int32_t p = p0;
    // ascending offsets: the first and last diagonal bound the tile's X rows
    bool all_in = full && xvec && p1 > p0;
    if (all_in) {
        const int64_t omin = dia_offset[p0], omax = dia_offset[p1 - 1];
        all_in = jlo + omin >= 0 && jhi + omax <= n;
    }
    if (all_in) {
        const X *xb = xs + (r0 + tw + g * U) * ldx;  // the lane's first row at offset 0
        const VT *vb = dia_val + tw + g * U;
        // the lane's U values of a diagonal in one load when they are aligned
        const bool vvec = (U & (U - 1)) == 0 && (n_b % U) == 0;
        auto run = [&](auto Mc, int32_t off) {
            constexpr int MM = decltype(Mc)::value;
            VT v[MM][U];
            X xv[U + MM - 1][QV];
            const VT *vp = vb + (int64_t)p * n_b;
#pragma unroll
            for (int d = 0; d < MM; d++) ld_slice<VT, U>(vp + (int64_t)d * n_b, vvec, U, v[d]);
            const X *xp = xb + (int64_t)off * ldx;
#pragma unroll
            for (int j = 0; j < U + MM - 1; j++)
                ld_slice<X, QV>(xp + (int64_t)j * ldx, true, QV, xv[j]);
#pragma unroll
            for (int d = 0; d < MM; d++)
#pragma unroll
                for (int u = 0; u < U; u++)
#pragma unroll
                    for (int m = 0; m < QV; m++)
                        acc[u][m] = mm_fma(wd(v[d][u]), wd(xv[u + d][m]), acc[u][m]);
            p += MM;
        };
        while (p < p1) {
            const int32_t o0 = dia_offset[p];
            int m = 1;
            if (p + 1 < p1 && dia_offset[p + 1] == o0 + 1) {
                m = 2;
                if (p + 2 < p1 && dia_offset[p + 2] == o0 + 2) m = 3;
            }
            if (m == 3) run(std::integral_constant<int, 3>{}, o0);
            else if (m == 2) run(std::integral_constant<int, 2>{}, o0);
            else run(std::integral_constant<int, 1>{}, o0);
        }
    } else {
        // edge tiles: one diagonal at a time, every row checked
        for (; p < p1; p++) {
            const int64_t off = dia_offset[p];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const Acc v = t[u] < rows ? wd(dia_val[(int64_t)p * n_b + t[u]]) : Acc(0);
                const int64_t j = r0 + t[u] + off;
                X xv[QV];
                if (t[u] < rows && j >= 0 && j < n) {
                    ld_slice<X, QV>(xs + j * ldx, xvec, lim, xv);
                } else {
#pragma unroll
                    for (int m = 0; m < QV; m++) xv[m] = X(0);
                }
#pragma unroll
                for (int m = 0; m < QV; m++) acc[u][m] = mm_fma(v, wd(xv[m]), acc[u][m]);
            }
        }
    }
    mm_store<VT, KC, U>(t, rows, r0, Ym + c0 + cq, ldy, yvec, lim, acc);
}

// Tile shapes; index = the handle's SpMM variant: 0, 2, 3 run tiles with
// U = 3, 4, 5 rows per lane, 1 the strided tile (U, D) = (2, 2), which keeps
// two diagonals' loads in flight where a matrix has no runs of offsets.
// Passes of one or two columns use the strided tile (2, 4) only.
constexpr int SPMM_DEFAULT = 2;

template <typename VT, int KC, int U, int D>
int spmm_pass(const mhdc_matrix *A, int32_t c0, int32_t k, const void *X, int64_t ldx, void *Y,
              int64_t ldy, cudaStream_t st)
{
    using XT = typename MmTr<VT>::X;
    constexpr int RW = Slice<XT, KC>::G * U;
    const int32_t tpb = (int32_t)((A->n_b + RW - 1) / RW);
    const int64_t tiles = (int64_t)tpb * A->n_blocks;
    const int64_t grid = (tiles + MM_WARPS - 1) / MM_WARPS;
    k_mhdc_spmm<VT, KC, U, D><<<(unsigned)grid, MM_THREADS, 0, st>>>(
        A->n, A->n_b, tpb, tiles, c0, k, A->dia_ptr, A->dia_offset,
        static_cast<const VT *>(A->dia_val), A->csr_row_ptr, A->csr_col,
        static_cast<const VT *>(A->csr_val), static_cast<const XT *>(X), ldx,
        static_cast<typename MmTr<VT>::Y *>(Y), ldy);
    MHDC_LAUNCH_CHECK("k_mhdc_spmm");
    return MHDC_OK;
}

template <typename VT, int KC, int U>
int spmm_run_pass(const mhdc_matrix *A, int32_t c0, int32_t k, const void *X, int64_t ldx, void *Y,
                  int64_t ldy, cudaStream_t st)
{
    using XT = typename MmTr<VT>::X;
    constexpr int RW = Slice<XT, KC>::G * U;
    const int32_t tpb = (int32_t)((A->n_b + RW - 1) / RW);
    const int64_t tiles = (int64_t)tpb * A->n_blocks;
    const int64_t grid = (tiles + MM_WARPS - 1) / MM_WARPS;
    k_mhdc_spmm_run<VT, KC, U><<<(unsigned)grid, MM_THREADS, 0, st>>>(
        A->n, A->n_b, tpb, tiles, c0, k, A->dia_ptr, A->dia_offset,
        static_cast<const VT *>(A->dia_val), A->csr_row_ptr, A->csr_col,
        static_cast<const VT *>(A->csr_val), static_cast<const XT *>(X), ldx,
        static_cast<typename MmTr<VT>::Y *>(Y), ldy);
    MHDC_LAUNCH_CHECK("k_mhdc_spmm_run");
    return MHDC_OK;
}

template <typename VT, int KC>
int spmm_shape(int v, const mhdc_matrix *A, int32_t c0, int32_t k, const void *X, int64_t ldx,
               void *Y, int64_t ldy, cudaStream_t st)
{
    if constexpr (KC <= 2) {
        return spmm_pass<VT, KC, 2, 4>(A, c0, k, X, ldx, Y, ldy, st);
    } else {
        switch (v) {
        case 0: return spmm_run_pass<VT, KC, 3>(A, c0, k, X, ldx, Y, ldy, st);
        case 1: return spmm_pass<VT, KC, 2, 2>(A, c0, k, X, ldx, Y, ldy, st);
        case 3: return spmm_run_pass<VT, KC, 5>(A, c0, k, X, ldx, Y, ldy, st);
        default: return spmm_run_pass<VT, KC, 4>(A, c0, k, X, ldx, Y, ldy, st);
        }
    }
}

template <typename VT>
int spmm_typed(const mhdc_matrix *A, int v, int k, const void *X, int64_t ldx, void *Y,
               int64_t ldy, cudaStream_t st)
{
    // column passes of at most 16; the pass width follows k (a ragged last
    // pass loads and stores element by element)
    for (int32_t c0 = 0; c0 < k; c0 += 16) {
        const int kc = (k - c0 < 16) ? k - c0 : 16;
        int rc;
        if (kc > 8) rc = spmm_shape<VT, 16>(v, A, c0, k, X, ldx, Y, ldy, st);
        else if (kc > 4) rc = spmm_shape<VT, 8>(v, A, c0, k, X, ldx, Y, ldy, st);
        else if (kc > 2) rc = spmm_shape<VT, 4>(v, A, c0, k, X, ldx, Y, ldy, st);
        else if (kc > 1) rc = spmm_shape<VT, 2>(v, A, c0, k, X, ldx, Y, ldy, st);
        else rc = spmm_shape<VT, 1>(v, A, c0, k, X, ldx, Y, ldy, st);
        if (rc != MHDC_OK) return rc;
    }
    return MHDC_OK;
}

int spmm_variant(const mhdc_matrix *A, int v, int k, const void *X, int64_t ldx, void *Y,
                 int64_t ldy, cudaStream_t st)
{
    if (v < 0 || v >= MHDC_NUM_SPMM_VARIANTS) v = SPMM_DEFAULT;
    switch (A->dtype) {
    case MHDC_F64: return spmm_typed<double>(A, v, k, X, ldx, Y, ldy, st);
    case MHDC_F32: return spmm_typed<float>(A, v, k, X, ldx, Y, ldy, st);
    default: return spmm_typed<__nv_bfloat16>(A, v, k, X, ldx, Y, ldy, st);
    }
}

}  // namespace

int launch_spmm(mhdc_matrix *A, int k, const void *d_X, int64_t ldx, void *d_Y, int64_t ldy,
                cudaStream_t stream)
{
    if (A->n == 0) return MHDC_OK;
    if (k == 1 && ldx == 1 && ldy == 1) return launch_spmv(A, d_X, d_Y, stream);
    return spmm_variant(A, A->spmm_variant, k, d_X, ldx, d_Y, ldy, stream);
}

int tune_spmm(mhdc_matrix *A, int k, const void *d_X, int64_t ldx, void *d_Y, int64_t ldy,
              cudaStream_t stream, int32_t *best, float *times_us)
{
    if (A->n == 0) {
        if (best) *best = -1;
        return MHDC_OK;
    }
    cudaEvent_t e0, e1;
    MHDC_CUDA_TRY(cudaEventCreate(&e0));
    MHDC_CUDA_TRY(cudaEventCreate(&e1));
    int best_v = -1;
    float best_t = 0.f;
    const int reps = 10;
    int rc = MHDC_OK;
    for (int v = 0; v < MHDC_NUM_SPMM_VARIANTS && rc == MHDC_OK; v++) {
        for (int r = 0; r < 2 && rc == MHDC_OK; r++)
            rc = spmm_variant(A, v, k, d_X, ldx, d_Y, ldy, stream);
        cudaEventRecord(e0, stream);
        for (int r = 0; r < reps && rc == MHDC_OK; r++)
            rc = spmm_variant(A, v, k, d_X, ldx, d_Y, ldy, stream);
        cudaEventRecord(e1, stream);
        if (rc != MHDC_OK) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            set_error("cudaEventSynchronize", e);
            rc = MHDC_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const float us = ms * 1e3f / reps;
        if (times_us) times_us[v] = us;
        if (best_v < 0 || us < best_t) {
            best_v = v;
            best_t = us;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MHDC_OK) return rc;
    A->spmm_variant = best_v;
    if (best) *best = best_v;
    return MHDC_OK;
}

}  // namespace mhdc
