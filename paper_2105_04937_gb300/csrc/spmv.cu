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
// accumulates in registers; y is written once.  A persistent grid of
// (SMs x resident CTAs) walks the tiles.
#include <cstring>

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

template <typename VT, int U, bool VEC>
__global__ void __launch_bounds__(SPMV_THREADS)
k_mhdc_spmv(int64_t n, int32_t n_b, int32_t tpb, int64_t n_tiles,
            const int32_t *__restrict__ dia_ptr, const int32_t *__restrict__ dia_offset,
            const VT *__restrict__ dia_val, const int32_t *__restrict__ csr_row_ptr,
            const int32_t *__restrict__ csr_col, const VT *__restrict__ csr_val,
            const typename Tr<VT>::X *__restrict__ x, typename Tr<VT>::Y *__restrict__ y)
{
    using Acc = typename Tr<VT>::Acc;
    using X = typename Tr<VT>::X;
    constexpr int V = VEC ? Tr<VT>::V : 1;
    constexpr int RW = 32 * V * U;
    const int lane = threadIdx.x & 31;
    const bool x_vec = VEC && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    const int64_t wstride = (int64_t)gridDim.x * SPMV_WARPS;
    for (int64_t w = (int64_t)blockIdx.x * SPMV_WARPS + (threadIdx.x >> 5); w < n_tiles;
         w += wstride) {
        const int64_t ib = w / tpb;
        const int32_t tw = (int32_t)(w - ib * tpb) * RW;
        const int64_t r0 = ib * (int64_t)n_b;
        const int32_t rows = (int32_t)((n - r0 < n_b) ? (n - r0) : n_b);
        if (tw >= rows) continue;  // warp-uniform

        Acc acc[U][V];
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
            for (int m = 0; m < V; m++) acc[u][m] = Acc(0);

        // CSR remainder rows of the tile (Fig. 13, first loop)
        const int32_t tend = (tw + RW < rows) ? (tw + RW) : rows;
        const int32_t q0 = csr_row_ptr[r0 + tw], q1 = csr_row_ptr[r0 + tend];
        if (q0 != q1) {
#pragma unroll
            for (int u = 0; u < U; u++) {
#pragma unroll
                for (int m = 0; m < V; m++) {
                    const int32_t t = tw + (u * 32 + lane) * V + m;
                    if (t < rows) {
                        const int64_t i = r0 + t;
                        const int32_t a = csr_row_ptr[i], b = csr_row_ptr[i + 1];
                        for (int32_t k = a; k < b; k++)
                            acc[u][m] += widen(csr_val[k]) * widen(ldg_elem(x + csr_col[k]));
                    }
                }
            }
        }

        // the block's partial diagonals (Fig. 13, second loop)
        const int32_t p0 = dia_ptr[ib], p1 = dia_ptr[ib + 1];
#pragma unroll 2
        for (int32_t p = p0; p < p1; p++) {
            const int64_t off = dia_offset[p];
            const VT *vp = dia_val + (int64_t)p * n_b;
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int32_t t = tw + (u * 32 + lane) * V;
                if (t < rows) {
                    VT v[V];
                    if constexpr (VEC) {
                        const uint4 r = ld_stream16(vp + t);
                        memcpy(v, &r, 16);
                    } else {
                        v[0] = vp[t];
                    }
                    const int64_t j = r0 + t + off;
                    if (t + V <= rows && j >= 0 && j + V <= n) {
                        X xv[V];
                        if constexpr (VEC) {
                            if (x_vec && (j % V) == 0) {
                                const uint4 r = __ldg(reinterpret_cast<const uint4 *>(x + j));
                                memcpy(xv, &r, 16);
                            } else {
#pragma unroll
                                for (int m = 0; m < V; m++) xv[m] = ldg_elem(x + j + m);
                            }
                        } else {
                            xv[0] = ldg_elem(x + j);
                        }
#pragma unroll
                        for (int m = 0; m < V; m++) acc[u][m] += widen(v[m]) * widen(xv[m]);
                    } else {
#pragma unroll
                        for (int m = 0; m < V; m++) {
                            const int64_t jm = j + m;
                            if (t + m < rows && jm >= 0 && jm < n)
                                acc[u][m] += widen(v[m]) * widen(ldg_elem(x + jm));
                        }
                    }
                }
            }
        }

#pragma unroll
        for (int u = 0; u < U; u++) {
            const int32_t t = tw + (u * 32 + lane) * V;
#pragma unroll
            for (int m = 0; m < V; m++)
                if (t + m < rows) y[r0 + t + m] = acc[u][m];
        }
    }
}

// Plain CSR (Fig. 2): S lanes per row, lanes stride over the row's entries,
// butterfly reduction.  All lanes of a warp run the same number of iterations.
template <int S>
__device__ __forceinline__ void csr_rows(int64_t n, const int32_t *__restrict__ rp,
                                         const int32_t *__restrict__ col,
                                         const double *__restrict__ val,
                                         const double *__restrict__ x, double *__restrict__ y)
{
    constexpr int RPW = 32 / S;
    const int lane = threadIdx.x & 31, sub = lane & (S - 1);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t wr = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * RPW; wr < n;
         wr += nwarps * RPW) {
        const int64_t row = wr + lane / S;
        double s = 0.0;
        if (row < n) {
            const int32_t a = rp[row], b = rp[row + 1];
            for (int32_t k = a + sub; k < b; k += S) s += val[k] * __ldg(x + col[k]);
        }
#pragma unroll
        for (int d = S / 2; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (sub == 0 && row < n) y[row] = s;
    }
}

// Lanes per row from the mean row length c = nnz / n, decided on the device
// (every thread reads row_ptr[n]) so the launch needs no host read-back.
__global__ void __launch_bounds__(256)
k_csr_spmv(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
           const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y)
{
    const double c = (double)__ldg(rp + n) / (double)n;
    if (c <= 3.0) csr_rows<2>(n, rp, col, val, x, y);
    else if (c <= 6.0) csr_rows<4>(n, rp, col, val, x, y);
    else if (c <= 12.0) csr_rows<8>(n, rp, col, val, x, y);
    else if (c <= 24.0) csr_rows<16>(n, rp, col, val, x, y);
    else csr_rows<32>(n, rp, col, val, x, y);
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

struct Variant {
    const void *fn;
    int rw;  // rows per warp tile
};

template <typename VT>
Variant pick_variant(int32_t n_b)
{
    constexpr int V = Tr<VT>::V;
    const bool vec = (n_b % V) == 0;
    if (vec) {
        if (n_b >= 2 * 32 * V * 2) return {(const void *)k_mhdc_spmv<VT, 2, true>, 32 * V * 2};
        return {(const void *)k_mhdc_spmv<VT, 1, true>, 32 * V};
    }
    if (n_b >= 32 * 4) return {(const void *)k_mhdc_spmv<VT, 4, false>, 32 * 4};
    return {(const void *)k_mhdc_spmv<VT, 1, false>, 32};
}

Variant variant_for(const mhdc_matrix *A)
{
    switch (A->dtype) {
    case MHDC_F64: return pick_variant<double>(A->n_b);
    case MHDC_F32: return pick_variant<float>(A->n_b);
    default: return pick_variant<__nv_bfloat16>(A->n_b);
    }
}

}  // namespace

int spmv_grid_for(const mhdc_matrix *A)
{
    if (A->n == 0) return 0;
    const Variant v = variant_for(A);
    const int64_t tpb = (A->n_b + v.rw - 1) / v.rw;
    const int64_t tiles = tpb * A->n_blocks;
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fn, SPMV_THREADS, 0);
    if (occ < 1) occ = 1;
    const int64_t need = (tiles + SPMV_WARPS - 1) / SPMV_WARPS;
    const int64_t cap = (int64_t)num_sms() * occ;
    return (int)(need < cap ? need : cap);
}

int launch_spmv(const mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t stream)
{
    if (A->n == 0) return MHDC_OK;
    const Variant v = variant_for(A);
    int32_t tpb = (int32_t)((A->n_b + v.rw - 1) / v.rw);
    int64_t tiles = (int64_t)tpb * A->n_blocks;
    int grid = A->spmv_grid > 0 ? A->spmv_grid : spmv_grid_for(A);
    int64_t n = A->n;
    int32_t n_b = A->n_b;
    const void *dv = A->dia_val, *cv = A->csr_val;
    const int32_t *dp = A->dia_ptr, *doff = A->dia_offset, *crp = A->csr_row_ptr, *cc = A->csr_col;
    void *args[] = {&n, &n_b, &tpb, &tiles, (void *)&dp, (void *)&doff, (void *)&dv, (void *)&crp,
                    (void *)&cc, (void *)&cv, (void *)&d_x, &d_y};
    MHDC_CUDA_TRY(cudaLaunchKernel(v.fn, dim3(grid), dim3(SPMV_THREADS), args, 0, stream));
    return MHDC_OK;
}

int launch_csr(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
               const double *x, double *y, cudaStream_t stream)
{
    if (n == 0) return MHDC_OK;
    const int64_t need = (n + 63) / 64;
    const int64_t cap = (int64_t)num_sms() * 8;
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    k_csr_spmv<<<grid, 256, 0, stream>>>(n, rp, col, val, x, y);
    MHDC_LAUNCH_CHECK("k_csr_spmv");
    return MHDC_OK;
}

int launch_spmm(const mhdc_matrix *, int, const void *, int64_t, void *, int64_t, cudaStream_t)
{
    set_error_msg("mhdc_spmm: not available in this build");
    return MHDC_ERR_UNSUPPORTED;
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
