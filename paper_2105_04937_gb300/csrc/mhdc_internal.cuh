// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mhdc.h"

// A built matrix: every array is device memory owned by the handle.
struct mhdc_matrix {
    int64_t n = 0, nnz = 0, nnz_rem = 0, P = 0, n_blocks = 0;
    int32_t n_b = 0, dtype = 0, mode = 0;
    double theta = 0.0;
    int device = 0;
    int32_t *dia_ptr = nullptr;      // [n_blocks + 1]
    int32_t *dia_offset = nullptr;   // [P]
    void *dia_val = nullptr;         // [P * n_b] of dtype
    int32_t *csr_row_ptr = nullptr;  // [n + 1]
    int32_t *csr_col = nullptr;      // [nnz_rem]
    void *csr_val = nullptr;         // [nnz_rem] of dtype
    void *x_stage = nullptr;         // host-call staging buffers (lazy)
    void *y_stage = nullptr;
    // pipelined host calls (mhdc_spmv_host_async, lazy): ASYNC_SLOTS staging
    // slots, streams for copies in, products and copies out, per-slot events
    static constexpr int ASYNC_SLOTS = 3;
    void *ax[ASYNC_SLOTS] = {}, *ay[ASYNC_SLOTS] = {};
    cudaStream_t as_in = nullptr, as_comp = nullptr, as_out = nullptr;
    cudaEvent_t ae_in[ASYNC_SLOTS] = {}, ae_comp[ASYNC_SLOTS] = {}, ae_done[ASYNC_SLOTS] = {};
    bool a_used[ASYNC_SLOTS] = {};
    int64_t a_calls = 0;
    int64_t rem_block_rows = 0;      // rows of blocks whose remainder is nonempty
    int64_t bytes_model = 0;
    int64_t bytes_device = 0;
    int spmv_grid = 0;               // CTAs of the SpMV launch
    int variant = -1;                // SpMV tile shape (-1: chosen from n_b)
    int spmm_variant = -1;           // SpMM tile shape (-1: default)
    int *status = nullptr;           // device word: bit 0 = a bounded wait gave up,
                                     // bit 1 = a bounds check of a checked product failed
    unsigned long long *sched = nullptr;  // [2] next tile, finished CTAs of a product
                                          // with persistent tile scheduling (zero between)
    bool checked = false;            // products run the bounds-checked kernel
    // FP64 handles: values split into FP32 (hi, lo) pairs for the emulated product
    float2 *dia_dw = nullptr;        // [P * n_b]
    float2 *csr_dw = nullptr;        // [nnz_rem]
    float2 *x_dw = nullptr;          // [n]: x split by each emulated product
    bool dw_ok = false;              // values inside the window, <= DW_MAX_TERMS terms per row
    bool dw_prepared = false;        // the FP32-pair arrays above exist (made on first use)
};

// One matrix of a batch, as the batched kernel reads it (device memory).
struct BatchMat {
    int64_t n;
    int64_t tile0;      // first warp tile of this matrix in the batch's tile list
    int32_t n_b, tpb;   // rows per block, warp tiles per block
    int32_t vec, pad;   // 16-byte value loads possible (n_b % V == 0)
    const int32_t *dia_ptr, *dia_offset;
    const void *dia_val;
    const int32_t *csr_row_ptr, *csr_col;
    const void *csr_val;
};

// A batch of handles (same dtype) for mhdc_batch_spmv; it does not own them.
struct mhdc_batch {
    int32_t m = 0, dtype = 0;
    int device = 0;
    BatchMat *d_mats = nullptr;
    unsigned long long *d_ctr = nullptr;  // [next tile, finished CTAs]
    int64_t total_tiles = 0;
    int64_t total_nnz = 0;
    int grid = 0;
    cudaStream_t cap_stream = nullptr;    // stream the graph is captured on
    cudaGraphExec_t graph = nullptr;
    const void *const *g_xs = nullptr;    // pointer arrays baked into the graph
    void *const *g_ys = nullptr;
};

namespace mhdc {

inline size_t value_size(int dtype)
{
    return dtype == MHDC_F64 ? 8 : dtype == MHDC_F32 ? 4 : 2;
}
inline size_t y_size(int dtype) { return dtype == MHDC_F64 ? 8 : 4; }

// Every device allocation and free of the library (alloc.cu): cudaMalloc /
// cudaFree / stream-ordered pool calls, with a live count and the host-side
// allocation-failure hook of mhdc_debug_fail_alloc.
cudaError_t dmalloc(void **p, size_t bytes);
void dfree(void *p);
cudaError_t dmalloc_pool(void **p, size_t bytes, cudaMemPool_t pool, cudaStream_t st);
void dfree_async(void *p, cudaStream_t st);

// Record the details of the last failure of this thread (mhdc_last_error).
void set_error(const char *where, cudaError_t e);
void set_error_msg(const char *msg);

inline int cuda_status(cudaError_t e)
{
    return e == cudaErrorMemoryAllocation ? MHDC_ERR_OOM : MHDC_ERR_CUDA;
}

// Build (both selection modes); defined in build.cu.
int build_matrix(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
                 int32_t n_b, double theta, int32_t dtype, int mode, cudaStream_t stream,
                 mhdc_matrix **out);
int build_matrix_dia(int64_t n, int32_t nd, const int32_t *d_offset, const double *d_val,
                     int32_t n_b, double theta, int32_t dtype, cudaStream_t stream,
                     mhdc_matrix **out);
void free_matrix(mhdc_matrix *A);
// Stream-ordered temporaries from the library's pool (build.cu).
int tmp_alloc(void **p, size_t bytes, cudaStream_t st);
void tmp_free(void *p, cudaStream_t st);
int feature_hist(int64_t n, const int32_t *rp, const int32_t *col, int32_t n_b,
                 cudaStream_t st, unsigned long long *h_ent, unsigned long long *h_dia);
int build_noalloc(int64_t n, const int32_t *rp, const int32_t *col, const double *val, int32_t n_b,
                  double theta, int32_t dtype, int32_t *dia_ptr, int32_t *dia_offset, void *dia_val,
                  int64_t cap_P, int32_t *csr_row_ptr, int32_t *csr_col, void *csr_val,
                  int64_t cap_rem, int64_t *h_P, int64_t *h_nnz_rem, cudaStream_t st);

// Products; defined in spmv.cu.
int launch_spmv(mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t stream);
int launch_dia(const mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t stream);
int launch_csr(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
               const double *x, double *y, cudaStream_t stream);
int launch_stream_bench(int64_t N, const double *A, const double *B, const int32_t *I, double *C,
                        int indirect, cudaStream_t stream);
int spmv_grid_for(const mhdc_matrix *A);
int batch_prepare(mhdc_batch *B);
int batch_tile_rows(int dtype, int n_b, int *vec);
int launch_batch(mhdc_batch *B, const void *const *d_xs, void *const *d_ys, cudaStream_t st);
int launch_read_bench(int64_t N, const double *A, double *out, int grid, cudaStream_t stream);
int read_bench_grid();
int launch_fma_probe(int fp64, int iters, void *out, cudaStream_t stream);
bool tma_supported(const mhdc_matrix *A);
int launch_spmv_tma(const mhdc_matrix *A, int shape, const void *d_x, void *d_y,
                    cudaStream_t stream);
constexpr int NUM_REG_VARIANTS = 6;
constexpr int FIRST_DW_VARIANT = 10;
constexpr int FIRST_TMA_DW_VARIANT = 13;
constexpr int FIRST_XW_VARIANT = 16;
// variants 16-19: values and x staged in shared memory by TMA (x 16-byte aligned)
bool xw_supported(const mhdc_matrix *A, const void *d_x);
int launch_spmv_xw(const mhdc_matrix *A, int shape, const void *d_x, void *d_y,
                   cudaStream_t stream);
int launch_spmv_tma_dw(mhdc_matrix *A, int shape, const void *d_x, void *d_y,
                       cudaStream_t stream);
// Emulated FP64 (FP32 pairs): nonzero |a|, |x| must lie in [2^DW_EMIN, 2^DW_EMAX]
// and a row may have at most DW_MAX_TERMS terms (error bound, see spmv.cu).
constexpr int DW_EMIN = -45;
constexpr int DW_EMAX = 60;
constexpr int DW_MAX_TERMS = 48;
int prepare_dw(mhdc_matrix *A, cudaStream_t st);
// prepare_dw once per handle (the emulated variants and the tuner call it).
int ensure_dw(mhdc_matrix *A, cudaStream_t st);
// an FP64 handle whose values passed the window check, n_b even
inline bool emulation_possible(const mhdc_matrix *A)
{
    return A->dw_ok && A->dtype == MHDC_F64 && (A->n_b % 2) == 0;
}
int tune_spmv(mhdc_matrix *A, const void *d_x, void *d_y, cudaStream_t stream, int32_t *best,
              float *times_us);

// SpMM; defined in spmm.cu.
int launch_spmm(mhdc_matrix *A, int k, const void *d_X, int64_t ldx, void *d_Y,
                int64_t ldy, cudaStream_t stream);
int tune_spmm(mhdc_matrix *A, int k, const void *d_X, int64_t ldx, void *d_Y, int64_t ldy,
              cudaStream_t stream, int32_t *best, float *times_us);

// The 16 bytes starting `sh` bytes (sh < 16, a multiple of the element size)
// into the 32-byte window (lo, hi): two aligned loads replace V element loads
// when x[j .. j+V) is not 16-byte aligned.  `sh` is warp-uniform.
__device__ __forceinline__ uint4 window16(const uint4 &lo, const uint4 &hi, int sh)
{
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    const int bs = (sh & 3) * 8;
    uint32_t o[5];
    switch (sh >> 2) {
    case 0: o[0] = w[0]; o[1] = w[1]; o[2] = w[2]; o[3] = w[3]; o[4] = w[4]; break;
    case 1: o[0] = w[1]; o[1] = w[2]; o[2] = w[3]; o[3] = w[4]; o[4] = w[5]; break;
    case 2: o[0] = w[2]; o[1] = w[3]; o[2] = w[4]; o[3] = w[5]; o[4] = w[6]; break;
    default: o[0] = w[3]; o[1] = w[4]; o[2] = w[5]; o[3] = w[6]; o[4] = w[7]; break;
    }
    if (bs == 0) return make_uint4(o[0], o[1], o[2], o[3]);
    return make_uint4(__funnelshift_r(o[0], o[1], bs), __funnelshift_r(o[1], o[2], bs),
                      __funnelshift_r(o[2], o[3], bs), __funnelshift_r(o[3], o[4], bs));
}

// ---- CSR remainder rows (Fig. 13, first loop) of every product kernel
//
// FP32 / BF16 handles accumulate in FP32, except a remainder row with more
// than REM_LONG entries: it is summed in FP64 (each product of two stored
// FP32 / BF16 values is exact in FP64) and rounded once to FP32, so its error
// no longer grows with the row's length at FP32's unit roundoff.  The row
// then enters the FP32 accumulator as one term.  FP64 handles are unchanged.
constexpr int REM_LONG = 64;

__device__ __forceinline__ double rem_in(double v) { return v; }
__device__ __forceinline__ float rem_in(float v) { return v; }
__device__ __forceinline__ float rem_in(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double rem_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rem_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Adds the remainder entries [a, b) of one row to acc (zero on entry in
// every kernel), in column order, one FMA per entry.
template <typename Acc, typename VT, typename X>
__device__ __forceinline__ void rem_row_add(Acc &acc, int32_t a, int32_t b,
                                            const int32_t *__restrict__ col,
                                            const VT *__restrict__ val, const X *__restrict__ x)
{
    if constexpr (sizeof(Acc) < sizeof(double)) {
        if (b - a > REM_LONG) {
            double s = 0.0;
            for (int32_t k = a; k < b; k++)
                s = fma((double)rem_in(val[k]), (double)rem_in(__ldg(x + col[k])), s);
            acc += (Acc)s;  // rounded to nearest even once; exact while acc is zero
            return;
        }
    }
    for (int32_t k = a; k < b; k++) acc = rem_fma(rem_in(val[k]), rem_in(__ldg(x + col[k])), acc);
}

// The remainder rows of one lane, R at a time, with the operations of
// rem_row_add (each row from zero in s[r], column order, one FMA per entry,
// rows longer than REM_LONG through its FP64 path) but with the loads of all
// R rows in flight together: each round loads the next E entries of every
// row -- columns and values, then the gathers of x, all independent --
// before the FMAs of the round (rem_row_add walks the rows one after the
// other).  Row r holds the entries [a[r], b[r]); a[r] >= b[r] is an empty row.
template <int R, int E, typename Acc, typename VT, typename X>
__device__ __forceinline__ void rem_rows_add(Acc (&s)[R], int32_t (&a)[R], const int32_t (&b)[R],
                                             const int32_t *__restrict__ col,
                                             const VT *__restrict__ val,
                                             const X *__restrict__ x)
{
    if constexpr (sizeof(Acc) < sizeof(double)) {
#pragma unroll
        for (int r = 0; r < R; r++)
            if (b[r] - a[r] > REM_LONG) {
                rem_row_add(s[r], a[r], b[r], col, val, x);
                a[r] = b[r];
            }
    }
    for (;;) {
        bool more = false;
#pragma unroll
        for (int r = 0; r < R; r++) more |= a[r] < b[r];
        if (!more) break;
        int32_t c[R][E];
        VT v[R][E];
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int e = 0; e < E; e++) {
                const bool in = e < b[r] - a[r];
                c[r][e] = in ? col[a[r] + e] : 0;
                v[r][e] = in ? val[a[r] + e] : VT(0);
            }
        X xv[R][E];
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int e = 0; e < E; e++) xv[r][e] = e < b[r] - a[r] ? __ldg(x + c[r][e]) : X(0);
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int e = 0; e < E; e++)
                if (e < b[r] - a[r]) s[r] = rem_fma(rem_in(v[r][e]), rem_in(xv[r][e]), s[r]);
#pragma unroll
        for (int r = 0; r < R; r++) a[r] = b[r] - a[r] > E ? a[r] + E : b[r];
    }
}

// Row i (= r0 + t, block ib) of the native FP64 product, one thread: the
// remainder from zero in column order, then the block's diagonals in
// ascending order (a zero where i + off leaves [0, n)), each term one FMA --
// the operations of every native FP64 tile, so the same bits.  The emulated
// tiles recompute with it the rows whose FP32-pair sum came out NaN: the rows
// that read an x outside the emulation window (marked NaN by the split).
__device__ __forceinline__ double native_row(int64_t i, int32_t t, int64_t ib, int64_t n,
                                             int32_t n_b, const int32_t *__restrict__ dia_ptr,
                                             const int32_t *__restrict__ dia_offset,
                                             const double *__restrict__ dia_val,
                                             const int32_t *__restrict__ csr_row_ptr,
                                             const int32_t *__restrict__ csr_col,
                                             const double *__restrict__ csr_val,
                                             const double *__restrict__ x)
{
    double s = 0.0;
    for (int32_t q = csr_row_ptr[i]; q < csr_row_ptr[i + 1]; q++)
        s = fma(csr_val[q], x[csr_col[q]], s);
    for (int32_t p = dia_ptr[ib]; p < dia_ptr[ib + 1]; p++) {
        const int64_t j = i + dia_offset[p];
        s = fma(dia_val[(int64_t)p * n_b + t], (j >= 0 && j < n) ? x[j] : 0.0, s);
    }
    return s;
}

// Bounds-checked products (mhdc_set_checked): the extents of a handle's
// arrays and its status word.  ck_in(ck, lo, hi, ext) is true when the
// index range [lo, hi) lies inside [0, ext); otherwise it sets bit 1 of the
// status word (mhdc_check then reports MHDC_ERR_DEVICE_CHECK) and the caller
// skips the access.
struct BoundsCheck {
    int64_t n_blocks, P, dia_slots, nnz_rem;
    int *status;
};
constexpr int STATUS_BOUNDS = 2;

__device__ __forceinline__ bool ck_in(const BoundsCheck &ck, int64_t lo, int64_t hi, int64_t ext)
{
    if (lo >= 0 && lo <= hi && hi <= ext) return true;
    atomicOr(ck.status, STATUS_BOUNDS);
    return false;
}

// rem_row_add with every index checked: the entry range against the
// remainder's extent, each column against [0, n).  An access that fails is
// skipped (the entry counts as 0).
template <typename Acc, typename VT, typename X>
__device__ __forceinline__ void rem_row_add_ck(Acc &acc, int32_t a, int32_t b,
                                               const int32_t *__restrict__ col,
                                               const VT *__restrict__ val, const X *__restrict__ x,
                                               int64_t n, const BoundsCheck &ck)
{
    if (!ck_in(ck, a, b, ck.nnz_rem)) return;
    auto xat = [&](int32_t k) -> X {
        const int32_t c = col[k];
        return ck_in(ck, c, (int64_t)c + 1, n) ? __ldg(x + c) : X(0);
    };
    if constexpr (sizeof(Acc) < sizeof(double)) {
        if (b - a > REM_LONG) {
            double s = 0.0;
            for (int32_t k = a; k < b; k++) s = fma((double)rem_in(val[k]), (double)rem_in(xat(k)), s);
            acc += (Acc)s;
            return;
        }
    }
    for (int32_t k = a; k < b; k++) acc = rem_fma(rem_in(val[k]), rem_in(xat(k)), acc);
}

// Exclusive prefix sum of m int32 values into out[0..m] (out[m] = total);
// scratch must hold scan_scratch_elems(m) int32.  Defined in scan.cu.
int64_t scan_scratch_elems(int64_t m);
int exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t m, int32_t *scratch,
                       cudaStream_t stream);

}  // namespace mhdc

#define MHDC_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) {                              \
            mhdc::set_error(#expr, e_);                       \
            return mhdc::cuda_status(e_);                     \
        }                                                     \
    } while (0)

#define MHDC_LAUNCH_CHECK(name)                               \
    do {                                                      \
        cudaError_t e_ = cudaGetLastError();                  \
        if (e_ != cudaSuccess) {                              \
            mhdc::set_error(name, e_);                        \
            return MHDC_ERR_CUDA;                             \
        }                                                     \
    } while (0)
