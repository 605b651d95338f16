// extern "C" entry points of include/mhdc.h: argument checks, dispatch to the
// kernels, and per-thread error text.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mhdc_internal.cuh"

namespace mhdc {

static thread_local char g_last_error[256] = "";

void set_error(const char *where, cudaError_t e)
{
    snprintf(g_last_error, sizeof g_last_error, "%s: %s (%d)", where, cudaGetErrorString(e),
             (int)e);
}

void set_error_msg(const char *msg) { snprintf(g_last_error, sizeof g_last_error, "%s", msg); }

}  // namespace mhdc

using namespace mhdc;

extern "C" {

const char *mhdc_last_error(void) { return g_last_error; }

const char *mhdc_strerror(int code)
{
    switch (code) {
    case MHDC_OK: return "ok";
    case MHDC_ERR_INVALID_ARG: return "invalid argument";
    case MHDC_ERR_BAD_CSR: return "invalid CSR input";
    case MHDC_ERR_OOM: return "device out of memory";
    case MHDC_ERR_CUDA: return "CUDA error";
    case MHDC_ERR_UNSUPPORTED: return "unsupported";
    case MHDC_ERR_DEVICE_CHECK: return "device-side check failed";
    case MHDC_ERR_TIMEOUT: return "device-side wait timed out";
    default: return "unknown status";
    }
}

int mhdc_build(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
               int32_t n_b, double theta, int32_t dtype, void *stream, mhdc_handle *out)
{
    return build_matrix(n, d_row_ptr, d_col, d_val, n_b, theta, dtype, MHDC_MODE_BLOCK,
                        (cudaStream_t)stream, out);
}

int mhdc_build_dia(int64_t n, int32_t nd, const int32_t *d_offset, const double *d_val, int32_t n_b,
                   double theta, int32_t dtype, void *stream, mhdc_handle *out)
{
    return build_matrix_dia(n, nd, d_offset, d_val, n_b, theta, dtype, (cudaStream_t)stream, out);
}

int hdc_build(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
              int32_t n_b, double theta, int32_t dtype, void *stream, mhdc_handle *out)
{
    return build_matrix(n, d_row_ptr, d_col, d_val, n_b, theta, dtype, MHDC_MODE_GLOBAL,
                        (cudaStream_t)stream, out);
}

int mhdc_spmv(mhdc_handle A, const void *d_x, void *d_y, void *stream)
{
    if (!A || (A->n > 0 && (!d_x || !d_y))) {
        set_error_msg("mhdc_spmv: null argument");
        return MHDC_ERR_INVALID_ARG;
    }
    return launch_spmv(A, d_x, d_y, (cudaStream_t)stream);
}

int mhdc_spmv_host(mhdc_handle A, const void *h_x, void *h_y, void *stream)
{
    if (!A || (A->n > 0 && (!h_x || !h_y))) {
        set_error_msg("mhdc_spmv_host: null argument");
        return MHDC_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bx = value_size(A->dtype) * (size_t)A->n, by = y_size(A->dtype) * (size_t)A->n;
    if (!A->x_stage) MHDC_CUDA_TRY(dmalloc(&A->x_stage, bx ? bx : 16));
    if (!A->y_stage) MHDC_CUDA_TRY(dmalloc(&A->y_stage, by ? by : 16));
    MHDC_CUDA_TRY(cudaMemcpyAsync(A->x_stage, h_x, bx, cudaMemcpyHostToDevice, st));
    int rc = launch_spmv(A, A->x_stage, A->y_stage, st);
    if (rc != MHDC_OK) return rc;
    MHDC_CUDA_TRY(cudaMemcpyAsync(h_y, A->y_stage, by, cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    return MHDC_OK;
}

int mhdc_dia_spmv(mhdc_handle A, const void *d_x, void *d_y, void *stream)
{
    if (!A || (A->n > 0 && (!d_x || !d_y))) {
        set_error_msg("mhdc_dia_spmv: null argument");
        return MHDC_ERR_INVALID_ARG;
    }
    if (A->mode != MHDC_MODE_GLOBAL) {
        set_error_msg("mhdc_dia_spmv: needs a handle from hdc_build (same diagonals in every block)");
        return MHDC_ERR_UNSUPPORTED;
    }
    return launch_dia(A, d_x, d_y, (cudaStream_t)stream);
}

int mhdc_spmv_host_async(mhdc_handle A, const void *h_x, void *h_y)
{
    if (!A || (A->n > 0 && (!h_x || !h_y))) {
        set_error_msg("mhdc_spmv_host_async: null argument");
        return MHDC_ERR_INVALID_ARG;
    }
    if (A->n == 0) return MHDC_OK;
    const size_t bx = value_size(A->dtype) * (size_t)A->n, by = y_size(A->dtype) * (size_t)A->n;
    constexpr int NS = mhdc_matrix::ASYNC_SLOTS;
    if (!A->ae_done[NS - 1]) {  // first call (or one that failed to set up): make what is missing
        const unsigned fl = cudaStreamNonBlocking;
        if (!A->as_in) MHDC_CUDA_TRY(cudaStreamCreateWithFlags(&A->as_in, fl));
        if (!A->as_comp) MHDC_CUDA_TRY(cudaStreamCreateWithFlags(&A->as_comp, fl));
        if (!A->as_out) MHDC_CUDA_TRY(cudaStreamCreateWithFlags(&A->as_out, fl));
        for (int k = 0; k < NS; k++) {
            if (!A->ax[k]) MHDC_CUDA_TRY(dmalloc(&A->ax[k], bx));
            if (!A->ay[k]) MHDC_CUDA_TRY(dmalloc(&A->ay[k], by));
            if (!A->ae_in[k]) MHDC_CUDA_TRY(cudaEventCreateWithFlags(&A->ae_in[k], cudaEventDisableTiming));
            if (!A->ae_comp[k])
                MHDC_CUDA_TRY(cudaEventCreateWithFlags(&A->ae_comp[k], cudaEventDisableTiming));
            if (!A->ae_done[k])
                MHDC_CUDA_TRY(cudaEventCreateWithFlags(&A->ae_done[k], cudaEventDisableTiming));
        }
    }
    const int s = (int)(A->a_calls % NS);
    // the call NS back used this slot: its copy-out must be complete
    if (A->a_used[s]) MHDC_CUDA_TRY(cudaEventSynchronize(A->ae_done[s]));
    MHDC_CUDA_TRY(cudaMemcpyAsync(A->ax[s], h_x, bx, cudaMemcpyHostToDevice, A->as_in));
    MHDC_CUDA_TRY(cudaEventRecord(A->ae_in[s], A->as_in));
    MHDC_CUDA_TRY(cudaStreamWaitEvent(A->as_comp, A->ae_in[s], 0));
    int rc = launch_spmv(A, A->ax[s], A->ay[s], A->as_comp);
    if (rc != MHDC_OK) return rc;
    MHDC_CUDA_TRY(cudaEventRecord(A->ae_comp[s], A->as_comp));
    MHDC_CUDA_TRY(cudaStreamWaitEvent(A->as_out, A->ae_comp[s], 0));
    MHDC_CUDA_TRY(cudaMemcpyAsync(h_y, A->ay[s], by, cudaMemcpyDeviceToHost, A->as_out));
    MHDC_CUDA_TRY(cudaEventRecord(A->ae_done[s], A->as_out));
    A->a_used[s] = true;
    A->a_calls++;
    return MHDC_OK;
}

int mhdc_host_wait(mhdc_handle A)
{
    if (!A) {
        set_error_msg("mhdc_host_wait: null handle");
        return MHDC_ERR_INVALID_ARG;
    }
    for (int k = 0; k < mhdc_matrix::ASYNC_SLOTS; k++)
        if (A->a_used[k]) MHDC_CUDA_TRY(cudaEventSynchronize(A->ae_done[k]));
    return MHDC_OK;
}

int mhdc_spmm(mhdc_handle A, int32_t k, const void *d_X, int64_t ldx, void *d_Y, int64_t ldy,
              void *stream)
{
    if (!A || k < 1 || k > 64 || ldx < k || ldy < k || (A->n > 0 && (!d_X || !d_Y))) {
        set_error_msg("mhdc_spmm: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    return launch_spmm(A, k, d_X, ldx, d_Y, ldy, (cudaStream_t)stream);
}

int mhdc_spmm_set_variant(mhdc_handle A, int32_t v)
{
    if (!A || v < -1 || v >= MHDC_NUM_SPMM_VARIANTS) {
        set_error_msg("mhdc_spmm_set_variant: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    A->spmm_variant = v;
    return MHDC_OK;
}

int mhdc_spmm_tune(mhdc_handle A, int32_t k, const void *d_X, int64_t ldx, void *d_Y,
                   int64_t ldy, void *stream, int32_t *best, float *times_us)
{
    if (!A || k < 1 || k > 64 || ldx < k || ldy < k || (A->n > 0 && (!d_X || !d_Y))) {
        set_error_msg("mhdc_spmm_tune: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    return tune_spmm(A, k, d_X, ldx, d_Y, ldy, (cudaStream_t)stream, best, times_us);
}

int csr_spmv(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
             const double *d_x, double *d_y, void *stream)
{
    if (n < 0 || (n > 0 && (!d_row_ptr || !d_x || !d_y))) {
        set_error_msg("csr_spmv: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    return launch_csr(n, d_row_ptr, d_col, d_val, d_x, d_y, (cudaStream_t)stream);
}

int mhdc_export(mhdc_handle A, int32_t *h_dia_ptr, int32_t *h_dia_offset, void *h_dia_val,
                int32_t *h_csr_row_ptr, int32_t *h_csr_col, void *h_csr_val)
{
    if (!A) {
        set_error_msg("mhdc_export: null handle");
        return MHDC_ERR_INVALID_ARG;
    }
    const size_t sv = value_size(A->dtype);
    MHDC_CUDA_TRY(cudaDeviceSynchronize());
    if (h_dia_ptr)
        MHDC_CUDA_TRY(cudaMemcpy(h_dia_ptr, A->dia_ptr, sizeof(int32_t) * (A->n_blocks + 1),
                                 cudaMemcpyDeviceToHost));
    if (h_dia_offset && A->P)
        MHDC_CUDA_TRY(cudaMemcpy(h_dia_offset, A->dia_offset, sizeof(int32_t) * A->P,
                                 cudaMemcpyDeviceToHost));
    if (h_dia_val && A->P)
        MHDC_CUDA_TRY(cudaMemcpy(h_dia_val, A->dia_val, sv * (size_t)A->P * (size_t)A->n_b,
                                 cudaMemcpyDeviceToHost));
    if (h_csr_row_ptr)
        MHDC_CUDA_TRY(cudaMemcpy(h_csr_row_ptr, A->csr_row_ptr, sizeof(int32_t) * (A->n + 1),
                                 cudaMemcpyDeviceToHost));
    if (h_csr_col && A->nnz_rem)
        MHDC_CUDA_TRY(cudaMemcpy(h_csr_col, A->csr_col, sizeof(int32_t) * A->nnz_rem,
                                 cudaMemcpyDeviceToHost));
    if (h_csr_val && A->nnz_rem)
        MHDC_CUDA_TRY(cudaMemcpy(h_csr_val, A->csr_val, sv * (size_t)A->nnz_rem,
                                 cudaMemcpyDeviceToHost));
    return MHDC_OK;
}

int mhdc_info(mhdc_handle A, mhdc_info_t *out)
{
    if (!A || !out) {
        set_error_msg("mhdc_info: null argument");
        return MHDC_ERR_INVALID_ARG;
    }
    memset(out, 0, sizeof *out);
    out->n = A->n;
    out->nnz = A->nnz;
    out->nnz_rem = A->nnz_rem;
    out->P = A->P;
    out->n_blocks = A->n_blocks;
    out->n_b = A->n_b;
    out->dtype = A->dtype;
    out->mode = A->mode;
    out->variant = A->variant;
    out->emulated_ok = !A->dw_prepared ? -1 : A->dw_ok ? 1 : 0;
    out->theta = A->theta;
    out->alpha = A->P ? (double)(A->nnz - A->nnz_rem) / ((double)A->P * (double)A->n_b) : 0.0;
    out->beta = A->nnz ? (double)A->nnz_rem / (double)A->nnz : 0.0;
    out->bytes_model = A->bytes_model;
    out->bytes_device = A->bytes_device;
    return MHDC_OK;
}

int mhdc_stats(mhdc_handle A, double *alpha, double *beta, int64_t *P, int64_t *bytes)
{
    mhdc_info_t inf;
    const int rc = mhdc_info(A, &inf);
    if (rc != MHDC_OK) return rc;
    if (alpha) *alpha = inf.alpha;
    if (beta) *beta = inf.beta;
    if (P) *P = inf.P;
    if (bytes) *bytes = inf.bytes_model;
    return MHDC_OK;
}

int mhdc_set_variant(mhdc_handle A, int32_t v)
{
    if (!A || v < -1 || v >= MHDC_NUM_VARIANTS) {
        set_error_msg("mhdc_set_variant: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    if (v >= FIRST_DW_VARIANT && v < FIRST_XW_VARIANT) {  // emulated arrays: made on first use
        int rc = ensure_dw(A, nullptr);
        if (rc != MHDC_OK) return rc;
        MHDC_CUDA_TRY(cudaStreamSynchronize(nullptr));
    }
    A->variant = v;
    return MHDC_OK;
}

int mhdc_tune(mhdc_handle A, const void *d_x, void *d_y, void *stream, int32_t *best,
              float *times_us)
{
    if (!A || (A->n > 0 && (!d_x || !d_y))) {
        set_error_msg("mhdc_tune: null argument");
        return MHDC_ERR_INVALID_ARG;
    }
    int rc = ensure_dw(A, (cudaStream_t)stream);
    if (rc != MHDC_OK) return rc;
    return tune_spmv(A, d_x, d_y, (cudaStream_t)stream, best, times_us);
}

int mhdc_check(mhdc_handle A)
{
    if (!A) {
        set_error_msg("mhdc_check: null handle");
        return MHDC_ERR_INVALID_ARG;
    }
    int h = 0;
    MHDC_CUDA_TRY(cudaDeviceSynchronize());
    MHDC_CUDA_TRY(cudaMemcpy(&h, A->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        MHDC_CUDA_TRY(cudaMemset(A->status, 0, sizeof(int)));
        if (h & STATUS_BOUNDS) {
            set_error_msg("a bounds check of a checked product failed (the access was skipped)");
            return MHDC_ERR_DEVICE_CHECK;
        }
        set_error_msg("a bounded device-side wait gave up");
        return MHDC_ERR_TIMEOUT;
    }
    return MHDC_OK;
}

int mhdc_set_checked(mhdc_handle A, int32_t on)
{
    if (!A || (on != 0 && on != 1)) {
        set_error_msg("mhdc_set_checked: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    A->checked = on != 0;
    return MHDC_OK;
}

int mhdc_batch_create(int32_t m, const mhdc_handle *mats, mhdc_batch_handle *out)
{
    if (m < 1 || !mats || !out) {
        set_error_msg("mhdc_batch_create: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    for (int32_t i = 0; i < m; i++) {
        if (!mats[i] || mats[i]->dtype != mats[0]->dtype) {
            set_error_msg("mhdc_batch_create: null handle or mixed dtypes");
            return MHDC_ERR_INVALID_ARG;
        }
    }
    std::vector<BatchMat> h((size_t)m);
    int64_t tiles = 0, nnz = 0;
    for (int32_t i = 0; i < m; i++) {
        const mhdc_matrix *A = mats[i];
        int vec = 0;
        const int rw = batch_tile_rows(A->dtype, A->n_b, &vec);
        BatchMat &b = h[(size_t)i];
        b.n = A->n;
        b.n_b = A->n_b;
        b.tpb = (int32_t)((A->n_b + rw - 1) / rw);
        b.vec = vec;
        b.pad = 0;
        b.tile0 = tiles;
        b.dia_ptr = A->dia_ptr;
        b.dia_offset = A->dia_offset;
        b.dia_val = A->dia_val;
        b.csr_row_ptr = A->csr_row_ptr;
        b.csr_col = A->csr_col;
        b.csr_val = A->csr_val;
        tiles += (int64_t)b.tpb * A->n_blocks;
        nnz += A->nnz;
    }
    mhdc_batch *B = new mhdc_batch();
    B->m = m;
    B->dtype = mats[0]->dtype;
    B->total_tiles = tiles;
    B->total_nnz = nnz;
    cudaGetDevice(&B->device);
    cudaError_t e = dmalloc((void **)&B->d_mats, sizeof(BatchMat) * (size_t)m);
    if (e == cudaSuccess) e = dmalloc((void **)&B->d_ctr, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = cudaMemcpy(B->d_mats, h.data(), sizeof(BatchMat) * (size_t)m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(B->d_ctr, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking);
    int rc = e == cudaSuccess ? batch_prepare(B) : MHDC_ERR_CUDA;
    if (e != cudaSuccess) set_error("mhdc_batch_create", e);
    if (rc != MHDC_OK) {
        mhdc_batch_destroy(B);
        return e == cudaErrorMemoryAllocation ? MHDC_ERR_OOM : rc;
    }
    *out = B;
    return MHDC_OK;
}

int mhdc_batch_spmv(mhdc_batch_handle B, const void *const *d_xs, void *const *d_ys, void *stream)
{
    if (!B || !d_xs || !d_ys) {
        set_error_msg("mhdc_batch_spmv: null argument");
        return MHDC_ERR_INVALID_ARG;
    }
    return launch_batch(B, d_xs, d_ys, (cudaStream_t)stream);
}

int mhdc_batch_spmv_graph(mhdc_batch_handle B, const void *const *d_xs, void *const *d_ys,
                          void *stream)
{
    if (!B || !d_xs || !d_ys) {
        set_error_msg("mhdc_batch_spmv_graph: null argument");
        return MHDC_ERR_INVALID_ARG;
    }
    if (!B->graph || B->g_xs != d_xs || B->g_ys != d_ys) {
        if (B->graph) {
            cudaGraphExecDestroy(B->graph);
            B->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        MHDC_CUDA_TRY(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = launch_batch(B, d_xs, d_ys, B->cap_stream);
        cudaError_t e = cudaStreamEndCapture(B->cap_stream, &g);
        if (rc != MHDC_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) {
            set_error("cudaStreamEndCapture", e);
            return MHDC_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&B->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            B->graph = nullptr;
            set_error("cudaGraphInstantiate", e);
            return MHDC_ERR_CUDA;
        }
        B->g_xs = d_xs;
        B->g_ys = d_ys;
    }
    MHDC_CUDA_TRY(cudaGraphLaunch(B->graph, (cudaStream_t)stream));
    return MHDC_OK;
}

int mhdc_batch_destroy(mhdc_batch_handle B)
{
    if (!B) return MHDC_OK;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    dfree(B->d_mats);
    dfree(B->d_ctr);
    delete B;
    return MHDC_OK;
}

int mhdc_destroy(mhdc_handle A)
{
    free_matrix(A);
    return MHDC_OK;
}

int mhdc_stream_bench(int64_t N, const double *d_A, const double *d_B, const int32_t *d_I,
                      double *d_C, int32_t indirect, void *stream)
{
    if (N < 0 || (N > 0 && (!d_A || !d_B || !d_C || (indirect && !d_I)))) {
        set_error_msg("mhdc_stream_bench: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    return launch_stream_bench(N, d_A, d_B, d_I, d_C, indirect, (cudaStream_t)stream);
}

int mhdc_build_noalloc(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col,
                       const double *d_val, int32_t n_b, double theta, int32_t dtype,
                       int32_t *d_dia_ptr, int32_t *d_dia_offset, void *d_dia_val, int64_t cap_P,
                       int32_t *d_csr_row_ptr, int32_t *d_csr_col, void *d_csr_val,
                       int64_t cap_rem, int64_t *h_P, int64_t *h_nnz_rem, void *stream)
{
    return build_noalloc(n, d_row_ptr, d_col, d_val, n_b, theta, dtype, d_dia_ptr, d_dia_offset,
                         d_dia_val, cap_P, d_csr_row_ptr, d_csr_col, d_csr_val, cap_rem, h_P,
                         h_nnz_rem, (cudaStream_t)stream);
}

int mhdc_read_bench(int64_t N, const double *d_A, double *d_out, void *stream)
{
    if (N < 0 || (N & 1) || (N > 0 && (!d_A || !d_out)) || ((uintptr_t)d_A & 15)) {
        set_error_msg("mhdc_read_bench: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    return launch_read_bench(N, d_A, d_out, read_bench_grid(), (cudaStream_t)stream);
}

int mhdc_read_bench_ctas(void) { return read_bench_grid(); }

int mhdc_fma_bench(int32_t fp64, int32_t iters, void *d_out, void *stream)
{
    if (iters < 1 || !d_out) {
        set_error_msg("mhdc_fma_bench: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    return launch_fma_probe(fp64, iters, d_out, (cudaStream_t)stream);
}

}  // extern "C"
