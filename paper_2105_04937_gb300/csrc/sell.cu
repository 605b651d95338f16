// SELL-C-sigma baseline (Kreutzer, Hager, Wellein, Fehske, Bishop, SIAM J.
// Sci. Comput. 36(5), 2014): the ELL-type format the paper names as future
// work (Sec. 7), built on the device from CSR and multiplied in FP64 beside
// the CSR and M-HDC kernels.
//
// Rows are sorted by length, longest first, inside windows of sigma rows
// (ties keep the input order); the sorted rows form chunks of C consecutive
// rows, each padded to its longest row and stored column by column, so entry
// k of the C rows of a chunk is contiguous (one coalesced load per warp when
// C = 32).  A thread takes one sorted row and sums its own entries only (the
// padding is never multiplied), in column order with one FMA per entry: the
// operations of the CSR kernel, so y is bit-identical to csr_spmv.
#include <cmath>
#include <cstdint>

#include "mhdc_internal.cuh"

struct sell_matrix {
    int64_t n = 0, nnz = 0, chunks = 0, slots = 0;
    int32_t C = 0, sigma = 0;
    int32_t *perm = nullptr;       // [n] input row of sorted position
    int32_t *rowlen = nullptr;     // [n] length of the row at sorted position
    int32_t *chunk_ptr = nullptr;  // [chunks + 1] first slot of each chunk
    int32_t *col = nullptr;        // [slots]
    double *val = nullptr;         // [slots]
};

namespace mhdc {
namespace {

constexpr int SELL_SORT_MAX = 8192;  // window rows sorted in one CTA

__global__ void k_sell_len(int64_t n, const int32_t *__restrict__ rp, int32_t *len)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) len[i] = rp[i + 1] - rp[i];
}

// One CTA per window: sort (length descending, input row ascending) with a
// bitonic network over P2 >= sigma keys in shared memory.
__global__ void __launch_bounds__(512)
k_sell_sort(int64_t n, int32_t sigma, int32_t P2, const int32_t *__restrict__ len,
            int32_t *__restrict__ perm)
{
    extern __shared__ unsigned long long keys[];
    const int64_t w0 = (int64_t)blockIdx.x * sigma;
    const int64_t wn = (n - w0 < sigma) ? (n - w0) : sigma;
    for (int32_t j = threadIdx.x; j < P2; j += blockDim.x) {
        keys[j] = j < wn ? ((unsigned long long)(uint32_t)(INT32_MAX - len[w0 + j]) << 32) |
                               (unsigned long long)(uint32_t)j
                         : ~0ull;
    }
    __syncthreads();
    for (int32_t k = 2; k <= P2; k <<= 1) {
        for (int32_t j = k >> 1; j > 0; j >>= 1) {
            for (int32_t i = threadIdx.x; i < P2; i += blockDim.x) {
                const int32_t l = i ^ j;
                if (l > i) {
                    const unsigned long long a = keys[i], b = keys[l];
                    if ((a > b) == ((i & k) == 0)) {
                        keys[i] = b;
                        keys[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int32_t j = threadIdx.x; j < wn; j += blockDim.x)
        perm[w0 + j] = (int32_t)(w0 + (int64_t)(keys[j] & 0xFFFFFFFFull));
}

__global__ void k_sell_identity(int64_t n, int32_t *perm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = (int32_t)i;
}

// rowlen at sorted positions and chunk widths x C (slots per chunk); the
// 64-bit total of all chunks goes to *total (one atomic per warp) so that the
// host can reject layouts past the int32 slot index before the scan is used
__global__ void k_sell_chunks(int64_t n, int32_t C, int64_t chunks, const int32_t *__restrict__ perm,
                              const int32_t *__restrict__ len, int32_t *rowlen, int32_t *slots,
                              unsigned long long *total)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long mine = 0;
    if (c < chunks) {
        int32_t w = 0;
        for (int64_t r = c * C; r < (c + 1) * C && r < n; r++) {
            const int32_t l = len[perm[r]];
            rowlen[r] = l;
            w = l > w ? l : w;
        }
        mine = (unsigned long long)w * (unsigned long long)C;
        slots[c] = mine > (unsigned long long)INT32_MAX ? 0 : (int32_t)mine;
    }
    for (int d = 16; d > 0; d >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, d);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(total, mine);
}

// one thread per (sorted row, entry): slot chunk_ptr[c] + k * C + r; the
// padding slots keep column 0 and value +0.0 (never read by the product)
__global__ void k_sell_fill(int64_t n, int32_t C, const int32_t *__restrict__ rp,
                            const int32_t *__restrict__ col_in, const double *__restrict__ val_in,
                            const int32_t *__restrict__ perm, const int32_t *__restrict__ chunk_ptr,
                            int32_t *__restrict__ col, double *__restrict__ val)
{
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n) return;
    const int64_t c = pos / C, r = pos - c * C;
    const int32_t i = perm[pos];
    const int32_t a = rp[i], b = rp[i + 1];
    const int64_t base = chunk_ptr[c] + r;
    for (int32_t k = a; k < b; k++) {
        col[base + (int64_t)(k - a) * C] = col_in[k];
        val[base + (int64_t)(k - a) * C] = val_in[k];
    }
}

constexpr int SELL_THREADS = 256;

__global__ void __launch_bounds__(SELL_THREADS)
k_sell_spmv(int64_t n, int32_t C, const int32_t *__restrict__ perm,
            const int32_t *__restrict__ rowlen, const int32_t *__restrict__ chunk_ptr,
            const int32_t *__restrict__ col, const double *__restrict__ val,
            const double *__restrict__ x, double *__restrict__ y)
{
    const int64_t pos = (int64_t)blockIdx.x * SELL_THREADS + threadIdx.x;
    if (pos >= n) return;
    const int64_t c = pos / C, r = pos - c * C;
    const int64_t base = chunk_ptr[c] + r;
    const int32_t len = rowlen[pos];
    double s = 0.0;
    int32_t k = 0;
    for (; k + 4 <= len; k += 4) {  // four entries' loads in flight, FMAs in order
        const int64_t q = base + (int64_t)k * C;
        const double v0 = __ldg(val + q), v1 = __ldg(val + q + C), v2 = __ldg(val + q + 2 * C),
                     v3 = __ldg(val + q + 3 * C);
        const int32_t c0 = __ldg(col + q), c1 = __ldg(col + q + C), c2 = __ldg(col + q + 2 * C),
                      c3 = __ldg(col + q + 3 * C);
        const double x0 = __ldg(x + c0), x1 = __ldg(x + c1), x2 = __ldg(x + c2), x3 = __ldg(x + c3);
        s = fma(v0, x0, s);
        s = fma(v1, x1, s);
        s = fma(v2, x2, s);
        s = fma(v3, x3, s);
    }
    for (; k < len; k++) {
        const int64_t q = base + (int64_t)k * C;
        s = fma(__ldg(val + q), __ldg(x + __ldg(col + q)), s);
    }
    y[perm[pos]] = s;
}

void free_sell(sell_matrix *S)
{
    if (!S) return;
    dfree(S->perm);
    dfree(S->rowlen);
    dfree(S->chunk_ptr);
    dfree(S->col);
    dfree(S->val);
    delete S;
}

int alloc(void **p, size_t bytes)
{
    cudaError_t e = dmalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMalloc", e);
        return cuda_status(e);
    }
    return MHDC_OK;
}

#define SRC(expr)                         \
    do {                                  \
        int rc_ = (expr);                 \
        if (rc_ != MHDC_OK) return rc_;   \
    } while (0)

// Temporaries of one build, released on every exit.
struct Tmp {
    cudaStream_t st;
    void *p[4] = {};
    ~Tmp()
    {
        for (void *q : p) tmp_free(q, st);
    }
};

int sell_fill(sell_matrix *S, const int32_t *rp, const int32_t *col, const double *val,
              cudaStream_t st)
{
    const int64_t n = S->n;
    Tmp t{st};
    SRC(tmp_alloc(&t.p[0], sizeof(int32_t) * (size_t)n, st));
    int32_t *len = static_cast<int32_t *>(t.p[0]);
    k_sell_len<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, rp, len);
    MHDC_LAUNCH_CHECK("k_sell_len");
    SRC(alloc((void **)&S->perm, sizeof(int32_t) * (size_t)n));
    if (S->sigma > 1) {
        int32_t P2 = 1;
        while (P2 < S->sigma) P2 <<= 1;
        const size_t smem = sizeof(unsigned long long) * (size_t)P2;
        MHDC_CUDA_TRY(cudaFuncSetAttribute(k_sell_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
        const int64_t windows = (n + S->sigma - 1) / S->sigma;
        k_sell_sort<<<(unsigned)windows, 512, smem, st>>>(n, S->sigma, P2, len, S->perm);
        MHDC_LAUNCH_CHECK("k_sell_sort");
    } else {
        k_sell_identity<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, S->perm);
        MHDC_LAUNCH_CHECK("k_sell_identity");
    }
    S->chunks = (n + S->C - 1) / S->C;
    SRC(alloc((void **)&S->rowlen, sizeof(int32_t) * (size_t)n));
    SRC(alloc((void **)&S->chunk_ptr, sizeof(int32_t) * (size_t)(S->chunks + 1)));
    SRC(tmp_alloc(&t.p[1], sizeof(int32_t) * (size_t)S->chunks, st));
    SRC(tmp_alloc(&t.p[2], sizeof(int32_t) * (size_t)scan_scratch_elems(S->chunks), st));
    SRC(tmp_alloc(&t.p[3], sizeof(unsigned long long), st));
    int32_t *slots = static_cast<int32_t *>(t.p[1]);
    unsigned long long *total64 = static_cast<unsigned long long *>(t.p[3]);
    MHDC_CUDA_TRY(cudaMemsetAsync(total64, 0, sizeof(unsigned long long), st));
    k_sell_chunks<<<(unsigned)((S->chunks + 255) / 256), 256, 0, st>>>(
        n, S->C, S->chunks, S->perm, len, S->rowlen, slots, total64);
    MHDC_LAUNCH_CHECK("k_sell_chunks");
    unsigned long long h_total = 0;
    MHDC_CUDA_TRY(cudaMemcpyAsync(&h_total, total64, sizeof h_total, cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_total > (unsigned long long)INT32_MAX) {
        set_error_msg("sell_build: more than 2^31 - 1 padded slots");
        return MHDC_ERR_UNSUPPORTED;
    }
    SRC(exclusive_scan_i32(slots, S->chunk_ptr, S->chunks, static_cast<int32_t *>(t.p[2]), st));
    const int32_t total = (int32_t)h_total;
    S->slots = total;
    SRC(alloc((void **)&S->col, sizeof(int32_t) * (size_t)total));
    SRC(alloc((void **)&S->val, sizeof(double) * (size_t)total));
    MHDC_CUDA_TRY(cudaMemsetAsync(S->col, 0, sizeof(int32_t) * (size_t)total, st));
    MHDC_CUDA_TRY(cudaMemsetAsync(S->val, 0, sizeof(double) * (size_t)total, st));
    k_sell_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, S->C, rp, col, val, S->perm,
                                                              S->chunk_ptr, S->col, S->val);
    MHDC_LAUNCH_CHECK("k_sell_fill");
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    return MHDC_OK;
}

}  // namespace
}  // namespace mhdc

using namespace mhdc;

extern "C" {

int sell_build(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
               int32_t C, int32_t sigma, void *stream, sell_handle *out)
{
    if (!out || !d_row_ptr || n < 1 || n >= INT32_MAX || C < 1 || C > 1024 || sigma < 1 ||
        sigma > SELL_SORT_MAX) {
        set_error_msg("sell_build: invalid argument");
        return MHDC_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int32_t nnz = 0;
    MHDC_CUDA_TRY(cudaMemcpyAsync(&nnz, d_row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MHDC_CUDA_TRY(cudaStreamSynchronize(st));
    if (nnz < 0 || (nnz > 0 && (!d_col || !d_val))) {
        set_error_msg("sell_build: bad row_ptr[n] or null arrays");
        return MHDC_ERR_INVALID_ARG;
    }
    sell_matrix *S = new sell_matrix();
    S->n = n;
    S->nnz = nnz;
    S->C = C;
    S->sigma = sigma;
    const int rc = sell_fill(S, d_row_ptr, d_col, d_val, st);
    if (rc != MHDC_OK) {
        cudaStreamSynchronize(st);
        free_sell(S);
        return rc;
    }
    *out = S;
    return MHDC_OK;
}

int sell_spmv(sell_handle S, const double *d_x, double *d_y, void *stream)
{
    if (!S || !d_x || !d_y) {
        set_error_msg("sell_spmv: null argument");
        return MHDC_ERR_INVALID_ARG;
    }
    k_sell_spmv<<<(unsigned)((S->n + SELL_THREADS - 1) / SELL_THREADS), SELL_THREADS, 0,
                  (cudaStream_t)stream>>>(S->n, S->C, S->perm, S->rowlen, S->chunk_ptr, S->col,
                                          S->val, d_x, d_y);
    MHDC_LAUNCH_CHECK("k_sell_spmv");
    return MHDC_OK;
}

int sell_info(sell_handle S, int64_t *n, int64_t *nnz, int64_t *slots, int64_t *chunks)
{
    if (!S) {
        set_error_msg("sell_info: null handle");
        return MHDC_ERR_INVALID_ARG;
    }
    if (n) *n = S->n;
    if (nnz) *nnz = S->nnz;
    if (slots) *slots = S->slots;
    if (chunks) *chunks = S->chunks;
    return MHDC_OK;
}

int sell_export(sell_handle S, int32_t *h_perm, int32_t *h_rowlen, int32_t *h_chunk_ptr,
                int32_t *h_col, double *h_val)
{
    if (!S) {
        set_error_msg("sell_export: null handle");
        return MHDC_ERR_INVALID_ARG;
    }
    const size_t n = (size_t)S->n, c = (size_t)S->chunks + 1, s = (size_t)S->slots;
    if (h_perm) MHDC_CUDA_TRY(cudaMemcpy(h_perm, S->perm, 4 * n, cudaMemcpyDeviceToHost));
    if (h_rowlen) MHDC_CUDA_TRY(cudaMemcpy(h_rowlen, S->rowlen, 4 * n, cudaMemcpyDeviceToHost));
    if (h_chunk_ptr) MHDC_CUDA_TRY(cudaMemcpy(h_chunk_ptr, S->chunk_ptr, 4 * c, cudaMemcpyDeviceToHost));
    if (h_col && s) MHDC_CUDA_TRY(cudaMemcpy(h_col, S->col, 4 * s, cudaMemcpyDeviceToHost));
    if (h_val && s) MHDC_CUDA_TRY(cudaMemcpy(h_val, S->val, 8 * s, cudaMemcpyDeviceToHost));
    return MHDC_OK;
}

int sell_destroy(sell_handle S)
{
    if (S) {
        cudaDeviceSynchronize();
        free_sell(S);
    }
    return MHDC_OK;
}

}  // extern "C"
