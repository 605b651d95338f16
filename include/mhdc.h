/*
 * mhdc.h -- C ABI of the M-HDC sparse matrix-vector library (sm_103a).
 *
 * Method: Fukaya, Ishida, Miura, Iwashita, Nakashima, "Accelerating the SpMV
 * kernel on standard CPUs by exploiting the partially diagonal structures"
 * (arXiv 2105.04937).  The product is y = A x for an n x n real sparse A
 * (Sec. 3.1).  In the M-HDC format (Sec. 4.3, Figs. 11-12) the rows are cut
 * into blocks of n_b rows (the paper's "bl"); inside each block the partial
 * diagonals that are dense enough are stored DIA-style (one offset and n_b
 * contiguous values each) and every other nonzero goes to a CSR remainder.
 *
 * Conventions for every call:
 *   - Indices are zero-based int32, sizes int64.  A diagonal's offset is
 *     off = j - i (the kernels of Figs. 5, 9, 10, 13 read x[i + off]).
 *   - Pointers named d_* are device pointers on the current CUDA device;
 *     pointers named h_* are host pointers.  `stream` is a cudaStream_t (NULL
 *     for the legacy default stream).
 *   - The caller keeps ownership of every array it passes; a handle owns the
 *     device arrays it holds and frees them in mhdc_destroy.
 *   - Calls return MHDC_OK (0) or a negative error code; nothing throws across
 *     the ABI.  mhdc_strerror() names a code.
 *   - Value dtype is fixed per handle: F64 handles take FP64 x and write FP64
 *     y; F32 handles take FP32 x and write FP32 y; BF16 handles take BF16 x
 *     and write FP32 y.  Accumulation is FP64 for F64 and FP32 otherwise,
 *     except that a CSR remainder row with more than 64 entries is summed in
 *     FP64 and rounded once into the FP32 accumulator (every product kernel:
 *     mhdc_spmv, mhdc_dia_spmv, mhdc_spmm, the batch calls).
 */
#ifndef MHDC_H
#define MHDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mhdc_matrix *mhdc_handle;
typedef struct sell_matrix *sell_handle;

/* Storage precision of matrix values and x. */
enum mhdc_dtype { MHDC_F64 = 0, MHDC_F32 = 1, MHDC_BF16 = 2 };

/* Which diagonals go to the DIA part (see mhdc_build / hdc_build). */
enum mhdc_mode { MHDC_MODE_BLOCK = 0, MHDC_MODE_GLOBAL = 1 };

enum mhdc_status {
    MHDC_OK = 0,
    MHDC_ERR_INVALID_ARG = -1,   /* bad size, null pointer, unknown dtype, ... */
    MHDC_ERR_BAD_CSR = -2,       /* CSR input fails the checks of mhdc_build */
    MHDC_ERR_OOM = -3,           /* a device allocation failed */
    MHDC_ERR_CUDA = -4,          /* a CUDA runtime call or launch failed */
    MHDC_ERR_UNSUPPORTED = -5,   /* valid request this build does not handle */
    MHDC_ERR_DEVICE_CHECK = -6,  /* a kernel's own bounds check fired */
    MHDC_ERR_TIMEOUT = -7        /* a bounded device-side wait gave up */
};

/* Summary of a built handle (mhdc_info). */
typedef struct {
    int64_t n;             /* rows = columns */
    int64_t nnz;           /* stored entries of the input CSR */
    int64_t nnz_rem;       /* entries in the CSR remainder */
    int64_t P;             /* number of partial diagonals (sum over blocks) */
    int64_t n_blocks;      /* ceil(n / n_b) */
    int32_t n_b;           /* rows per block */
    int32_t dtype;         /* enum mhdc_dtype */
    int32_t mode;          /* enum mhdc_mode */
    int32_t variant;       /* SpMV tile shape in use (-1: default) */
    int32_t emulated_ok;   /* 1: FP64 handle whose values allow variants 10-15, 0: not,
                              -1: not known yet (the FP32-pair arrays are made on first
                              use: mhdc_set_variant(v >= 10) or mhdc_tune) */
    int32_t reserved;
    double theta;          /* density threshold used */
    double alpha;          /* filling rate: (nnz - nnz_rem) / (P * n_b)   (Sec. 5.3.3) */
    double beta;           /* CSR rate: nnz_rem / nnz                     (Sec. 5.3.1) */
    int64_t bytes_model;   /* algorithmic bytes of one y = A x: V_A + V_x + V_y (Sec. 5.1),
                              x read once; csr_row_ptr counted for blocks with a
                              nonempty remainder plus two words per block */
    int64_t bytes_device;  /* device memory held by the handle */
} mhdc_info_t;

/*
 * mhdc_build -- convert a CSR matrix to M-HDC (Sec. 4.3; selection rule of
 * Sec. 4.3, storage of Fig. 12), entirely on the device.
 *
 *   n            rows (= columns), 0 <= n < 2^31 - 1
 *   d_row_ptr    int32[n + 1], row_ptr[0] = 0, nondecreasing, row_ptr[n] = nnz < 2^31
 *   d_col        int32[nnz], columns of each row strictly increasing, in [0, n)
 *   d_val        double[nnz]  (d_col and d_val may be NULL when nnz = 0)
 *   n_b          rows per block, >= 1 (the paper's bl)
 *   theta        density threshold, finite and >= 0: in block ib the partial
 *                diagonal of offset d is kept iff its count N(d, ib) >= 1 and
 *                (double)N >= theta * rows(ib), rows(ib) = min(n_b, n - ib*n_b)
 *   dtype        enum mhdc_dtype: values are rounded to it once, at build
 *                (FP64 -> FP32 nearest-even, then FP32 -> BF16 nearest-even)
 *   stream       stream to run on; the call synchronizes it (sizes are read back)
 *   out          receives the new handle (unchanged on error)
 *
 * The input arrays are only read and may be freed after the call.  Invalid
 * CSR (decreasing row_ptr, column out of range, unsorted or duplicate columns)
 * returns MHDC_ERR_BAD_CSR and builds nothing.  Layout built (device):
 * dia_ptr int32[n_blocks + 1]; dia_offset int32[P], ascending inside a block;
 * dia_val dtype[P * n_b] with dia_val[p * n_b + t] = a(r0 + t, r0 + t + off_p)
 * (+0.0 where that entry is absent or outside the matrix); remainder
 * csr_row_ptr int32[n + 1], csr_col int32[nnz_rem], csr_val dtype[nnz_rem] in
 * the input's order.
 */
int mhdc_build(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
               int32_t n_b, double theta, int32_t dtype, void *stream, mhdc_handle *out);

/*
 * hdc_build -- the HDC format (Sec. 3.4) stored blocked for the B-HDC kernel
 * (Sec. 4.2, Fig. 10): diagonals are chosen over the whole matrix (count
 * N(d) >= 1 and >= theta * n) and every block of n_b rows holds its piece of
 * each chosen diagonal.  Arguments, layout and errors as mhdc_build; the
 * handle works with every other call.
 */
int hdc_build(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
              int32_t n_b, double theta, int32_t dtype, void *stream, mhdc_handle *out);

/*
 * mhdc_build_dia -- the M-HDC format straight from DIA input (the layout of
 * Sec. 3.3, Fig. 4), as a stencil code holds its matrix, without a CSR copy.
 * The entries are the positions (i, i + offset[d]) inside the matrix whose
 * value is nonzero; the handle equals the one mhdc_build gives for the CSR
 * matrix of those entries (same selection of Sec. 4.3, layout of Fig. 12,
 * rounding, remainder in column order), entirely on the device.
 *
 *   n          rows (= columns), 1 <= n < 2^31 - 1; entries fewer than 2^31
 *   nd         number of diagonals, 0 <= nd <= 65535
 *   d_offset   int32[nd] (device), strictly increasing, each in (-n, n)
 *   d_val      double[nd * n] (device): d_val[d * n + i] = a(i, i + offset[d]);
 *              values at positions outside the matrix are ignored, zeros
 *              are not entries
 *   n_b, theta, dtype, stream, out   as mhdc_build (the call synchronizes)
 *
 * The arrays are read only during the call.  Errors: MHDC_ERR_INVALID_ARG
 * for bad sizes or offsets (checked on the device), MHDC_ERR_UNSUPPORTED for
 * 2^31 or more entries, MHDC_ERR_OOM / MHDC_ERR_CUDA.
 */
int mhdc_build_dia(int64_t n, int32_t nd, const int32_t *d_offset, const double *d_val, int32_t n_b,
                   double theta, int32_t dtype, void *stream, mhdc_handle *out);

/*
 * mhdc_spmv -- y = A x with the M-HDC kernel (Fig. 13): for every row block,
 * the remainder rows plus, for each of the block's diagonals, dia_val * x
 * shifted by its offset; y is written once per row (overwritten).
 *
 *   d_x   n values of the handle's x dtype (device)
 *   d_y   n values of the handle's y dtype (device); must not overlap d_x
 * Asynchronous on `stream`; may be captured in a CUDA graph (a replay
 * computes what a direct call computes, for every variant).  Products on one
 * stream may start their launches while the previous kernel drains, but each
 * reads its x only after the stream's earlier work has completed (y of one
 * call may be x of the next).  Products of one handle must not overlap on
 * the GPU (issue them on one stream): the emulated variants split x into a
 * buffer of the handle, and a matrix whose CSR remainder holds 5 % or more
 * of the nonzeros hands its row tiles out through a counter of the handle.
 */
int mhdc_spmv(mhdc_handle A, const void *d_x, void *d_y, void *stream);

/*
 * mhdc_spmv_host -- mhdc_spmv on host buffers: copies h_x (n values, pinned
 * host memory recommended) to a device buffer owned by the handle, runs the
 * product and copies y back to h_y, all on `stream`, then synchronizes it.
 */
int mhdc_spmv_host(mhdc_handle A, const void *h_x, void *h_y, void *stream);

/*
 * mhdc_spmv_host_async -- mhdc_spmv_host without waiting, for a sequence of
 * products on host data: the copy of h_x (pinned host memory, n values of
 * the handle's x dtype) into one of three device slots, the product and
 * the copy of y back to h_y (pinned, n values of the y dtype) are queued on
 * the handle's own streams for copies in, products and copies out, chained
 * by events, so that the copy-in of one call and the copy-out of an earlier
 * one overlap the product between them.  When the call returns, the call
 * made three calls earlier has completed: its h_y holds the result and its
 * h_x / h_y may be reused; h_x and h_y of the last three calls must stay
 * untouched until a later call or mhdc_host_wait.  The caller's streams are
 * not used; the product runs the handle's tile shape (mhdc_set_variant).
 *
 * mhdc_host_wait -- wait until every queued host call of the handle has
 * completed (all h_y written).
 * Neither call is thread-safe for one handle (calls on different handles are
 * independent).
 */
int mhdc_spmv_host_async(mhdc_handle A, const void *h_x, void *h_y);
int mhdc_host_wait(mhdc_handle A);

/*
 * mhdc_spmm -- Y = A X for k right-hand sides (the M-HDC kernel of Fig. 13
 * applied to k vectors at once, reading A once per pass of up to 16 columns).
 *
 *   k        number of right-hand sides, 1 <= k <= 64
 *   d_X      row-major n x k block of x dtype, leading dimension ldx >= k
 *   d_Y      row-major n x k block of y dtype, leading dimension ldy >= k
 * Each (row, column) is summed as mhdc_spmv sums a row: the CSR remainder in
 * column order, then the diagonals in ascending order.  X and Y rows are
 * moved in 16-byte slices when X + column, Y + column and the leading
 * dimensions are aligned to the slice (else element by element).
 * Asynchronous on `stream`.
 *
 * mhdc_spmm_set_variant -- SpMM tile shape v (0..MHDC_NUM_SPMM_VARIANTS-1;
 *   -1: the default, 2): 0, 2, 3 give each lane 3, 4, 5 consecutive rows and
 *   share X rows between the diagonals of a run of consecutive offsets; 1
 *   gives each lane 2 strided rows and loads 2 diagonals at a time.  Every
 *   shape gives the same Y.
 * mhdc_spmm_tune -- time every shape on (d_X, d_Y) with k columns (Y is
 *   overwritten), keep the fastest in the handle, write its id to *best and,
 *   if times_us is not NULL, each shape's mean time in microseconds to
 *   times_us[MHDC_NUM_SPMM_VARIANTS].  Synchronous.
 */
#define MHDC_NUM_SPMM_VARIANTS 4
int mhdc_spmm(mhdc_handle A, int32_t k, const void *d_X, int64_t ldx, void *d_Y, int64_t ldy,
              void *stream);
int mhdc_spmm_set_variant(mhdc_handle A, int32_t v);
int mhdc_spmm_tune(mhdc_handle A, int32_t k, const void *d_X, int64_t ldx, void *d_Y,
                   int64_t ldy, void *stream, int32_t *best, float *times_us);

/*
 * mhdc_dia_spmv -- y = A x in the unblocked DIA order (Sec. 3.3, Fig. 5) for a
 * handle made by hdc_build: y is first set to the CSR remainder's product
 * (zero for rows without remainder), then every diagonal is one pass over
 * all n rows, y[i] += val * x[i + offset], so y is read and written once per
 * diagonal (the main-memory traffic the DIA model of Sec. 5.2 counts).  Each
 * row sees the same operations in the same order as mhdc_spmv, so y is
 * bit-identical to mhdc_spmv on the same handle.
 *
 *   d_x, d_y   as mhdc_spmv (must not overlap)
 * Launches 1 + D kernels (D diagonals) on `stream`, asynchronous.
 * MHDC_ERR_UNSUPPORTED for handles from mhdc_build (block-wise selection:
 * blocks hold different diagonals).
 */
int mhdc_dia_spmv(mhdc_handle A, const void *d_x, void *d_y, void *stream);

/*
 * csr_spmv -- the plain FP64 CSR kernel (Sec. 3.2, Fig. 2): y[i] =
 * sum_k val[k] x[col[k]] over row i.  Arrays as mhdc_build's input (not
 * checked here); d_x, d_y double[n].  Asynchronous on `stream`.
 */
int csr_spmv(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
             const double *d_x, double *d_y, void *stream);

/*
 * mhdc_export -- copy a handle's arrays to host memory (for parity checks).
 * Any pointer may be NULL to skip that array.  Sizes from mhdc_info:
 * dia_ptr int32[n_blocks + 1], dia_offset int32[P], dia_val dtype[P * n_b],
 * csr_row_ptr int32[n + 1], csr_col int32[nnz_rem], csr_val dtype[nnz_rem].
 * Synchronous.
 */
int mhdc_export(mhdc_handle A, int32_t *h_dia_ptr, int32_t *h_dia_offset, void *h_dia_val,
                int32_t *h_csr_row_ptr, int32_t *h_csr_col, void *h_csr_val);

/* mhdc_info -- fill *out with the handle's sizes and statistics. */
int mhdc_info(mhdc_handle A, mhdc_info_t *out);

/*
 * mhdc_stats -- the statistics of the performance model (Sec. 5.3): alpha,
 * the filling rate of the stored diagonals (entries / (P * n_b)); beta, the
 * share of the nonzeros left in the CSR remainder; P, the stored partial
 * diagonals; bytes, the model's main-memory bytes of one product
 * (mhdc_info_t.bytes_model).  Any output pointer may be NULL.  Host call,
 * no device work; MHDC_ERR_INVALID_ARG for a NULL handle.
 */
int mhdc_stats(mhdc_handle A, double *alpha, double *beta, int64_t *P, int64_t *bytes);

/*
 * Tile shapes of the M-HDC product (no counterpart in the paper, whose kernel
 * is a CPU loop nest): variants 0-5 load dia_val into registers (a warp owns
 * 32 x 16 B x U rows and loads D diagonals before accumulating; a matrix too
 * small to fill the GPU with such tiles runs 32-row tiles of one row a lane
 * instead, whatever the variant, with the same sums); variants 6-9
 * stream dia_val through shared memory with TMA bulk copies (one producer
 * warp, several consumer warps, an mbarrier ring; they need n_b * value size
 * to be a multiple of 16 bytes, else they run variant -1).  Variants 0-9
 * and 16-19 compute the same sums in the same order per row (bit-identical y).
 * Variants 10-15 (FP64 handles only; others run variant -1) emulate the FP64
 * product (10-12 in registers, 13-15 streamed by TMA like 6-9) with pairs of
 * FP32 numbers (values and x split into hi + lo, about
 * 49 significant bits; products and sums by error-free transformations): on
 * GB300 the FP64 pipe is about 64x slower than FP32, and these variants move
 * the arithmetic to the FP32 pipe.  Their per-row error stays below
 * (5.2 k + 18) 2^-48 sum_j |a_ij||x_j| for a row of k terms, under 9.6e-13 *
 * sum_j |a_ij||x_j| (inside the FP64 tolerance 1e-12), as long as every
 * nonzero |a_ij| and |x_j| lies in [2^-45, 2^60] and a row has at most 48
 * terms.  The handle checks its values and row lengths at build (outside the
 * window every emulated variant runs variant -1); each product splits x on
 * the device, and a row that reads an x outside the window (or not finite) is
 * computed with the native FP64 arithmetic instead -- the bits variant -1
 * gives for that row.
 * Variants 16-19 stage both operands in shared memory with TMA bulk copies:
 * the values as in 6-9 and, per run of nearby diagonals of a block, one
 * window of x that every diagonal of the run reads (the 27 diagonals of a
 * 27-point stencil share 3 windows).  They need what 6-9 need and a 16-byte
 * aligned x (else they run variant -1), and give the same y as 0-9.
 *
 * mhdc_set_variant -- use variant v for this handle (-1: default chosen from n_b).
 *                     The first v in 10-15 on an FP64 handle makes its FP32-pair
 *                     arrays (device memory as large as dia_val and csr_val)
 *                     on the legacy default stream and waits for them; if they
 *                     cannot be allocated it returns MHDC_ERR_OOM, keeps no part
 *                     of them and leaves the variant unchanged.
 * mhdc_tune        -- (makes the FP32-pair arrays of an FP64 handle first, as
 *                     mhdc_set_variant does, with the same MHDC_ERR_OOM rule)
 *                     time every variant on (d_x, d_y) (overwriting d_y), keep
 *                     the fastest in the handle, write its id to *best and, if
 *                     times_us is not NULL, each variant's mean time in
 *                     microseconds to times_us[MHDC_NUM_VARIANTS].  Synchronous.
 */
#define MHDC_NUM_VARIANTS 20
int mhdc_set_variant(mhdc_handle A, int32_t v);
int mhdc_tune(mhdc_handle A, const void *d_x, void *d_y, void *stream, int32_t *best,
              float *times_us);

/*
 * mhdc_check -- read and clear the handle's device status word: returns
 * MHDC_ERR_DEVICE_CHECK if a bounds check of a checked product (below)
 * failed, else MHDC_ERR_TIMEOUT if a bounded device-side wait of an earlier
 * product on this handle gave up (its y is then incomplete), else MHDC_OK.
 * Synchronizes the device.
 *
 * mhdc_set_checked -- on = 1: from now on mhdc_spmv and mhdc_spmv_host(_async)
 * on this handle run a bounds-checked product (the default tile shape,
 * whatever mhdc_set_variant chose): before every access the index into
 * dia_ptr, dia_offset, dia_val, csr_row_ptr, csr_col, csr_val, x and y is
 * compared with that array's extent; a failed check skips the access (the
 * term counts as 0, a y row is not written) and mhdc_check reports it.  An
 * in-bounds product gives the same y as the unchecked default.  A debugging
 * aid, slower than the tuned kernels; the other products (SpMM, DIA order,
 * batch) are not affected.  on = 0 switches it off.  Host-only.
 */
int mhdc_check(mhdc_handle A);
int mhdc_set_checked(mhdc_handle A, int32_t on);

/*
 * Batched product: y_i = A_i x_i for m handles in one persistent launch (no
 * counterpart in the paper; it serves many small systems, where one launch
 * per matrix leaves the GPU idle).  Warps take chunks of row tiles of all
 * matrices from a global counter, so uneven sizes balance.
 *
 * mhdc_batch_create  -- batch of m >= 1 handles of one dtype (host array
 *                       `mats`); the handles must outlive the batch, which
 *                       only references them.  Every matrix runs the native
 *                       arithmetic of its dtype (the register tile of
 *                       variants 0-5), whatever its handle's variant.
 *                       Synchronous.
 * mhdc_batch_spmv    -- one launch on `stream`: d_xs and d_ys are DEVICE arrays
 *                       of m device pointers (x_i: n_i values of the x dtype,
 *                       y_i: n_i values of the y dtype).  Launches of one batch
 *                       must not overlap on the GPU (they share a counter).
 * mhdc_batch_spmv_graph -- the same launch captured once in a CUDA graph (on a
 *                       stream owned by the batch) and replayed on `stream`;
 *                       recaptured when d_xs or d_ys change.  The pointer
 *                       arrays are read at run time, so their contents (and the
 *                       vectors) may change between replays.
 * mhdc_batch_destroy -- free the batch (not the handles).
 */
typedef struct mhdc_batch *mhdc_batch_handle;
int mhdc_batch_create(int32_t m, const mhdc_handle *mats, mhdc_batch_handle *out);
int mhdc_batch_spmv(mhdc_batch_handle B, const void *const *d_xs, void *const *d_ys, void *stream);
int mhdc_batch_spmv_graph(mhdc_batch_handle B, const void *const *d_xs, void *const *d_ys,
                          void *stream);
int mhdc_batch_destroy(mhdc_batch_handle B);

/*
 * Parameter selection (an extension of Sec. 6.4.3 and Sec. 7: the
 * paper fixes theta = 0.6 and a swept block width, and leaves the choice of
 * format as future work).  A candidate is (n_b, theta, dtype) from a fixed
 * grid of MHDC_NUM_CANDIDATES: dtype in {F64, F32, BF16} (index / 15),
 * n_b in {512, 1024, 2048, 4096, 8192} ((index % 15) / 3), theta in
 * {0.5, 0.6, 0.8} (index % 3).
 *
 * mhdc_candidate   -- candidate idx as an mhdc_params.
 * mhdc_features    -- MHDC_NUM_FEATURES floats to host h_features: for block
 *                     sizes 256, 1024, 4096, the fraction of stored entries
 *                     on partial diagonals whose filling rate N(d,ib)/rows(ib)
 *                     falls in each of 10 bins, then log1p(diagonals per
 *                     block in each bin) / 8; then log2(1 + nnz/n) / 6,
 *                     log2(n) / 24, log2(1 + nnz) / 32 and 1.  Computed on the
 *                     device from a valid CSR (see mhdc_build).  Synchronous.
 * mhdc_autotune    -- the exhaustive autotuner: builds every candidate and
 *                     times `reps` products of each (default tile shape);
 *                     h_times_us[MHDC_NUM_CANDIDATES] receives the mean time
 *                     in microseconds, or -1 for a candidate that could not
 *                     be built for lack of memory.  Synchronous.
 * mhdc_select      -- choose parameters for a CSR matrix and a tolerance tol
 *                     on the per-row error relative to sum_j |a_ij||x_j|: a
 *                     dtype is allowed if its worst-case bound for rows of
 *                     nnz/n terms is <= tol (F64 always).  flags:
 *                     MHDC_SELECT_PAPER (0): theta 0.6, n_b 4096, cheapest
 *                       allowed dtype (the paper's fixed policy);
 *                     MHDC_SELECT_MLP: the candidate the MLP `mlp` predicts
 *                       fastest (mlp maps MHDC_NUM_FEATURES to
 *                       MHDC_NUM_CANDIDATES predicted log relative times);
 *                     MHDC_SELECT_AUTOTUNE: the fastest measured candidate;
 *                     MHDC_SELECT_MODEL: the fewest bytes by the paper's
 *                       model (Sec. 5.3.3) evaluated on the features.
 *                     Synchronous.
 *
 * The MLP (no counterpart in the paper): n_in -> n_hidden -> n_hidden ->
 * n_out, ReLU after the hidden layers, FP32 parameters W1 [h x in], b1 [h],
 * W2 [h x h], b2 [h], W3 [out x h], b3 [out] (contiguous in that order),
 * He-uniform initialisation from `seed`.  Batches are row-major device
 * arrays: X [batch x n_in], Y / T / M [batch x n_out].  The loss is the
 * masked mean squared error sum M (Y - T)^2 / sum M; mhdc_mlp_grad returns
 * its gradient (host array of mhdc_mlp_num_params floats) and value;
 * mhdc_mlp_train_step applies one Adam step (b1 0.9, b2 0.999, eps 1e-8).
 */
#define MHDC_NUM_FEATURES 64
#define MHDC_NUM_CANDIDATES 45
enum { MHDC_SELECT_PAPER = 0, MHDC_SELECT_MLP = 1, MHDC_SELECT_AUTOTUNE = 2, MHDC_SELECT_MODEL = 4 };
typedef struct {
    int32_t n_b;
    int32_t dtype;
    double theta;
    int32_t variant;
    int32_t reserved;
} mhdc_params;
typedef struct mhdc_mlp *mhdc_mlp_handle;

int mhdc_num_candidates(void);
int mhdc_candidate(int32_t idx, mhdc_params *out);
int mhdc_features(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, void *stream,
                  float *h_features);
int mhdc_autotune(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
                  int32_t reps, void *stream, float *h_times_us);
int mhdc_select(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
                double tol, int32_t flags, mhdc_mlp_handle mlp, void *stream, mhdc_params *out);
int mhdc_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed,
                    mhdc_mlp_handle *out);
int64_t mhdc_mlp_num_params(mhdc_mlp_handle M);
int mhdc_mlp_get_params(mhdc_mlp_handle M, float *h_params);
int mhdc_mlp_set_params(mhdc_mlp_handle M, const float *h_params);
int mhdc_mlp_forward(mhdc_mlp_handle M, int32_t batch, const float *d_X, float *d_Y, void *stream);
int mhdc_mlp_grad(mhdc_mlp_handle M, int32_t batch, const float *d_X, const float *d_T,
                  const float *d_M, float *h_grads, float *h_loss, void *stream);
int mhdc_mlp_train_step(mhdc_mlp_handle M, int32_t batch, const float *d_X, const float *d_T,
                        const float *d_M, float lr, void *stream, float *h_loss);
int mhdc_mlp_destroy(mhdc_mlp_handle M);

/* mhdc_destroy -- free the handle and its device arrays (NULL is a no-op). */
int mhdc_destroy(mhdc_handle A);

/* mhdc_strerror -- static text for a status code. */
const char *mhdc_strerror(int code);

/* mhdc_last_error -- details of the last failed call on this host thread
 * (which call or kernel, and the CUDA error text); "" if none yet. */
const char *mhdc_last_error(void);

/*
 * Allocation-failure injection, for testing the cleanup paths of every call
 * (the paper has no counterpart).  Every device allocation of the library
 * (cudaMalloc and its stream-ordered pool) passes one host-side counter.
 *
 * mhdc_debug_fail_alloc -- from now on, the n-th allocation attempt fails as
 *   if the device were out of memory (nothing is allocated and no CUDA call
 *   is made; the calling entry point returns MHDC_ERR_OOM after releasing
 *   what it had allocated).  n = 0 disarms.  Resets the attempt counter.
 *   Setting the environment variable MHDC_FAULT_ALLOC=n arms the same hook
 *   for the whole process at its first allocation.  Not thread-safe against
 *   concurrent library calls that allocate.
 * mhdc_debug_alloc_stats -- allocation attempts since the last arming, and
 *   allocations made and not yet freed by the library (any pointer may be
 *   NULL).  Host-only; always MHDC_OK.
 */
int mhdc_debug_fail_alloc(int64_t n);
int mhdc_debug_alloc_stats(int64_t *attempts, int64_t *live);

/*
 * mhdc_stream_bench -- the paper's memory benchmarks (Sec. 6.2, Figs. 19-20)
 * on the device: C[i] += A[i] * B[i] (indirect == 0) or C[i] += A[i] * B[I[i]]
 * (indirect != 0), FP64 arrays of N elements and an int32 index array.
 * Used to measure the effective bandwidth w_mem of Eq. (2).  Asynchronous.
 */
int mhdc_stream_bench(int64_t N, const double *d_A, const double *d_B, const int32_t *d_I,
                      double *d_C, int32_t indirect, void *stream);

/*
 * mhdc_read_bench -- read-only member of the memory benchmarks above: each of
 * mhdc_read_bench_ctas() CTAs writes the bitwise XOR of the 64-bit words of
 * its share of d_A (N doubles, N even, d_A 16-byte aligned) to d_out[cta]
 * (d_out read as uint64).  It measures the bandwidth a kernel that only reads
 * can reach (SpMV traffic is almost all reads: V_A + V_x against V_y,
 * Sec. 5.1) with integer work only, so the FP64 pipe does not limit it.
 * Asynchronous.
 */
int mhdc_read_bench(int64_t N, const double *d_A, double *d_out, void *stream);
int mhdc_read_bench_ctas(void);

/*
 * mhdc_fma_bench -- arithmetic-throughput probe (no counterpart in the paper):
 * mhdc_read_bench_ctas() CTAs of 256 threads each run iters rounds of 8
 * independent FMA chains, in FP64 if fp64 != 0 else FP32, and write one
 * value per thread to d_out (double or float, ctas * 256 entries).  Timing it
 * gives the measured FMA rate: total FMAs = ctas * 256 * 8 * iters.  On GB300
 * the FP64 rate, not HBM, bounds an FP64 SpMV.  Asynchronous.
 */
int mhdc_fma_bench(int32_t fp64, int32_t iters, void *d_out, void *stream);

/*
 * mhdc_build_noalloc -- the conversion of mhdc_build, written into arrays the
 * caller provides, with no device memory allocated by the call.  The paper
 * has no counterpart; this exists for callers that cannot allocate device
 * memory: a process that carves all its device memory out of one pool at
 * start-up, code on a latency-critical path where cudaMalloc would stall or
 * fail, or a binding that may only pass buffers it already owns.
 *
 * Limits: n <= 262144 rows and nnz <= 262144 stored entries; larger inputs
 * return MHDC_ERR_INVALID_ARG with a message saying so.  All temporaries live
 * in one file-scope device array of about 14 MB, which every GPU that loads
 * this library holds until the process exits.  Every call looks that
 * array's address up (cudaGetSymbolAddress) with the calling thread's device
 * current, so a device reset between calls is harmless; the first call on a
 * device also loads the library's conversion kernels there, so make it before
 * any stream capture.
 * Every call shares the array and it keeps the last call's contents: calls
 * that overlap on the GPU (other streams, other threads) race and must not be
 * issued; the call clears what must start at zero itself.
 *
 *   n, d_row_ptr, d_col, d_val, n_b, theta, dtype
 *                as mhdc_build (n >= 1; d_col, d_val may be NULL if nnz = 0)
 *   d_dia_ptr    int32[ceil(n / n_b) + 1]                     (output)
 *   d_dia_offset int32[cap_P], d_dia_val dtype[cap_P * n_b]  (output)
 *   d_csr_row_ptr int32[n + 1]                                (output)
 *   d_csr_col    int32[cap_rem], d_csr_val dtype[cap_rem]     (output)
 *   h_P, h_nnz_rem  host: receive P and the remainder's nnz
 *   stream       stream to run on; the call synchronizes it
 * Output layout and values are exactly those mhdc_export returns for the
 * same input.  If P > cap_P or nnz_rem > cap_rem the call returns
 * MHDC_ERR_INVALID_ARG with the sizes needed in *h_P / *h_nnz_rem (cap_rem =
 * nnz always suffices; P <= nnz).  Invalid CSR returns MHDC_ERR_BAD_CSR.
 */
int mhdc_build_noalloc(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col,
                       const double *d_val, int32_t n_b, double theta, int32_t dtype,
                       int32_t *d_dia_ptr, int32_t *d_dia_offset, void *d_dia_val, int64_t cap_P,
                       int32_t *d_csr_row_ptr, int32_t *d_csr_col, void *d_csr_val,
                       int64_t cap_rem, int64_t *h_P, int64_t *h_nnz_rem, void *stream);

/*
 * SELL-C-sigma baseline (Kreutzer, Hager, Wellein, Fehske, Bishop, SIAM J.
 * Sci. Comput. 36(5), 2014): the ELL-type format the paper leaves to future
 * work (Sec. 7), for comparison with CSR and M-HDC on the same GPU.  FP64.
 *
 * sell_build -- from CSR (arrays as mhdc_build, not checked beyond
 *   row_ptr[n]): rows sorted by length, longest first, inside windows of
 *   sigma rows (ties keep input order); chunks of C consecutive sorted rows,
 *   each padded to its longest row and stored column by column (slot
 *   chunk_ptr[c] + k * C + r holds entry k of row r of chunk c; padding:
 *   column 0, value +0.0).  1 <= C <= 1024 (32 = one warp per chunk),
 *   1 <= sigma <= 8192 (1: no sorting).  Synchronizes `stream`; *out
 *   receives the handle (device memory owned by it).
 * sell_spmv -- y = A x (FP64 device arrays of n values; must not overlap):
 *   one thread per sorted row sums its own entries (never the padding) in
 *   column order with one FMA each, so y is bit-identical to csr_spmv.
 *   Asynchronous on `stream`.
 * sell_info -- rows, entries, stored slots (entries + padding), chunks.
 * sell_export -- copy perm[n] (input row of each sorted position),
 *   rowlen[n] (its length), chunk_ptr[chunks + 1], col[slots], val[slots] to
 *   host memory; any pointer may be NULL.  Synchronous.
 * sell_destroy -- free the handle (waits for the device).
 * Errors as mhdc_build; MHDC_ERR_UNSUPPORTED past 2^31 - 1 slots.
 */
int sell_build(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col, const double *d_val,
               int32_t C, int32_t sigma, void *stream, sell_handle *out);
int sell_spmv(sell_handle S, const double *d_x, double *d_y, void *stream);
int sell_info(sell_handle S, int64_t *n, int64_t *nnz, int64_t *slots, int64_t *chunks);
int sell_export(sell_handle S, int32_t *h_perm, int32_t *h_rowlen, int32_t *h_chunk_ptr,
                int32_t *h_col, double *h_val);
int sell_destroy(sell_handle S);

#ifdef __cplusplus
}
#endif

#endif /* MHDC_H */
