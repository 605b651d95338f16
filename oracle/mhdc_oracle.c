/*
 * CPU oracle for the M-HDC sparse matrix-vector product.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file; the product library never
 * does, and this file shares no code with it.  Everything here is plain,
 * sequential-per-row FP64 C written to be checked against the paper by eye:
 *
 *   Fukaya, Ishida, Miura, Iwashita, Nakashima, "Accelerating the SpMV kernel
 *   on standard CPUs by exploiting the partially diagonal structures"
 *   (arXiv 2105.04937).
 *
 * Notation follows the paper: a row block has `bl` rows (block ib covers rows
 * [ib*bl, min((ib+1)*bl, n))), a diagonal offset is off = j - i (the sign the
 * paper's kernels use when they read x[i+off]), theta is the density
 * threshold, dia_ptr / dia_offset / dia_val / csr_row_ptr / csr_col_ind /
 * csr_val are the arrays of the M-HDC format (Sec. 4.3, Fig. 12).
 *
 * Readings taken where the paper is silent (each is also a test):
 *   - a partial diagonal is selected iff its count is >= 1 and
 *     (double)count >= theta * (double)rows(ib), rows(ib) = rows of the block
 *     (the last block may be short); positions outside the matrix count in
 *     the denominator, as in the paper's worked example (Fig. 11);
 *   - within a block the selected offsets are stored in ascending order;
 *   - dia_val of partial diagonal p is bl long and indexed by the local row
 *     t = i - ib*bl (Fig. 12); absent and out-of-range positions hold +0.0;
 *   - the CSR remainder keeps the input's row and column order;
 *   - reduced-precision storage rounds FP64 -> FP32 to nearest-even and then
 *     FP32 -> BF16 to nearest-even (both written here from IEEE 754).
 *
 * Parity status: every function below is pinned by the CPU tests (the
 * paper's worked examples, dense brute force, closed forms, round trips,
 * library rounding); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_F64 = 0, ORC_F32 = 1, ORC_BF16 = 2 };

/* ------------------------------------------------------------------------ */
/* CSR input check (Sec. 3.2: zero-based row_ptr, col_ind; row_ptr[n] = nnz) */
/* Returns 0 if valid; 1 row_ptr[0] != 0; 2 row_ptr decreasing; 3 column out
 * of [0, n); 4 columns of a row not strictly increasing (unsorted/duplicate). */
int orc_csr_check(int64_t n, const int32_t *row_ptr, const int32_t *col)
{
    if (row_ptr[0] != 0) return 1;
    for (int64_t i = 0; i < n; i++)
        if (row_ptr[i + 1] < row_ptr[i]) return 2;
    for (int64_t i = 0; i < n; i++) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
            if (col[k] < 0 || (int64_t)col[k] >= n) return 3;
            if (k > row_ptr[i] && col[k] <= col[k - 1]) return 4;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The CSR kernel (Fig. 2): y[i] = sum_k val[k] * x[col_ind[k]].             */
void orc_csr_spmv(int64_t n, const int32_t *row_ptr, const int32_t *col,
                  const double *val, const double *x, double *y, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
            s += val[k] * x[col[k]];
        y[i] = s;
    }
}

/* sum_j |a_ij| |x_j| for every row. */
void orc_csr_absrow(int64_t n, const int32_t *row_ptr, const int32_t *col,
                    const double *val, const double *x, double *out, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; i++) {
        double a = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
            a += fabs(val[k]) * fabs(x[col[k]]);
        out[i] = a;
    }
}

/* ------------------------------------------------------------------------ */
/* Rounding to the storage precisions, from the IEEE 754 definitions.        */

/* FP64 -> FP32, round to nearest, ties to even. */
static uint32_t f64_to_f32_bits(double v)
{
    uint64_t u;
    memcpy(&u, &v, 8);
    uint32_t sign = (uint32_t)(u >> 63) << 31;
    int e = (int)((u >> 52) & 0x7FF);
    uint64_t m = u & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF)                                 /* inf or NaN */
        return m ? (sign | 0x7FC00000u | (uint32_t)(m >> 29)) : (sign | 0x7F800000u);
    if (e == 0) return sign;                        /* FP64 zero/subnormal: < 2^-1022 */
    int E = e - 1023;                               /* value = sig * 2^(E-52) */
    uint64_t sig = (1ull << 52) | m;
    uint64_t q, rem, half;
    if (E >= -126) {                                /* FP32 normal range */
        q = sig >> 29;
        rem = sig & ((1ull << 29) - 1);
        half = 1ull << 28;
        if (rem > half || (rem == half && (q & 1))) q++;
        if (q == (1ull << 24)) { q >>= 1; E++; }
        if (E > 127) return sign | 0x7F800000u;     /* overflow to infinity */
        return sign | ((uint32_t)(E + 127) << 23) | (uint32_t)(q & 0x7FFFFF);
    }
    /* FP32 subnormal: units of 2^-149, q = sig * 2^(E-52+149) */
    int shift = -97 - E;
    if (shift > 53) return sign;                    /* below half the smallest subnormal */
    q = sig >> shift;
    rem = sig & ((1ull << shift) - 1);
    half = 1ull << (shift - 1);
    if (rem > half || (rem == half && (q & 1))) q++;
    return sign | (uint32_t)q;                      /* q == 2^23 encodes the smallest normal */
}

/* FP32 -> BF16 (upper 16 bits), round to nearest, ties to even. */
static uint16_t f32_to_bf16_bits(uint32_t u)
{
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x7FFFFFu))
        return (uint16_t)((u >> 16) | 0x40);        /* NaN stays a (quiet) NaN */
    uint32_t q = u >> 16, rem = u & 0xFFFFu;
    if (rem > 0x8000u || (rem == 0x8000u && (q & 1))) q++;
    return (uint16_t)q;                             /* a carry into the exponent is correct */
}

void orc_round_f32(int64_t m, const double *in, float *out)
{
    for (int64_t k = 0; k < m; k++) {
        uint32_t b = f64_to_f32_bits(in[k]);
        memcpy(&out[k], &b, 4);
    }
}

void orc_round_bf16(int64_t m, const double *in, uint16_t *out)
{
    for (int64_t k = 0; k < m; k++) out[k] = f32_to_bf16_bits(f64_to_f32_bits(in[k]));
}

void orc_bf16_to_f64(int64_t m, const uint16_t *in, double *out)
{
    for (int64_t k = 0; k < m; k++) {
        uint32_t b = (uint32_t)in[k] << 16;
        float f;
        memcpy(&f, &b, 4);
        out[k] = (double)f;
    }
}

static void store_value(int dtype, void *dst, int64_t pos, double v)
{
    if (dtype == ORC_F64) {
        ((double *)dst)[pos] = v;
    } else if (dtype == ORC_F32) {
        uint32_t b = f64_to_f32_bits(v);
        memcpy(&((float *)dst)[pos], &b, 4);
    } else {
        ((uint16_t *)dst)[pos] = f32_to_bf16_bits(f64_to_f32_bits(v));
    }
}

/* ------------------------------------------------------------------------ */
/* CSR -> M-HDC / B-HDC conversion (Sec. 3.4 and 4.3).                       */

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static int64_t rows_of_block(int64_t n, int64_t bl, int64_t ib)
{
    int64_t r0 = ib * bl;
    return (n - r0 < bl) ? (n - r0) : bl;
}

/*
 * Step 1 of the conversion: choose the (partial) diagonals kept in DIA form.
 *
 * global == 0 (M-HDC, Sec. 4.3): in block ib, count the stored entries on
 *   each offset d, N(d, ib), and keep d iff N >= 1 and N >= theta * rows(ib).
 * global == 1 (HDC, Sec. 3.4, stored blocked as the B-HDC kernel reads it):
 *   count N(d) over the whole matrix, keep d iff N >= 1 and N >= theta * n,
 *   and give every block the same list.
 *
 * Writes dia_ptr[n_blocks + 1] and the ascending offsets of each block into
 * dia_offset (capacity cap).  Returns the total number of partial diagonals,
 * or -1 if cap is too small.
 */
int64_t orc_select(int64_t n, const int32_t *row_ptr, const int32_t *col,
                   int64_t bl, double theta, int global,
                   int32_t *dia_ptr, int32_t *dia_offset, int64_t cap)
{
    int64_t n_blocks = (n + bl - 1) / bl;
    int64_t P = 0;
    dia_ptr[0] = 0;
    if (global) {
        /* N(d) for d in [-(n-1), n-1], indexed by d + n - 1 */
        int64_t *cnt = (int64_t *)calloc((size_t)(2 * n), sizeof(int64_t));
        int64_t nsel = 0;
        for (int64_t i = 0; i < n; i++)
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
                cnt[(int64_t)col[k] - i + n - 1]++;
        int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * n));
        for (int64_t d = -(n - 1); d <= n - 1; d++) {
            int64_t c = cnt[d + n - 1];
            if (c >= 1 && (double)c >= theta * (double)n) sel[nsel++] = (int32_t)d;
        }
        free(cnt);
        for (int64_t ib = 0; ib < n_blocks; ib++) {
            if (P + nsel > cap) { free(sel); return -1; }
            for (int64_t s = 0; s < nsel; s++) dia_offset[P + s] = sel[s];
            P += nsel;
            dia_ptr[ib + 1] = (int32_t)P;
        }
        free(sel);
        return P;
    }
    int64_t maxblk = 0;
    for (int64_t ib = 0; ib < n_blocks; ib++) {
        int64_t r0 = ib * bl, r1 = r0 + rows_of_block(n, bl, ib);
        int64_t m = (int64_t)row_ptr[r1] - row_ptr[r0];
        if (m > maxblk) maxblk = m;
    }
    int64_t *offs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxblk > 0 ? maxblk : 1));
    for (int64_t ib = 0; ib < n_blocks; ib++) {
        int64_t rows = rows_of_block(n, bl, ib);
        int64_t r0 = ib * bl, r1 = r0 + rows;
        int64_t m = 0;
        for (int64_t i = r0; i < r1; i++)
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
                offs[m++] = (int64_t)col[k] - i;
        qsort(offs, (size_t)m, sizeof(int64_t), cmp_i64);
        for (int64_t a = 0; a < m;) {
            int64_t b = a;
            while (b < m && offs[b] == offs[a]) b++;
            int64_t c = b - a;                      /* N(d, ib) for d = offs[a] */
            if (c >= 1 && (double)c >= theta * (double)rows) {
                if (P >= cap) { free(offs); return -1; }
                dia_offset[P++] = (int32_t)offs[a];
            }
            a = b;
        }
        dia_ptr[ib + 1] = (int32_t)P;
    }
    free(offs);
    return P;
}

/* Position of offset d in the ascending list s[0..m), or -1. */
static int64_t find_offset(const int32_t *s, int64_t m, int64_t d)
{
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (s[mid] < d) lo = mid + 1; else hi = mid;
    }
    return (lo < m && s[lo] == d) ? lo : -1;
}

/*
 * Step 2 of the conversion (Fig. 12): scatter every stored entry either into
 * dia_val[p * bl + (i - r0)] of its block's selected diagonal p, or into the
 * CSR remainder (input order kept).  dia_val (P * bl slots, dtype `dtype`) is
 * filled with +0.0 first.  csr_row_ptr has n + 1 entries; csr_col / csr_val
 * need room for nnz entries.  Returns the remainder's nnz.
 */
int64_t orc_fill(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
                 int64_t bl, int dtype, const int32_t *dia_ptr, const int32_t *dia_offset,
                 void *dia_val, int32_t *csr_row_ptr, int32_t *csr_col, void *csr_val)
{
    int64_t n_blocks = (n + bl - 1) / bl;
    int64_t P = dia_ptr[n_blocks];
    for (int64_t s = 0; s < P * bl; s++) store_value(dtype, dia_val, s, 0.0);
    int64_t nr = 0;
    csr_row_ptr[0] = 0;
    for (int64_t ib = 0; ib < n_blocks; ib++) {
        int64_t r0 = ib * bl, r1 = r0 + rows_of_block(n, bl, ib);
        const int32_t *sel = dia_offset + dia_ptr[ib];
        int64_t nsel = dia_ptr[ib + 1] - dia_ptr[ib];
        for (int64_t i = r0; i < r1; i++) {
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
                int64_t p = find_offset(sel, nsel, (int64_t)col[k] - i);
                if (p >= 0) {
                    store_value(dtype, dia_val, (dia_ptr[ib] + p) * bl + (i - r0), val[k]);
                } else {
                    csr_col[nr] = col[k];
                    store_value(dtype, csr_val, nr, val[k]);
                    nr++;
                }
            }
            csr_row_ptr[i + 1] = (int32_t)nr;
        }
    }
    return nr;
}

/*
 * HDC in the paper's unblocked form (Sec. 3.4, Fig. 7): the selected global
 * diagonals stored n long and indexed by row, dia_val[d * n + i] = a(i, i+off_d).
 * Returns the number of selected diagonals (at most cap) and fills the
 * remainder like orc_fill.  *nnz_rem receives the remainder's nnz.
 */
int64_t orc_hdc_global(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
                       double theta, int32_t *dia_offset, int64_t cap, double *dia_val,
                       int32_t *csr_row_ptr, int32_t *csr_col, double *csr_val, int64_t *nnz_rem)
{
    int32_t dptr[2];
    int64_t nd = orc_select(n, row_ptr, col, n, theta, 1, dptr, dia_offset, cap);
    if (nd < 0) return -1;
    for (int64_t s = 0; s < nd * n; s++) dia_val[s] = 0.0;
    int64_t nr = 0;
    csr_row_ptr[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
            int64_t p = find_offset(dia_offset, nd, (int64_t)col[k] - i);
            if (p >= 0) {
                dia_val[p * n + i] = val[k];
            } else {
                csr_col[nr] = col[k];
                csr_val[nr] = val[k];
                nr++;
            }
        }
        csr_row_ptr[i + 1] = (int32_t)nr;
    }
    *nnz_rem = nr;
    return nd;
}

/* ------------------------------------------------------------------------ */
/* The M-HDC kernel (Fig. 13), FP64, over the row blocks [ib_begin, ib_end).
 * Per block: the CSR rows of the block first (y[i] = s), then
 * y[i] += dia_val[k][i - r0] * x[i + off] over the block's diagonals k, for
 * the rows i of the block with 0 <= i + off < n.  Reduced-precision handles
 * are evaluated here on their stored values widened to FP64. */
void orc_mhdc_spmv_range(int64_t n, int64_t bl, int64_t ib_begin, int64_t ib_end,
                         const int32_t *dia_ptr, const int32_t *dia_offset,
                         const double *dia_val, const int32_t *csr_row_ptr,
                         const int32_t *csr_col, const double *csr_val, const double *x,
                         double *y, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t ib = ib_begin; ib < ib_end; ib++) {
        int64_t r0 = ib * bl, r1 = r0 + rows_of_block(n, bl, ib);
        for (int64_t i = r0; i < r1; i++) {
            double s = 0.0;
            for (int64_t k = csr_row_ptr[i]; k < csr_row_ptr[i + 1]; k++)
                s += csr_val[k] * x[csr_col[k]];
            y[i] = s;
        }
        for (int64_t k = dia_ptr[ib]; k < dia_ptr[ib + 1]; k++) {
            int64_t off = dia_offset[k];
            int64_t is = r0 > -off ? r0 : -off;
            int64_t ie = r1 < n - off ? r1 : n - off;
            for (int64_t i = is; i < ie; i++)
                y[i] += dia_val[k * bl + (i - r0)] * x[i + off];
        }
    }
}

void orc_mhdc_spmv(int64_t n, int64_t bl, const int32_t *dia_ptr, const int32_t *dia_offset,
                   const double *dia_val, const int32_t *csr_row_ptr, const int32_t *csr_col,
                   const double *csr_val, const double *x, double *y, int nthreads)
{
    orc_mhdc_spmv_range(n, bl, 0, (n + bl - 1) / bl, dia_ptr, dia_offset, dia_val, csr_row_ptr,
                        csr_col, csr_val, x, y, nthreads);
}

/* Round trip: list the nonzero entries held by an M-HDC structure (DIA
 * positions inside the matrix with a nonzero value, then the remainder), as
 * (row, col, value).  Returns the number written (room for cap). */
int64_t orc_mhdc_to_coo(int64_t n, int64_t bl, const int32_t *dia_ptr, const int32_t *dia_offset,
                        const double *dia_val, const int32_t *csr_row_ptr, const int32_t *csr_col,
                        const double *csr_val, int64_t cap, int64_t *ro, int32_t *co, double *vo)
{
    int64_t n_blocks = (n + bl - 1) / bl;
    int64_t m = 0;
    for (int64_t ib = 0; ib < n_blocks; ib++) {
        int64_t r0 = ib * bl, rows = rows_of_block(n, bl, ib);
        for (int64_t k = dia_ptr[ib]; k < dia_ptr[ib + 1]; k++) {
            for (int64_t t = 0; t < rows; t++) {
                int64_t i = r0 + t, j = i + dia_offset[k];
                double v = dia_val[k * bl + t];
                if (j < 0 || j >= n || v == 0.0) continue;
                if (m >= cap) return -1;
                ro[m] = i; co[m] = (int32_t)j; vo[m] = v; m++;
            }
        }
    }
    for (int64_t i = 0; i < n; i++)
        for (int64_t k = csr_row_ptr[i]; k < csr_row_ptr[i + 1]; k++) {
            if (m >= cap) return -1;
            ro[m] = i; co[m] = csr_col[k]; vo[m] = csr_val[k]; m++;
        }
    return m;
}

/* Per-row sum_j |a_ij| |x_j| and term count of an M-HDC structure (DIA
 * positions inside the matrix, including stored zeros, plus the remainder). */
void orc_mhdc_absrow(int64_t n, int64_t bl, const int32_t *dia_ptr, const int32_t *dia_offset,
                     const double *dia_val, const int32_t *csr_row_ptr, const int32_t *csr_col,
                     const double *csr_val, const double *x, double *abs_out, int64_t *terms_out)
{
    int64_t n_blocks = (n + bl - 1) / bl;
    for (int64_t ib = 0; ib < n_blocks; ib++) {
        int64_t r0 = ib * bl, r1 = r0 + rows_of_block(n, bl, ib);
        for (int64_t i = r0; i < r1; i++) {
            double a = 0.0;
            int64_t t = 0;
            for (int64_t k = csr_row_ptr[i]; k < csr_row_ptr[i + 1]; k++, t++)
                a += fabs(csr_val[k]) * fabs(x[csr_col[k]]);
            for (int64_t k = dia_ptr[ib]; k < dia_ptr[ib + 1]; k++) {
                int64_t j = i + dia_offset[k];
                t++;
                if (j >= 0 && j < n) a += fabs(dia_val[k * bl + (i - r0)]) * fabs(x[j]);
            }
            abs_out[i] = a;
            terms_out[i] = t;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* The memory benchmarks of Sec. 6.2 (Figs. 19 and 20), FP64 with INT32 index. */
/* ------------------------------------------------------------------------ */
/* DIA input (Sec. 3.3, Fig. 4) -> CSR (Sec. 3.2).  val[d * n + i] holds
 * a(i, i + offset[d]) for the nd diagonals (offsets strictly increasing);
 * positions with i + offset[d] outside [0, n) and zero values are not
 * entries (the structural reading: a zero stored in DIA is padding).
 * Columns of a row come out increasing because the offsets are.  Pass
 * row_ptr only (col, out = NULL) to count; returns nnz, or -1 when the
 * offsets are not strictly increasing or cap is too small. */
int64_t orc_dia_to_csr(int64_t n, int64_t nd, const int32_t *offset, const double *val,
                       int32_t *row_ptr, int32_t *col, double *out, int64_t cap)
{
    for (int64_t d = 1; d < nd; d++)
        if (offset[d] <= offset[d - 1]) return -1;
    int64_t k = 0;
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        for (int64_t d = 0; d < nd; d++) {
            const int64_t j = i + offset[d];
            if (j < 0 || j >= n) continue;
            const double a = val[d * n + i];
            if (a == 0.0) continue;
            if (col) {
                if (k >= cap) return -1;
                col[k] = (int32_t)j;
                out[k] = a;
            }
            k++;
        }
        row_ptr[i + 1] = (int32_t)k;
    }
    return k;
}

void orc_stream_direct(int64_t N, const double *A, const double *B, double *C)
{
    for (int64_t i = 0; i < N; i++) C[i] += A[i] * B[i];
}

void orc_stream_indirect(int64_t N, const double *A, const double *B, const int32_t *I, double *C)
{
    for (int64_t i = 0; i < N; i++) C[i] += A[i] * B[I[i]];
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
