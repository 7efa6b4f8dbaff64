/*
 * Oracle for the SELL-C-sigma augmented SpMMV -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded C in double precision.  It exists to check the
 * CUDA library; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may call it.  It shares no code, header or table with the CUDA
 * path.
 *
 * What it follows (GHOST, arxiv 1507.08101):
 *  - SELL-C-sigma layout (Sec. "Sparse matrix storage"): rows cut into chunks
 *    of C rows; each chunk padded with trailing zeros to the length of its
 *    longest row and stored column by column; before chunk assembly the rows of
 *    each window of sigma consecutive rows are sorted by their nonzero count.
 *  - Augmented product (Sec. "Kernel fusion"):
 *        y = alpha (A - gamma I) x + beta y,
 *    optionally chained with <y,y>, <x,y>, <x,x> and z = delta z + eta y, each
 *    part enabled on its own; gamma may differ per vector of the block.
 *  - Transposed product and the sampled product over the pattern (the
 *    derivatives of y = A x with respect to x and to the stored values).
 *
 * Readings where the paper is silent:
 *  - the sort is by row length DESCENDING and STABLE (ties keep the original
 *    row order); windows start at row 0, the last one may be short;
 *  - only rows are permuted: column indices and x, y, z stay in the caller's
 *    row order;
 *  - a padded entry stores value 0 and the column of the last real entry of
 *    its row (column 0 for an empty row or a padding row); a padding row (the
 *    tail of the last chunk) has length 0 and permutation entry -1;
 *  - the dot products and z use the NEW y;
 *  - with more columns than rows, the shift and the x-dots take x's first
 *    N rows (I is the leading N x N identity).
 *
 * Sums (row sums and dot products) use Neumaier's compensated summation so the
 * oracle's own rounding error is far below that of the kernels it checks.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ summation */

typedef struct {
    double s, c;
} nsum; /* Neumaier running sum */

static void nsum_add(nsum *a, double t) {
    double u = a->s + t;
    if (fabs(a->s) >= fabs(t))
        a->c += (a->s - u) + t;
    else
        a->c += (t - u) + a->s;
    a->s = u;
}

static double nsum_get(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------ SELL-C-sigma structure */

typedef struct {
    int64_t len;
    int64_t row;
} lenrow;

/* longer rows first; equal lengths keep the original row order (stable) */
static int cmp_lenrow(const void *pa, const void *pb) {
    const lenrow *a = (const lenrow *)pa, *b = (const lenrow *)pb;
    if (a->len != b->len) return a->len > b->len ? -1 : 1;
    return a->row < b->row ? -1 : (a->row > b->row ? 1 : 0);
}

/*
 * Row permutation, per-slot row lengths, chunk lengths and chunk offsets.
 * perm has nch*C entries (slot -> original row, -1 for padding rows),
 * slotlen has nch*C entries, chunklen nch, chunkptr nch+1 (offsets of each
 * chunk in the value/column arrays).  Returns the number of stored entries.
 */
int64_t orc_sell_structure(int64_t N, const int64_t *rowptr, int C, int64_t sigma,
                           int32_t *perm, int32_t *slotlen, int32_t *chunklen, int64_t *chunkptr) {
    int64_t nch = (N + C - 1) / C;
    int64_t nslots = nch * C;
    lenrow *buf = (lenrow *)malloc(sizeof(lenrow) * (size_t)(sigma < N ? sigma : (N > 0 ? N : 1)));
    for (int64_t w0 = 0; w0 < N; w0 += sigma) {
        int64_t w1 = w0 + sigma < N ? w0 + sigma : N;
        for (int64_t i = w0; i < w1; ++i) {
            buf[i - w0].len = rowptr[i + 1] - rowptr[i];
            buf[i - w0].row = i;
        }
        qsort(buf, (size_t)(w1 - w0), sizeof(lenrow), cmp_lenrow);
        for (int64_t i = w0; i < w1; ++i) perm[i] = (int32_t)buf[i - w0].row;
    }
    free(buf);
    for (int64_t s = N; s < nslots; ++s) perm[s] = -1;
    for (int64_t s = 0; s < nslots; ++s)
        slotlen[s] = perm[s] < 0 ? 0 : (int32_t)(rowptr[perm[s] + 1] - rowptr[perm[s]]);
    chunkptr[0] = 0;
    for (int64_t c = 0; c < nch; ++c) {
        int32_t m = 0;
        for (int r = 0; r < C; ++r)
            if (slotlen[c * C + r] > m) m = slotlen[c * C + r];
        chunklen[c] = m;
        chunkptr[c + 1] = chunkptr[c] + (int64_t)C * m;
    }
    return chunkptr[nch];
}

/* Fill the chunk-column-major SELL arrays: entry j of the row in slot r of
 * chunk c sits at chunkptr[c] + j*C + r. */
void orc_sell_fill(int64_t N, const int64_t *rowptr, const int32_t *col, const double *val, int C,
                   const int32_t *perm, const int32_t *chunklen, const int64_t *chunkptr,
                   int32_t *col_sell, double *val_sell) {
    int64_t nch = (N + C - 1) / C;
    for (int64_t c = 0; c < nch; ++c) {
        for (int r = 0; r < C; ++r) {
            int64_t s = c * C + r;
            int64_t i = perm[s];
            int64_t len = i < 0 ? 0 : rowptr[i + 1] - rowptr[i];
            int32_t padcol = len > 0 ? col[rowptr[i] + len - 1] : 0;
            for (int64_t j = 0; j < chunklen[c]; ++j) {
                int64_t pos = chunkptr[c] + j * C + r;
                if (j < len) {
                    col_sell[pos] = col[rowptr[i] + j];
                    val_sell[pos] = val[rowptr[i] + j];
                } else {
                    col_sell[pos] = padcol;
                    val_sell[pos] = 0.0;
                }
            }
        }
    }
}

/* Inverse of the two functions above: rebuild CSR in the original row order. */
void orc_sell_to_csr(int64_t N, int C, const int32_t *perm, const int32_t *slotlen,
                     const int64_t *chunkptr, const int32_t *col_sell, const double *val_sell,
                     int64_t *rowptr, int32_t *col, double *val) {
    int64_t nch = (N + C - 1) / C;
    int64_t *len = (int64_t *)calloc((size_t)(N > 0 ? N : 1), sizeof(int64_t));
    for (int64_t s = 0; s < nch * C; ++s)
        if (perm[s] >= 0) len[perm[s]] = slotlen[s];
    rowptr[0] = 0;
    for (int64_t i = 0; i < N; ++i) rowptr[i + 1] = rowptr[i] + len[i];
    for (int64_t s = 0; s < nch * C; ++s) {
        if (perm[s] < 0) continue;
        int64_t c = s / C, r = s % C, i = perm[s];
        for (int64_t j = 0; j < slotlen[s]; ++j) {
            col[rowptr[i] + j] = col_sell[chunkptr[c] + j * C + r];
            val[rowptr[i] + j] = val_sell[chunkptr[c] + j * C + r];
        }
    }
    free(len);
}

/* ------------------------------------------------------------------ augmented SpMMV (CSR) */

/*
 * y = alpha (A - diag(gamma) applied per column) x + beta y0, then the dot
 * products of the new y and z = delta z0 + eta y.  Block vectors are row-major
 * N x w with leading dimensions ldx, ldy, ldz.  Flags off mean alpha = 1,
 * gamma = 0, beta = 0 (y0 not read), no dots, z untouched.
 * dot receives [ <y,y>_0..w-1 | <x,y>_0..w-1 | <x,x>_0..w-1 ]; a slot whose
 * dot is not requested is left as it was.
 */
void orc_spmmv(int64_t N, int64_t ncols, const int64_t *rowptr, const int32_t *col, const double *val,
               int w, const double *x, int64_t ldx, double *y, int64_t ldy, const double *y0, int64_t ldy0,
               int do_scale, double alpha, int do_shift, const double *gamma, int do_axpby, double beta,
               int dot_yy, int dot_xy, int dot_xx, double *dot, int do_chain, double delta, double eta,
               double *z, int64_t ldz) {
    (void)ncols;
    nsum *dyy = (nsum *)calloc((size_t)w, sizeof(nsum));
    nsum *dxy = (nsum *)calloc((size_t)w, sizeof(nsum));
    nsum *dxx = (nsum *)calloc((size_t)w, sizeof(nsum));
    double a = do_scale ? alpha : 1.0;
    for (int64_t i = 0; i < N; ++i) {
        for (int k = 0; k < w; ++k) {
            nsum t = {0.0, 0.0};
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) nsum_add(&t, val[p] * x[col[p] * ldx + k]);
            double r = nsum_get(&t);
            /* row i of x is column i of A: the identity of the shift is the
             * leading N x N block (ncols >= N: a square A, or one process's
             * rows with the columns of its halo appended) */
            double xi = x[i * ldx + k];
            if (do_shift) r = r - gamma[k] * xi;
            r = a * r;
            if (do_axpby) r = r + beta * y0[i * ldy0 + k];
            y[i * ldy + k] = r;
            if (dot_yy) nsum_add(&dyy[k], r * r);
            if (dot_xy) nsum_add(&dxy[k], xi * r);
            if (dot_xx) nsum_add(&dxx[k], xi * xi);
            if (do_chain) z[i * ldz + k] = delta * z[i * ldz + k] + eta * r;
        }
    }
    for (int k = 0; k < w; ++k) {
        if (dot_yy) dot[k] = nsum_get(&dyy[k]);
        if (dot_xy) dot[w + k] = nsum_get(&dxy[k]);
        if (dot_xx) dot[2 * w + k] = nsum_get(&dxx[k]);
    }
    free(dyy);
    free(dxy);
    free(dxx);
}

/* The same product with the rows shared among OpenMP threads (a timing
 * baseline over all host cores; the tests pin orc_spmmv, and check that this
 * one gives the same y and z and dots equal to rounding).  Each thread keeps
 * its own compensated dot sums over a contiguous block of rows; the blocks'
 * sums are added in block order.  Without -fopenmp it runs on one thread. */
void orc_spmmv_omp(int64_t N, const int64_t *rowptr, const int32_t *col, const double *val, int w,
                   const double *x, int64_t ldx, double *y, int64_t ldy, const double *y0, int64_t ldy0,
                   int do_scale, double alpha, int do_shift, const double *gamma, int do_axpby, double beta,
                   int dot_yy, int dot_xy, int dot_xx, double *dot, int do_chain, double delta, double eta,
                   double *z, int64_t ldz, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    nsum *part = (nsum *)calloc((size_t)nthreads * 3 * (size_t)w, sizeof(nsum));
    const double a = do_scale ? alpha : 1.0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int tid = 0, nt = 1;
#ifdef _OPENMP
        tid = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        const int64_t i0 = N * tid / nt, i1 = N * (tid + 1) / nt;
        nsum *dyy = part + (size_t)tid * 3 * w, *dxy = dyy + w, *dxx = dxy + w;
        for (int64_t i = i0; i < i1; ++i) {
            for (int k = 0; k < w; ++k) {
                nsum t = {0.0, 0.0};
                for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) nsum_add(&t, val[p] * x[col[p] * ldx + k]);
                double r = nsum_get(&t);
                double xi = x[i * ldx + k];
                if (do_shift) r = r - gamma[k] * xi;
                r = a * r;
                if (do_axpby) r = r + beta * y0[i * ldy0 + k];
                y[i * ldy + k] = r;
                if (dot_yy) nsum_add(&dyy[k], r * r);
                if (dot_xy) nsum_add(&dxy[k], xi * r);
                if (dot_xx) nsum_add(&dxx[k], xi * xi);
                if (do_chain) z[i * ldz + k] = delta * z[i * ldz + k] + eta * r;
            }
        }
    }
    for (int k = 0; k < w; ++k) {
        nsum s[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        for (int t = 0; t < nthreads; ++t)
            for (int q = 0; q < 3; ++q) {
                const nsum *v = part + (size_t)t * 3 * w + (size_t)q * w + k;
                nsum_add(&s[q], v->s);
                nsum_add(&s[q], v->c);
            }
        if (dot_yy) dot[k] = nsum_get(&s[0]);
        if (dot_xy) dot[w + k] = nsum_get(&s[1]);
        if (dot_xx) dot[2 * w + k] = nsum_get(&s[2]);
    }
    free(part);
}

/* |A| |x| + |alpha gamma| |x| + |beta| |y0| per entry: the scale against
 * which a rounding error of the augmented product is measured. */
void orc_spmmv_scale(int64_t N, const int64_t *rowptr, const int32_t *col, const double *val, int w,
                     const double *x, int64_t ldx, const double *y0, int64_t ldy0, double alpha,
                     const double *gamma, double beta, int use_y0, double *s, int64_t lds) {
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < w; ++k) {
            double t = 0.0;
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) t += fabs(val[p] * x[col[p] * ldx + k]);
            double v = fabs(alpha) * t + fabs(alpha * gamma[k]) * fabs(x[i * ldx + k]);
            if (use_y0) v += fabs(beta) * fabs(y0[i * ldy0 + k]);
            s[i * lds + k] = v;
        }
}

/* ------------------------------------------------------------------ derivatives of y = A x */

/* dx = A^T g : dx[col(p), k] = sum over nonzeros p of val[p] * g[row(p), k].
 * dx is ncols x w row-major (ld = w).  Terms are added in CSR order. */
void orc_spmmv_transpose(int64_t N, int64_t ncols, const int64_t *rowptr, const int32_t *col,
                         const double *val, int w, const double *g, double *dx) {
    nsum *acc = (nsum *)calloc((size_t)(ncols * w > 0 ? ncols * w : 1), sizeof(nsum));
    for (int64_t i = 0; i < N; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            for (int k = 0; k < w; ++k) nsum_add(&acc[(int64_t)col[p] * w + k], val[p] * g[i * w + k]);
    for (int64_t q = 0; q < ncols * w; ++q) dx[q] = nsum_get(&acc[q]);
    free(acc);
}

/* dvals[p] = sum_k g[row(p), k] * x[col(p), k] for every stored nonzero p (CSR order). */
void orc_sampled_product(int64_t N, const int64_t *rowptr, const int32_t *col, int w, const double *g,
                         const double *x, double *dvals) {
    for (int64_t i = 0; i < N; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            nsum t = {0.0, 0.0};
            for (int k = 0; k < w; ++k) nsum_add(&t, g[i * w + k] * x[(int64_t)col[p] * w + k]);
            dvals[p] = nsum_get(&t);
        }
}
