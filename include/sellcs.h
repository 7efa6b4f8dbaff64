/*
 * sellcs.h -- C ABI of the GB300 SELL-C-sigma augmented SpMMV library.
 *
 * The operation (GHOST, arxiv 1507.08101, Sec. "Kernel fusion"):
 *
 *     y = alpha (A - gamma I) x + beta y
 *
 * for a sparse A in SELL-C-sigma storage (Sec. "Sparse matrix storage") and
 * dense block vectors x, y (Sec. "Dense matrices", "Block vectors"), optionally
 * chained with the dot products <y,y>, <x,y>, <x,x> of every vector of the
 * block and with z = delta z + eta y, each augmentation enabled on its own,
 * all in one pass over the matrix.
 *
 * General conventions
 *  - Every function returns SP_OK (0) or a negative SP_ERR_* code; nothing
 *    aborts the process.  sp_error_string() names a code.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Compute calls are asynchronous on that stream.  Calls that return sizes to
 *    the host (create, export, info) synchronise the stream.
 *  - Device memory for matrices and library-owned block vectors is allocated
 *    by the library with cudaMalloc (which may synchronise the device; the
 *    create calls synchronise their stream anyway) and freed by the matching
 *    destroy, after that call has synchronised its stream.  Temporaries of the
 *    compute calls (partial sums, host-dot buffers) are stream-ordered
 *    (cudaMallocAsync / cudaFreeAsync on the call's stream).  Block vectors are either allocated by
 *    the library (sp_dense_create) or are views of caller memory
 *    (sp_dense_view), which the library never frees.
 *  - Block vectors (x, y, z) are always in the caller's original row order;
 *    the sigma permutation is internal to the matrix.
 *  - Integer data (row pointers int64, column indices int32, permutation and
 *    padding) are kept exact.  Matrices need nrows, ncols < 2^31 and at most
 *    2^31 - 1 nonzeros per row (local indices are 32-bit, Sec. "Sparse matrix
 *    storage", local vs global indices); stored entries are counted in int64.
 *  - Thread safety: distinct handles may be used from distinct host threads.
 *    Calls that use the same matrix handle must be ordered (same stream, or
 *    synchronised): they share the handle's scratch (the partial sums of the
 *    fused reductions and the counters of the dynamic row order that
 *    products on row-major blocks of more than 4 columns use).
 */
#ifndef SELLCS_H
#define SELLCS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SP_API __attribute__((visibility("default")))
#else
#define SP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ errors */
#define SP_OK 0
#define SP_ERR_ARG (-1)         /* null pointer, bad flag combination, aliasing */
#define SP_ERR_DIM (-2)         /* shapes of A, x, y, z disagree */
#define SP_ERR_DTYPE (-3)       /* unsupported value / vector precision pair */
#define SP_ERR_CUDA (-4)        /* a CUDA runtime call failed */
#define SP_ERR_OOM (-5)         /* device allocation failed */
#define SP_ERR_TIMEOUT (-6)     /* a bounded device-side wait gave up */
#define SP_ERR_FORMAT (-7)      /* CSR input invalid (row pointers, column range) */
#define SP_ERR_UNSUPPORTED (-8) /* valid request this build does not implement */

SP_API const char *sp_error_string(int code);
/* Text of the last CUDA failure seen by this thread (diagnostics only). */
SP_API const char *sp_last_error_detail(void);

/* ------------------------------------------------------------------ types */
typedef enum { SP_F64 = 0, SP_F32 = 1, SP_BF16 = 2 } sp_dtype;
typedef enum { SP_ROW_MAJOR = 0, SP_COL_MAJOR = 1 } sp_layout;

typedef struct sp_mat sp_mat;     /* opaque: SELL-C-sigma matrix on the device */
typedef struct sp_dense sp_dense; /* opaque: dense block vector (owning or view) */

/* ------------------------------------------------------------------ sparse matrix */

/* Flags of sp_mat_create_csr / sp_mat_update_values. */
#define SP_MAT_CSR_ON_DEVICE (1u << 0)  /* rowptr, col, val are device pointers (else host) */
#define SP_MAT_VAL_F32 (1u << 1)        /* val points to float (else double) */
#define SP_MAT_WITH_TRANSPOSE (1u << 2) /* also build A^T in SELL-C-sigma (needed by sp_spmv_adjoint) */
/* Work order of the product kernels over this matrix (and its transpose); at
 * most one of the two.  Neither: chosen per call, the moving front when the
 * block vector x is larger than half of L2, the contiguous ranges otherwise.
 * The order changes only which warp computes which row, never a result. */
#define SP_MAT_ORDER_FRONT (1u << 3)  /* moving front: all warps work on one run of rows at a time */
#define SP_MAT_ORDER_RANGES (1u << 4) /* each warp owns one contiguous cost-balanced range of rows */
/* Vectors in SELL row order (the local permutation of GHOST's sparse-matrix
 * section applied to rows and columns alike; nrows == ncols): the
 * column indices are stored as slots (col' = the slot of row col), so x, y
 * and z of every product are indexed by slot: row s of them is user row
 * perm[s] (sp_mat_permute moves block vectors between the two orders).  The
 * products read x and write y, z at consecutive rows of a chunk.  Not with
 * SP_MAT_WITH_TRANSPOSE.  sp_mat_export_sell returns the stored (slot)
 * indices; sp_mat_to_csr returns the user's CSR. */
#define SP_MAT_PERMUTED_SPACE (1u << 5)

/*
 * Build a SELL-C-sigma matrix from CSR (GHOST: "construct a SELL-C-sigma matrix
 * from raw CRS data, i.e., row pointers, column indices, and values").
 *   nrows, ncols   matrix shape (nrows >= 0, ncols >= 1 unless nrows == 0)
 *   rowptr         int64[nrows+1], rowptr[0] = 0, non-decreasing
 *   col            int32[nnz], each in [0, ncols); any order inside a row (the
 *                  stored order is the given order)
 *   val            double[nnz] (float[nnz] with SP_MAT_VAL_F32), rounded once
 *                  to val_dtype (f64 -> f32 round-to-nearest-even; -> bf16 via
 *                  f32, both round-to-nearest-even)
 *   C              chunk height, 1 <= C <= 1024
 *   sigma          sort window, >= 1 (rows are sorted by length, longest first,
 *                  stably, inside each window of sigma rows starting at row 0)
 * The inputs are copied; they may be freed when the call returns.  The call
 * validates the CSR on the device and returns SP_ERR_FORMAT for a malformed
 * input (nothing is left allocated).  Synchronises the stream.
 */
SP_API int sp_mat_create_csr(sp_mat **out, int64_t nrows, int64_t ncols, const int64_t *rowptr,
                      const int32_t *col, const void *val, int C, int64_t sigma, sp_dtype val_dtype,
                      unsigned flags, void *stream);

/*
 * Replace the values of A (and of its transpose, if built) keeping the pattern
 * (GHOST: "each subsequent matrix construction only needs to update the
 * matrix values").  val is in the CSR order given at creation: double[nnz], or
 * float[nnz] with SP_MAT_VAL_F32; host unless SP_MAT_CSR_ON_DEVICE.
 * Asynchronous for device input.
 */
SP_API int sp_mat_update_values(sp_mat *A, const void *val, unsigned flags, void *stream);

/* New handle sharing A's pattern (and transpose pattern) with A's values
 * converted to val_dtype (from A's stored values).  Asynchronous. */
SP_API int sp_mat_clone_values(sp_mat **out, const sp_mat *A, sp_dtype val_dtype, void *stream);

typedef struct {
    int64_t nrows, ncols, nnz;
    int64_t nchunks;  /* ceil(nrows / C) */
    int64_t nstored;  /* entries stored including padding: sum_c C * chunklen[c] */
    int32_t C;
    int32_t maxrowlen;
    int64_t sigma;
    sp_dtype val_dtype;
    int32_t has_transpose;
} sp_mat_info_t;

SP_API int sp_mat_info(const sp_mat *A, sp_mat_info_t *info);

/*
 * Copy the SELL-C-sigma arrays to host buffers sized from sp_mat_info (any
 * pointer may be NULL to skip it):
 *   chunkptr int64[nchunks+1]  offset of each chunk in col/val
 *   chunklen int32[nchunks]    padded row length of each chunk
 *   slotlen  int32[nchunks*C]  real length of the row in each slot (0 = padding row)
 *   perm     int32[nchunks*C]  original row of each slot (-1 = padding row)
 *   col      int32[nstored]    column of entry j of slot r of chunk c at chunkptr[c] + j*C + r
 *   val      double[nstored]   values widened to double (padding entries are 0)
 * Padding entries carry the column of the last real entry of their row (0 for
 * an empty or padding row).  Synchronises the stream.
 */
SP_API int sp_mat_export_sell(const sp_mat *A, int64_t *chunkptr, int32_t *chunklen, int32_t *slotlen,
                       int32_t *perm, int32_t *col, double *val, void *stream);

/* Same for the transpose built with SP_MAT_WITH_TRANSPOSE (SP_ERR_ARG if absent). */
SP_API int sp_mat_export_sell_transpose(const sp_mat *A, int64_t *chunkptr, int32_t *chunklen,
                                 int32_t *slotlen, int32_t *perm, int32_t *col, double *val,
                                 void *stream);

/* Rebuild CSR (original row order) on the host: rowptr int64[nrows+1], col int32[nnz],
 * val double[nnz].  Synchronises the stream. */
SP_API int sp_mat_to_csr(const sp_mat *A, int64_t *rowptr, int32_t *col, double *val, void *stream);

/* Synchronises the given stream, then frees the device arrays. */
SP_API int sp_mat_destroy(sp_mat *A, void *stream);

/* ------------------------------------------------------------------ dense block vectors */

/*
 * A dense nrows x ncols block vector (GHOST ghost_densemat).  Row-major =
 * interleaved vectors, element (i,k) at ptr[i*ld + k]; column-major: ptr[k*ld + i].
 * dtype SP_F64 or SP_F32.
 */
SP_API int sp_dense_create(sp_dense **out, int64_t nrows, int32_t ncols, sp_dtype dtype, sp_layout layout,
                    void *stream);
/* View of caller device memory (never freed by the library).  ld >= ncols
 * (row-major) or ld >= nrows (column-major). */
SP_API int sp_dense_view(sp_dense **out, void *dev_ptr, int64_t nrows, int32_t ncols, int64_t ld,
                  sp_dtype dtype, sp_layout layout);
/* Compact view of columns [col0, col0+ncols) of src (GHOST "compact view"). */
SP_API int sp_dense_view_cols(sp_dense **out, const sp_dense *src, int32_t col0, int32_t ncols);
/* Device pointer and shape of a block vector (any output may be NULL). */
SP_API int sp_dense_data(const sp_dense *d, void **ptr, int64_t *nrows, int32_t *ncols, int64_t *ld,
                  sp_dtype *dtype, sp_layout *layout);
/* Frees the memory only if d owns it. */
SP_API int sp_dense_destroy(sp_dense *d, void *stream);

/*
 * Scattered views and copies (Sec. "Dense matrices": a view may select a
 * subset of a block's columns with gaps between them; a compact clone of such
 * a view may be the better operand, and the storage layout can be changed
 * while a block vector is copied).
 *   sp_dense_view_scattered  view of the columns cols[0..ncols) (distinct,
 *       each in [0, src->ncols); any order) of src (compact or scattered; the
 *       view never owns memory).  SP_ERR_DIM for a column out of range,
 *       SP_ERR_ARG for a repeated one.  Host only.
 *   sp_dense_columns  writes the view's columns as columns of the block at its
 *       base pointer (int32[ncols], may be NULL); returns 1 for a scattered
 *       view, 0 for a compact one, <0 on error.  sp_dense_data returns that
 *       base pointer for a scattered view.
 *   sp_dense_clone    a new compact block (owned, nrows x ncols, `layout`)
 *       holding a copy of src (any view).  Asynchronous after the allocation.
 *   sp_dense_copy     dst = src for two views of equal shape and dtype, any
 *       layouts and view kinds; SP_ERR_ARG if they share elements other than
 *       as the identical view (then it is a no-op).  Asynchronous.
 * sp_spmv accepts scattered x, y and z: it copies them into compact
 * temporaries (stream-ordered allocations), runs the product, and copies y
 * and z back; scattered x and y of one block must not share a column.  The
 * other compute calls return SP_ERR_ARG for a scattered view (reason in
 * sp_last_error_detail).
 */
SP_API int sp_dense_view_scattered(sp_dense **out, const sp_dense *src, int32_t ncols, const int32_t *cols);
SP_API int sp_dense_columns(const sp_dense *d, int32_t *cols);
SP_API int sp_dense_clone(sp_dense **out, const sp_dense *src, sp_layout layout, void *stream);
SP_API int sp_dense_copy(sp_dense *dst, const sp_dense *src, void *stream);

/* ------------------------------------------------------------------ augmented SpMMV */

/* Augmentation flags (each enables one part; GHOST_SPMV_* in the paper). */
#define SP_SPMV_SCALE (1u << 0)  /* multiply by alpha (else alpha = 1) */
#define SP_SPMV_SHIFT (1u << 1)  /* subtract gamma[0] x (one shift for all vectors) */
#define SP_SPMV_VSHIFT (1u << 2) /* subtract gamma[k] x_k (one shift per vector) */
#define SP_SPMV_AXPBY (1u << 3)  /* add beta y_old (else y_old is not read) */
#define SP_SPMV_DOT_YY (1u << 4) /* dot[k]       = <y_k, y_k> (new y) */
#define SP_SPMV_DOT_XY (1u << 5) /* dot[w + k]   = <x_k, y_k> (new y) */
#define SP_SPMV_DOT_XX (1u << 6) /* dot[2w + k]  = <x_k, x_k> */
#define SP_SPMV_CHAIN_AXPBY (1u << 7) /* z = delta z + eta y (new y) */
#define SP_SPMV_DOT_HOST (1u << 8)    /* dot is a host pointer: the call synchronises */
#define SP_SPMV_DOT_ANY (SP_SPMV_DOT_YY | SP_SPMV_DOT_XY | SP_SPMV_DOT_XX)

#define SP_MAX_VSHIFT 1024 /* widest block with per-vector shifts */
/* With float32 vectors a lane adds its dot-product terms in float over at most
 * SP_DOT_RUN_F32 of its rows; those float sums then go through a float tree of
 * at most 5 additions across the lanes of a column and into float64, in which
 * every later stage adds.  So every term passes through at most
 * SP_DOT_RUN_F32 + 5 float additions. */
#define SP_DOT_RUN_F32 32

typedef struct {
    uint32_t flags;
    double alpha, beta, delta, eta;
    const double *gamma; /* host: 1 value (SHIFT) or ncols(x) values (VSHIFT) */
    sp_dense *z;         /* CHAIN_AXPBY target, same shape as y */
    double *dot;         /* 3*w doubles [yy | xy | xx]; only requested slots are written */
} sp_spmv_opts;

#define SP_SPMV_OPTS_INIT {0u, 1.0, 0.0, 0.0, 1.0, NULL, NULL, NULL}

/*
 * y = alpha (A - gamma I) x + beta y with the requested augmentations
 * (GHOST ghost_spmv(y, A, x, opts)).
 *   x   ncols(A) x w, y (and z) nrows(A) x w; same dtype; row- or column-major
 *   Precision pairs (values / vectors): f64/f64 (f64 accumulation);
 *   f32/f64, bf16/f64, f32/f32, bf16/f32 (f32 accumulation of the row sums;
 *   the epilogue runs in the vector precision).  Dot products are returned
 *   in double; they are accumulated in double for f64 vectors, and for f32
 *   vectors in float over short runs of rows (SP_DOT_RUN_F32), then double.
 *   SHIFT, VSHIFT, DOT_XY and DOT_XX need ncols(A) >= nrows(A); they use the
 *   first nrows rows of x as the rows' own entries (I is the leading
 *   nrows x nrows identity: a square A, or one process's rows with the columns
 *   of its halo appended, see sp_dist_spmv).  SHIFT and VSHIFT are
 *   exclusive.  x must not overlap y or z, and z must not overlap y
 *   (SP_ERR_ARG).  The reductions are deterministic (fixed order).
 */
SP_API int sp_spmv(sp_dense *y, const sp_mat *A, const sp_dense *x, const sp_spmv_opts *opts, void *stream);

/*
 * The augmented product fused with the inner products of a tall and skinny
 * block V with the new y (the dense-matrix section's X = V^T W, here with
 * W = y, formed while y is written; for block orthogonalisation after a
 * product, the step the paper's block solvers pair with the SpMMV):
 *     y = alpha (A - gamma I) x + beta y  [z = delta z + eta y],  C = V^T y
 *   y, x, z, opts  as sp_spmv, with SCALE, SHIFT, VSHIFT, AXPBY and
 *                  CHAIN_AXPBY (the fused dots are refused: SP_ERR_ARG);
 *                  float64 values and vectors, row-major, w <= 8, each row a
 *                  whole number of the kernel's lane vectors and aligned to
 *                  them (else SP_ERR_UNSUPPORTED), and the matrix's chunk
 *                  height at least 32 / (lanes per row) (rows are not split
 *                  over lanes here; else SP_ERR_UNSUPPORTED); not for
 *                  SP_MAT_PERMUTED_SPACE
 *   V              nrows x m, float64, row-major, 1 <= m <= 8; must not
 *                  overlap y or z
 *   C              device, m x w float64, row-major with leading dimension
 *                  ldc >= w, overwritten with V^T y (the new y)
 * The sums of C are deterministic (fixed lane tree, warps and blocks in
 * order).  Shares the matrix's reduction scratch with sp_spmv's dots: calls
 * on one matrix must be ordered.  Asynchronous.
 */
SP_API int sp_spmv_vty(sp_dense *y, const sp_mat *A, const sp_dense *x, const sp_spmv_opts *opts, const sp_dense *V,
                       double *C, int64_t ldc, void *stream);

/* ------------------------------------------------------------------ derivatives */

/*
 * Adjoint of y = A x for a row-major g = dL/dy (nrows x w):
 *   dx    = A^T g            (ncols x w; needs SP_MAT_WITH_TRANSPOSE; NULL to skip)
 *   dvals[p] = sum_k g[row(p),k] x[col(p),k] for every nonzero p, in the CSR
 *           order given at creation (device array of nnz elements in the
 *           precision of x and g; NULL to skip).
 * x, g and dx share one dtype (f64 or f32) and are row-major.  Asynchronous.
 */
SP_API int sp_spmv_adjoint(sp_dense *dx, void *dvals, const sp_mat *A, const sp_dense *x, const sp_dense *g,
                    void *stream);

/*
 * Block vector between the user's row order and the SELL row order of A:
 *   to_sell != 0:  out[s, :] = in[perm[s], :]   for s < nrows
 *   to_sell == 0:  out[perm[s], :] = in[s, :]
 * (perm = the row permutation of A; the identity when sigma = 1).  in and out:
 * nrows x w device blocks of the same dtype, row-major, not overlapping.
 * Asynchronous on the stream.
 */
SP_API int sp_mat_permute(const sp_mat *A, sp_dense *out, const sp_dense *in, int to_sell, void *stream);

/* ------------------------------------------------------------------ tall and skinny kernels */

/*
 * The tall and skinny block-vector kernels of the dense-matrix section of the
 * paper (ghost_tsmttsm, ghost_tsmm, ghost_tsmm_inplace), with V n x m,
 * W n x k (m, k <= 32 << n) and the small X m x k, all row-major device
 * blocks of one dtype (SP_F64 or SP_F32):
 *   sp_tsmttsm   X <- alpha V^T W + beta X   (kahan != 0: Kahan-compensated
 *                sums, the variant the paper adds for large n).  The result
 *                does not depend on timing (per-block sums added in block
 *                order).  beta = 0: X is not read.
 *   sp_tsmm      W <- alpha V X + beta W; W may be V itself (in place, then
 *                k = m); any other overlap of W with V or X is SP_ERR_ARG.
 *                beta = 0: W is not read.
 * Errors: SP_ERR_ARG for a missing or column-major block, m or k below 1;
 * SP_ERR_DIM for mismatched shapes; SP_ERR_DTYPE for mixed or unsupported
 * dtypes; SP_ERR_UNSUPPORTED for m or k above 32.  Precision: products and
 * per-thread sums in the blocks' dtype, the sums of threads and blocks in
 * float64 ((sum, compensation) pairs for the Kahan variant).  sp_tsmttsm
 * takes 16 * m * k bytes per thread block (a few hundred blocks) for its
 * block sums, stream-ordered from the device's default memory pool, and
 * gives it back on the stream.  Asynchronous on the stream.
 */
SP_API int sp_tsmttsm(sp_dense *X, const sp_dense *V, const sp_dense *W, double alpha, double beta, int kahan,
                      void *stream);
SP_API int sp_tsmm(sp_dense *W, const sp_dense *V, const sp_dense *X, double alpha, double beta, void *stream);

/* ------------------------------------------------------------------ KPM moments */

/*
 * Chebyshev moments of the kernel polynomial method, the solver Sec. "Kernel
 * fusion" names as the user of the fused product: with A~ = (A - b I) / a,
 *     mu[k * w + c] = < x_c, T_k(A~) x_c >,   k = 0 .. nmom-1, c = 0 .. w-1.
 * Each Chebyshev step w_{n+1} = 2 A~ w_n - w_{n-1} is one sp_spmv (SCALE,
 * SHIFT, AXPBY with beta = -1) whose fused <y,y> and <x,y> give two moments
 * (mu_{2n} = 2 <w_n,w_n> - mu_0, mu_{2n+1} = 2 <w_{n+1},w_n> - mu_1), so
 * about nmom / 2 products.
 *   A      square matrix
 *   x      start block, nrows x w, row-major, device (read only)
 *   nmom   number of moments, >= 1
 *   a, b   scaling (a != 0, both finite); the spectrum of A should map into
 *          [-1, 1] for the moments to stay bounded
 *   mu     host array of nmom * w doubles, written
 * Allocates two nrows x w work blocks for the call; synchronises the stream.
 */
SP_API int sp_kpm_moments(const sp_mat *A, const sp_dense *x, int32_t nmom, double a, double b, double *mu,
                          void *stream);

/* ------------------------------------------------------------------ host block vectors */

/*
 * Pipelined products over block vectors in HOST memory (no counterpart in the
 * paper: the end-to-end form of sp_spmv for callers whose vectors live on the
 * host).  A plan owns three sets of device buffers for x, y, z and the dots
 * and three streams (copy-in, product, copy-out); call k uses set k mod 3, so
 * the copy-in of call k+1 and the copy-out of call k-1 overlap the product of
 * call k.  The product is sp_spmv's, with the same results.
 *   sp_host_plan_create   A: the matrix (not owned; it must outlive the plan);
 *                         w >= 1 block width; vec_dtype SP_F64 or SP_F32 (SP_F64
 *                         when A holds float64 values).  Allocates
 *                         3 * (ncols + 2 nrows) * w elements of device memory and
 *                         synchronises the device.
 *   sp_spmv_host          x: ncols x w, row-major, read; y_in: nrows x w, read when
 *                         opts has SP_SPMV_AXPBY (else may be NULL); y_out: nrows x w,
 *                         written; z_in / z_out: read / written with
 *                         SP_SPMV_CHAIN_AXPBY (opts->z is ignored); dot: 3 w host
 *                         doubles, the requested slots written (opts->dot is ignored).
 *                         Every pointer is host memory; page-locked memory gives
 *                         the overlap (pageable memory works but serialises).  The
 *                         call only enqueues: the caller must not touch any of the
 *                         buffers until sp_host_plan_sync returns, and a call whose
 *                         y_in (z_in) is an earlier call's y_out (z_out) needs a
 *                         sync in between.  Errors of the enqueued work surface at
 *                         sp_host_plan_sync.
 *   sp_host_plan_sync     waits for every enqueued call.
 *   sp_host_plan_destroy  waits, then frees the plan.
 */
typedef struct sp_host_plan sp_host_plan;
SP_API int sp_host_plan_create(sp_host_plan **out, const sp_mat *A, int32_t w, sp_dtype vec_dtype);
SP_API int sp_spmv_host(sp_host_plan *p, const void *x, const void *y_in, void *y_out, const void *z_in,
                        void *z_out, double *dot, const sp_spmv_opts *opts);
SP_API int sp_host_plan_sync(sp_host_plan *p);
SP_API int sp_host_plan_destroy(sp_host_plan *p);

/* ------------------------------------------------------------------ batched SpMMV */

/*
 * Many matrices of uneven size and block width in ONE persistent launch (no
 * counterpart in the paper beyond its block vectors; Sec. "Block vectors").
 * Each matrix's rows are cut into cost-balanced units that the resident warps
 * own statically, so the per-matrix dot products are deterministic.
 *   A[m]            matrices (all with the same value precision; not owned,
 *                   must outlive the batch)
 *   widths[m]       block width of matrix m, 1..SP_BATCH_MAX_W
 *   cols_per_lane   per matrix, the columns each lane owns (1,2,4,8; must
 *                   divide widths[m]); NULL or 0 entries: chosen automatically
 *   vec_dtype       SP_F64 (f64 values) or SP_F32 (f32 values: f32 or f64 vectors)
 * Synchronises the stream.
 */
#define SP_BATCH_MAX_W 8
typedef struct sp_batch sp_batch;
SP_API int sp_batch_create(sp_batch **out, int count, sp_mat *const *A, const int32_t *widths,
                           const int32_t *cols_per_lane, sp_dtype vec_dtype, void *stream);
/* Bind the block vectors: x[m] (ncols x w, row-major, ld = w), y[m] (nrows x w),
 * y0[m] the beta source (NULL or NULL entries: y itself).  Device pointers,
 * 16-byte aligned.  Synchronises the stream. */
SP_API int sp_batch_bind(sp_batch *b, const void *const *x, void *const *y, const void *const *y0,
                         void *stream);
/* y_m = alpha A_m x_m + beta y0_m for every m in one launch.  flags: any of
 * SP_SPMV_SCALE, SP_SPMV_AXPBY, SP_SPMV_DOT_YY/XY/XX; dots (device) receives
 * for matrix m at dots[m*3*SP_BATCH_MAX_W + q*SP_BATCH_MAX_W + k] the sums
 * q = 0: <y,y>, 1: <x,y>, 2: <x,x> of column k (a second small launch).
 * Asynchronous; graph-capturable once bound. */
SP_API int sp_batch_spmv(sp_batch *b, uint32_t flags, double alpha, double beta, double *dots, void *stream);
/* Units, grid and the lane layout chosen per matrix (host outputs, any may be NULL). */
SP_API int sp_batch_info(const sp_batch *b, int32_t *nunits, int32_t *grid, int32_t *cols_per_lane);
SP_API int sp_batch_destroy(sp_batch *b, void *stream);

/* ------------------------------------------------------------------ mixed-precision CG */

/*
 * Batched CG with iterative refinement for SPD matrices: per column the
 * float64 residual r = b - A x (batched float64 product), a float32 CG solve
 * of A d = r / ||r|| to relative reduction inner_tol (Chronopoulos-Gear form:
 * one batched product with fused <r,r>, <r,Ar> and one vector update per
 * iteration, graph_iters iterations per CUDA-graph replay), and the float64
 * update x += ||r|| d, until ||b - A x||_2 <= tol ||b||_2 for every column.
 * inner_f64 = 1 runs the inner solve in float64 (plain CG reference).
 */
typedef struct {
    double tol;
    double inner_tol;
    int32_t max_outer;
    int32_t max_inner;
    int32_t graph_iters;
    int32_t inner_f64;
} sp_cg_opts;
#define SP_CG_OPTS_INIT {1e-10, 1e-4, 40, 20000, 16, 0}
typedef struct {
    int32_t outer;          /* refinement steps taken */
    int32_t inner;          /* inner iterations summed over refinement steps (slowest column) */
    int32_t graph_launches; /* CUDA graph replays */
    int32_t converged;      /* 1 if every column met tol */
    double max_rel_residual;
} sp_cg_stats;
typedef struct sp_cg sp_cg;
/* A[m]: float64 square SPD matrices (not owned; a float32 copy is made),
 * widths[m] in 1..SP_BATCH_MAX_W, cpl64/cpl32: lane layouts (NULL = auto). */
SP_API int sp_cg_create(sp_cg **out, int count, sp_mat *const *A, const int32_t *widths, const int32_t *cpl64,
                        const int32_t *cpl32, void *stream);
/* b[m], x[m]: device float64 row-major n_m x w_m.  rel_res (host, sum of
 * widths, may be NULL) receives the final relative residual of each column.
 * Synchronous. */
SP_API int sp_cg_solve(sp_cg *cg, const double *const *b, double *const *x, const sp_cg_opts *opts,
                       sp_cg_stats *stats, double *rel_res, void *stream);
SP_API int sp_cg_destroy(sp_cg *cg, void *stream);

/* ------------------------------------------------------------------ row-partitioned product */

/*
 * The matrix distributed row-wise over processes (GHOST, Sec. "Data
 * parallelism": the system matrix is split row-wise, the work of a process
 * counted in rows or in nonzeros; Sec. "Heterogeneous execution": a share per
 * process, e.g. its device's memory bandwidth, and the figure of the row-wise
 * distribution: (1) weights, (2) one partial matrix per process, (3) the
 * remote column indices compressed).  Only the host-side plan and two device
 * calls live here; the exchange of the halo and the sum of the dot products
 * over processes are the caller's (a collective library, or copies).
 *
 * sp_dist_partition: contiguous row blocks.  bounds (int64[nparts + 1],
 * written) with bounds[0] = 0, bounds[nparts] = nrows, non-decreasing; part p
 * owns rows [bounds[p], bounds[p+1]).  The work of rows [0, r) is r, or
 * rowptr[r] when by_nnz (then rowptr is int64[nrows + 1] of the global CSR);
 * each inner boundary is the row boundary nearest to the point where the work
 * reaches the part's cumulative share (share: nparts finite weights >= 0, at
 * least one positive; NULL = equal).  Host only.  SP_ERR_FORMAT for
 * decreasing row pointers.
 */
SP_API int sp_dist_partition(int64_t nrows, const int64_t *rowptr, int nparts, const double *share, int by_nnz,
                             int64_t *bounds);

/*
 * sp_dist_plan_create: the plan of process `rank` for its rows.
 *   nglobal         global rows = global columns (square matrix)
 *   nranks, bounds  the partition (int64[nranks + 1], as sp_dist_partition writes)
 *   rowptr          int64[nloc + 1], rowptr[0] = 0: this process's rows only,
 *                   nloc = bounds[rank+1] - bounds[rank]
 *   gcol            int64[rowptr[nloc]] their GLOBAL column indices
 * Column compression (step 3 of the figure): a column c owned by this
 * process gets the local index c - bounds[rank]; the distinct remote columns,
 * in ascending global order, get nloc, nloc + 1, ... ("the halo"), so the halo
 * entries of one owner are contiguous and owners come in rank order.  Local
 * indices are 32-bit (Sec. "Sparse matrix storage", local vs global indices):
 * nloc + nhalo < 2^31 or SP_ERR_DIM.  Inputs are copied.  Host only.
 * SP_ERR_FORMAT for bad row pointers or columns outside [0, nglobal).
 *
 * sp_dist_plan_info: nloc, nhalo, nonzeros in owned / remote columns, and the
 *   rows this process sends (-1 before sp_dist_plan_set_sends).  Any output may
 *   be NULL.
 * sp_dist_plan_halo: halo_gidx (int64[nhalo]) the global row of each halo
 *   entry; recv_counts (int64[nranks]) how many of them each rank owns (0 for
 *   this rank).  Either may be NULL.
 * sp_dist_plan_columns: col_ext (int32[nnz]) every entry's local column in
 *   [0, nloc + nhalo), in the CSR order of the input: with the caller's
 *   rowptr and values, the nloc x (nloc + nhalo) matrix of the "no overlap"
 *   form (one product over x extended by its halo).
 * sp_dist_plan_split: the same entries split into the local part (rowptr_loc
 *   int64[nloc+1], col_loc int32, val_loc double: columns < nloc) and the
 *   remote part (rowptr_rem, col_rem, val_rem: columns nloc..nloc+nhalo-1),
 *   each row keeping its order; val is the double[nnz] of the input rows.
 *   Arrays are caller-owned host memory sized by sp_dist_plan_info.
 * sp_dist_plan_set_sends: what this process sends: send_counts (int64[nranks],
 *   0 for itself) rows to each rank, send_gidx the global rows, rank after
 *   rank, each list strictly ascending and owned by this process -- exactly
 *   the halo_gidx of the receiving rank restricted to this process's rows (the
 *   caller exchanges those lists once, e.g. with an all-to-all).  Host only;
 *   SP_ERR_ARG with the reason in sp_last_error_detail for a bad list.
 * sp_dist_plan_sends: the stored send counts (int64[nranks]) and local rows
 *   (int32[nsend]); either may be NULL.  SP_ERR_ARG before set_sends.
 * sp_dist_plan_destroy: frees the plan (and its device copy of the send list,
 *   after synchronising that device).
 */
typedef struct sp_dist_plan sp_dist_plan;
SP_API int sp_dist_plan_create(sp_dist_plan **out, int64_t nglobal, int nranks, const int64_t *bounds, int rank,
                               const int64_t *rowptr, const int64_t *gcol);
SP_API int sp_dist_plan_info(const sp_dist_plan *p, int64_t *nloc, int64_t *nhalo, int64_t *nnz_local,
                             int64_t *nnz_remote, int64_t *nsend);
SP_API int sp_dist_plan_halo(const sp_dist_plan *p, int64_t *halo_gidx, int64_t *recv_counts);
SP_API int sp_dist_plan_columns(const sp_dist_plan *p, int32_t *col_ext);
SP_API int sp_dist_plan_split(const sp_dist_plan *p, const double *val, int64_t *rowptr_loc, int32_t *col_loc,
                              double *val_loc, int64_t *rowptr_rem, int32_t *col_rem, double *val_rem);
SP_API int sp_dist_plan_set_sends(sp_dist_plan *p, const int64_t *send_counts, const int64_t *send_gidx);
SP_API int sp_dist_plan_sends(const sp_dist_plan *p, int64_t *send_counts, int32_t *send_local);
SP_API int sp_dist_plan_destroy(sp_dist_plan *p);

/*
 * sp_dist_pack: gathers the rows this process sends into send_buf (device,
 * nsend x w row-major, contiguous, rank after rank as set_sends ordered them)
 * from x (its first nloc rows; any layout; SP_F64 or SP_F32).  Asynchronous
 * on `stream`, except the first call on a plan, which copies the send list to
 * the device (cudaMalloc) and synchronises the stream.
 *
 * sp_dist_split_opts: the two passes of the overlapped product (host only):
 * pass 1 = the request without dots, chain and DOT_HOST (y = alpha (A_loc x -
 * gamma x) + beta y); pass 2 = y = alpha A_rem x + y (SCALE as requested,
 * AXPBY with beta = 1) with the requested dots, chain and DOT_HOST.
 *
 * sp_dist_spmv: the overlapped product (task mode of Sec. "Resource
 * management": the local part computed while the halo is in flight).
 *   A_loc  nloc x nloc (the split's local part), A_rem nloc x (nloc + nhalo)
 *   x      (nloc + nhalo) x w, row-major: rows 0..nloc-1 this process's x,
 *          rows nloc.. the halo (received in halo_gidx order)
 *   y, z   nloc x w; opts as sp_spmv
 *   halo_ready  a cudaEvent_t recorded once the halo rows of x are written,
 *          or NULL if they already are
 * Pass 1 is enqueued on `stream` at once; the stream then waits for
 * halo_ready and runs pass 2.  The dots are this process's partial sums:
 * their sum over processes (3 w doubles) is the product's.  Shift and dots
 * use x's first nloc rows.  y is read and written twice (the overlapped form
 * stores the result twice, as the paper notes).
 */
SP_API int sp_dist_pack(sp_dist_plan *p, const sp_dense *x, void *send_buf, void *stream);
SP_API int sp_dist_split_opts(const sp_spmv_opts *in, sp_spmv_opts *pass1, sp_spmv_opts *pass2);
SP_API int sp_dist_spmv(sp_dense *y, const sp_mat *A_loc, const sp_mat *A_rem, const sp_dense *x,
                        const sp_spmv_opts *opts, void *halo_ready, void *stream);

/* ------------------------------------------------------------------ no-allocation variant */

/*
 * sp_spmv_noalloc -- the augmented product of sp_spmv for callers that cannot
 * allocate device memory: for instance a process whose GPU memory is already
 * held by another allocator (a framework's caching pool), or a code path where
 * cudaMalloc and cudaFree are not allowed because they synchronise the device.
 * The paper has no counterpart of this entry point.
 *
 * It allocates nothing, on the device or the host.  Every input and output is
 * a plain device pointer owned by the caller:
 *   val, col, chunkptr, slotlen, perm  the SELL-C-sigma arrays in the layout
 *       sp_mat_export_sell describes (perm NULL: identity, i.e. sigma = 1);
 *       val in val_dtype
 *   nrows, ncols, C        matrix shape and chunk height (1..1024)
 *   x (ncols x w), y (nrows x w), z (nrows x w, or NULL without the chain):
 *       row-major with leading dimensions ldx, ldy, ldz, in vec_dtype
 *   w                      block width, 0..SP_NOALLOC_MAX_W
 *   flags, alpha, beta, gamma (host: 1 or w values), delta, eta, dot (device,
 *       3*w doubles): as in sp_spmv (SP_SPMV_DOT_HOST is rejected)
 * The scratch of the fused dot products is a static device array of
 * 3 * SP_NOALLOC_MAX_W * SP_NOALLOC_MAX_BLOCKS doubles (1.5 MiB) plus a ticket,
 * held by every GPU that loads this library until the process exits.  A block
 * width above SP_NOALLOC_MAX_W is rejected (SP_ERR_UNSUPPORTED, with the reason
 * in sp_last_error_detail).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Every call clears the ticket and
 * shares the array, so calls that overlap on the GPU (different streams, no
 * ordering) race and must not be issued.  Asynchronous on `stream`.
 * Speed: the call has no chunk lengths and no precomputed work partition, so
 * it runs the per-lane row loop over a block-strided assignment of rows to
 * warps.  On matrices whose row lengths vary widely (sorted windows, power-law
 * rows) that is slower than sp_spmv on a matrix handle, which balances the
 * warps' work and steps float64 chunks in lockstep.
 */
#define SP_NOALLOC_MAX_W 32
#define SP_NOALLOC_MAX_BLOCKS 2048
SP_API int sp_spmv_noalloc(const void *val, sp_dtype val_dtype, const int32_t *col, const int64_t *chunkptr,
                           const int32_t *slotlen, const int32_t *perm, int64_t nrows, int64_t ncols, int32_t C,
                           const void *x, int64_t ldx, void *y, int64_t ldy, void *z, int64_t ldz, int32_t w,
                           sp_dtype vec_dtype, uint32_t flags, double alpha, double beta, const double *gamma,
                           double delta, double eta, double *dot, void *stream);

/* ------------------------------------------------------------------ device info */
/* Streaming multiprocessor count of the current device (for grid sizing tests). */
SP_API int sp_device_sm_count(int *count);
/* Float64 fused multiply-add rate of the current device, measured (no
 * counterpart in the paper; the float64 products here are bound by that rate on
 * GB300, so their roofline needs the measured figure): every SM runs 2048
 * threads of 16 independent chains a <- fma(a, b, c) for 8192 steps; the best of
 * three timed launches (CUDA events, after one warm-up launch) gives
 * *tflops = 2 x fused multiply-adds / time in TFLOP/s and *ms its duration
 * (ms may be NULL).  Synchronises the stream; allocates 8 bytes
 * stream-ordered. */
SP_API int sp_device_fp64_rate(double *tflops, double *ms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SELLCS_H */
