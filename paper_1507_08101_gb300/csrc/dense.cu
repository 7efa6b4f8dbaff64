// Dense block vectors beyond the compact views (GHOST, Sec. "Dense
// matrices"): scattered views (a subset of the columns of a block, with gaps
// in the leading dimension), compact clones of any view in either storage
// layout (the paper: a compact clone of a scattered view may be the better
// operand, and the layout can be changed while copying), and copies between
// views of equal shape.  sp_spmv on scattered views works on compact clones
// and copies the results back (spmv_scattered).
#include <algorithm>
#include <set>
#include <vector>

#include "common.cuh"

namespace sp {

constexpr int kCopyCols = 64;  // columns per copy launch (the column maps travel as kernel parameters)

struct ColMap {
    int32_t c[kCopyCols];
};

// dst(i, c) = src(i, c) for rows [0, nrows) and columns [0, ncols) of one
// column tile; element (i, c) of a block at p + i * rs + map[c] * cs
template <class T>
__global__ void k_dense_copy(int64_t nrows, int ncols, const T *__restrict__ src, int64_t srs, int64_t scs, ColMap sm,
                             T *__restrict__ dst, int64_t drs, int64_t dcs, ColMap dm) {
    const int64_t n = nrows * ncols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / ncols;
        const int c = (int)(t - i * ncols);
        dst[i * drs + (int64_t)dm.c[c] * dcs] = src[i * srs + (int64_t)sm.c[c] * scs];
    }
}

// column j of the view as a column of the block at d->ptr
static int32_t col_of(const sp_dense *d, int32_t j) { return d->cols ? (*d->cols)[j] : j; }

int dense_copy(sp_dense *dst, const sp_dense *src, cudaStream_t s) {
    if (dst->nrows != src->nrows || dst->ncols != src->ncols) return SP_ERR_DIM;
    if (dst->dtype != src->dtype) return SP_ERR_DTYPE;
    if (dst->nrows == 0 || dst->ncols == 0) return SP_OK;
    const int64_t srs = src->layout == SP_ROW_MAJOR ? src->ld : 1, scs = src->layout == SP_ROW_MAJOR ? 1 : src->ld;
    const int64_t drs = dst->layout == SP_ROW_MAJOR ? dst->ld : 1, dcs = dst->layout == SP_ROW_MAJOR ? 1 : dst->ld;
    int sms = 1;
    SP_TRY(device_sm_count(&sms));
    for (int c0 = 0; c0 < dst->ncols; c0 += kCopyCols) {
        const int nc = std::min(kCopyCols, dst->ncols - c0);
        ColMap sm{}, dm{};
        for (int c = 0; c < nc; ++c) {
            sm.c[c] = col_of(src, c0 + c);
            dm.c[c] = col_of(dst, c0 + c);
        }
        const int64_t n = dst->nrows * nc;
        const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
        if (dst->dtype == SP_F64)
            k_dense_copy<double><<<blocks, 256, 0, s>>>(dst->nrows, nc, (const double *)src->ptr, srs, scs, sm,
                                                        (double *)dst->ptr, drs, dcs, dm);
        else
            k_dense_copy<float><<<blocks, 256, 0, s>>>(dst->nrows, nc, (const float *)src->ptr, srs, scs, sm,
                                                       (float *)dst->ptr, drs, dcs, dm);
        SP_CUDA(cudaGetLastError());
    }
    return SP_OK;
}

// true when the two views can touch a common element: views of one block
// (same base, leading dimension and layout) only through a common column;
// otherwise by their address ranges
bool dense_overlap(const sp_dense *a, const sp_dense *b) {
    if (a->nrows == 0 || b->nrows == 0 || a->ncols == 0 || b->ncols == 0) return false;
    if ((a->cols || b->cols) && a->ptr == b->ptr && a->ld == b->ld && a->layout == b->layout) {
        std::set<int32_t> ca;
        for (int32_t j = 0; j < a->ncols; ++j) ca.insert(col_of(a, j));
        for (int32_t j = 0; j < b->ncols; ++j)
            if (ca.count(col_of(b, j))) return true;
        return false;
    }
    const size_t es = dtype_size(a->dtype);
    auto ext = [&](const sp_dense *d, uintptr_t *lo, uintptr_t *hi) {
        int32_t cmax = 0;
        for (int32_t j = 0; j < d->ncols; ++j) cmax = std::max(cmax, col_of(d, j));
        const int64_t last = d->layout == SP_ROW_MAJOR ? (d->nrows - 1) * d->ld + cmax
                                                        : (int64_t)cmax * d->ld + (d->nrows - 1);
        *lo = (uintptr_t)d->ptr;
        *hi = (uintptr_t)d->ptr + (uintptr_t)(last * (int64_t)es + (int64_t)es - 1);
    };
    uintptr_t a0, a1, b0, b1;
    ext(a, &a0, &a1);
    ext(b, &b0, &b1);
    return a0 <= b1 && b0 <= a1;
}

// A compact row-major temporary with src's shape (stream-ordered), optionally
// filled from src.
static int compact_tmp(const sp_dense *src, Tmp &buf, sp_dense &view, bool fill, cudaStream_t s) {
    view = sp_dense{};
    view.nrows = src->nrows;
    view.ncols = src->ncols;
    view.ld = src->ncols;
    view.dtype = src->dtype;
    view.layout = SP_ROW_MAJOR;
    SP_TRY(buf.alloc((size_t)src->nrows * src->ncols * dtype_size(src->dtype)));
    view.ptr = buf.p;
    if (fill) SP_TRY(dense_copy(&view, src, s));
    return SP_OK;
}

int spmv_scattered(sp_dense *y, const sp_mat *A, const sp_dense *x, const sp_spmv_opts &o, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const bool chain = (o.flags & SP_SPMV_CHAIN_AXPBY) != 0;
    if (!x || !y || (chain && !o.z)) return SP_ERR_ARG;
    if (x->nrows == 0 || x->ncols == 0) return sp_spmv(y, A, x, &o, stream);
    if (dense_overlap(x, y) || (chain && (dense_overlap(o.z, x) || dense_overlap(o.z, y)))) return SP_ERR_ARG;
    Tmp bx(s), by(s), bz(s);
    sp_dense xc, yc, zc;
    const sp_dense *xp = x;
    sp_dense *yp = y, *zp = chain ? o.z : nullptr;
    if (dense_scattered(x)) {
        SP_TRY(compact_tmp(x, bx, xc, true, s));
        xp = &xc;
    }
    if (dense_scattered(y)) {
        SP_TRY(compact_tmp(y, by, yc, (o.flags & SP_SPMV_AXPBY) != 0, s));
        yp = &yc;
    }
    if (chain && dense_scattered(o.z)) {
        SP_TRY(compact_tmp(o.z, bz, zc, true, s));
        zp = &zc;
    }
    sp_spmv_opts o2 = o;
    o2.z = zp;
    SP_TRY(sp_spmv(yp, A, xp, &o2, stream));
    if (yp != y) SP_TRY(dense_copy(y, yp, s));
    if (chain && zp != o.z) SP_TRY(dense_copy(o.z, zp, s));
    return SP_OK;
}

}  // namespace sp

int sp_dense_view_scattered(sp_dense **out, const sp_dense *src, int32_t ncols, const int32_t *cols) {
    if (!out || !src || (ncols > 0 && !cols)) return SP_ERR_ARG;
    *out = nullptr;
    if (ncols < 0) return SP_ERR_DIM;
    auto v = std::make_shared<std::vector<int32_t>>(ncols);
    std::set<int32_t> seen;
    for (int32_t j = 0; j < ncols; ++j) {
        if (cols[j] < 0 || cols[j] >= src->ncols) return SP_ERR_DIM;
        if (!seen.insert(cols[j]).second) {
            sp_internal_set_detail("sp_dense_view_scattered", "a column is listed twice");
            return SP_ERR_ARG;
        }
        (*v)[j] = sp::col_of(src, cols[j]);
    }
    sp_dense *d = new sp_dense();
    *d = *src;
    d->owner.reset();
    d->ncols = ncols;
    d->cols = v;
    *out = d;
    return SP_OK;
}

int sp_dense_columns(const sp_dense *d, int32_t *cols) {
    if (!d) return SP_ERR_ARG;
    if (cols)
        for (int32_t j = 0; j < d->ncols; ++j) cols[j] = sp::col_of(d, j);
    return d->cols ? 1 : 0;
}

int sp_dense_clone(sp_dense **out, const sp_dense *src, sp_layout layout, void *stream) {
    if (!out || !src) return SP_ERR_ARG;
    *out = nullptr;
    sp_dense *d = nullptr;
    SP_TRY(sp_dense_create(&d, src->nrows, src->ncols, src->dtype, layout, stream));
    const int rc = sp::dense_copy(d, src, (cudaStream_t)stream);
    if (rc != SP_OK) {
        sp_dense_destroy(d, stream);
        return rc;
    }
    *out = d;
    return SP_OK;
}

int sp_dense_copy(sp_dense *dst, const sp_dense *src, void *stream) {
    if (!dst || !src) return SP_ERR_ARG;
    if (dst->ptr != src->ptr && sp::dense_overlap(dst, src)) return SP_ERR_ARG;
    if (dst->ptr == src->ptr && sp::dense_overlap(dst, src)) {
        // the same elements in the same places is a no-op; anything else overlaps
        bool same = dst->ld == src->ld && dst->layout == src->layout && dst->ncols == src->ncols;
        for (int32_t j = 0; same && j < dst->ncols; ++j) same = sp::col_of(dst, j) == sp::col_of(src, j);
        if (!same) return SP_ERR_ARG;
        return dst->nrows == src->nrows ? SP_OK : SP_ERR_DIM;
    }
    return sp::dense_copy(dst, src, (cudaStream_t)stream);
}
