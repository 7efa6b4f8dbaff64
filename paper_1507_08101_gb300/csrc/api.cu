// C ABI (include/sellcs.h): argument checking, memory ownership and dispatch.
// All arithmetic of the product runs in the kernels of the other units.
#include <atomic>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "spmv_kernel.cuh"

namespace sp {
template <class VT, class XT>
int launch_spmv_typed(const SpmvArgs &a, bool vec, int max_blocks, cudaStream_t s);
int launch_spmv_vty(const SpmvArgs &a, int max_blocks, cudaStream_t s);
int spmv_scattered(sp_dense *y, const sp_mat *A, const sp_dense *x, const sp_spmv_opts &o, void *stream);
}

static thread_local char g_detail[512] = "";

void sp_internal_set_detail(const char *prefix, const char *why) {
    snprintf(g_detail, sizeof(g_detail), "%s: %s", prefix, why);
}

void sp_internal_note_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_detail, sizeof(g_detail), "%s (%d) in %s at %s:%d", cudaGetErrorString(e), (int)e, what, file,
             line);
}

namespace sp {

int device_sm_count(int *n) {
    static int cached[64] = {0};
    int dev = 0;
    SP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SP_ERR_ARG;
    if (!cached[dev]) SP_CUDA(cudaDeviceGetAttribute(&cached[dev], cudaDevAttrMultiProcessorCount, dev));
    *n = cached[dev];
    return SP_OK;
}

void pool_keep_memory() {
    static std::atomic<bool> done[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return;
    }
    if (done[dev].load(std::memory_order_acquire)) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev].store(true, std::memory_order_release);
}

size_t device_l2_bytes() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cached[dev] && cudaDeviceGetAttribute(&cached[dev], cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (size_t)cached[dev];
}

// Scratch for the fused dot products: one partial per (value, block) for up to
// 8 resident blocks per SM (2048 threads / 256) and 3 x 32 values, plus the
// arrival ticket.
int spmv_scratch_need(int sm_count, size_t *bytes, int *max_blocks) {
    int mb = sm_count * (2048 / kMainThreads);
    *max_blocks = mb;
    *bytes = (size_t)mb * 3 * kMaxTileW * sizeof(double) + 256;
    return SP_OK;
}

static int ensure_scratch(sp_mat *A, cudaStream_t s) {
    if (A->scratch) return SP_OK;
    int sms = 1, mb = 0;
    size_t bytes = 0;
    SP_TRY(device_sm_count(&sms));
    SP_TRY(spmv_scratch_need(sms, &bytes, &mb));
    SP_TRY(dev_alloc(A->scratch, bytes, s));
    SP_CUDA(cudaMemsetAsync(A->scratch->ptr, 0, bytes, s));
    A->scratch_bytes = bytes;
    return SP_OK;
}

static int max_blocks_of(const sp_mat *A) {
    return (int)((A->scratch_bytes - 256) / (3 * kMaxTileW * sizeof(double)));
}

int launch_spmv(const SpmvLaunch &L, cudaStream_t s) {
    SpmvArgs a{};
    const Pattern &P = *L.P;
    a.val = L.val;
    a.col = (const int32_t *)P.col->ptr;
    a.chunkptr = (const int64_t *)P.chunkptr->ptr;
    a.chunklen = (const int32_t *)P.chunklen->ptr;
    a.slotlen = (const int32_t *)P.slotlen->ptr;
    a.perm = (P.sigma == 1 || P.permuted_space) ? nullptr : (const int32_t *)P.perm->ptr;
    a.nrows = P.nrows;
    a.nslots = P.nslots;
    a.C = P.C;
    a.w = L.w;
    a.x = L.x.ptr;
    a.xrs = L.x.rs;
    a.xcs = L.x.cs;
    a.y = (void *)L.y.ptr;
    a.yrs = L.y.rs;
    a.ycs = L.y.cs;
    a.z = (void *)L.z.ptr;
    a.zrs = L.z.rs;
    a.zcs = L.z.cs;
    a.flags = L.flags;
    a.alpha = L.alpha;
    a.beta = L.beta;
    a.delta = L.delta;
    a.eta = L.eta;
    a.dot = L.dot;
    a.dot_stride = L.dot_stride;
    a.dot_off = L.dot_off;
    a.partials = L.partials;
    a.ticket = L.ticket;
    a.sched = nullptr;
    a.sched_rounds = 0;
    a.wbounds = nullptr;
    a.wbounds_src = L.P;
    for (int k = 0; k < kMaxTileW; ++k) a.gamma[k] = (L.gamma && k < L.w) ? L.gamma[k] : 0.0;

    size_t xs = dtype_size(L.xdt);
    int cpl = host_cols_per_lane(xs, L.w);
    size_t align = std::min<size_t>(16, cpl * xs);
    auto aligned = [&](const VecDesc &v) {
        return v.cs == 1 && ((v.rs * xs) % align == 0) && ((uintptr_t)v.ptr % align == 0);
    };
    bool vec = (L.w % cpl == 0) && aligned(L.x) && aligned(L.y) &&
               (!(L.flags & SP_SPMV_CHAIN_AXPBY) || aligned(L.z));
    if (L.vdt == SP_F64 && L.xdt == SP_F64) return launch_spmv_typed<double, double>(a, vec, L.max_blocks, s);
    if (L.vdt == SP_F32 && L.xdt == SP_F64) return launch_spmv_typed<float, double>(a, vec, L.max_blocks, s);
    if (L.vdt == SP_F32 && L.xdt == SP_F32) return launch_spmv_typed<float, float>(a, vec, L.max_blocks, s);
    if (L.vdt == SP_BF16 && L.xdt == SP_F64)
        return launch_spmv_typed<__nv_bfloat16, double>(a, vec, L.max_blocks, s);
    if (L.vdt == SP_BF16 && L.xdt == SP_F32)
        return launch_spmv_typed<__nv_bfloat16, float>(a, vec, L.max_blocks, s);
    return SP_ERR_DTYPE;
}

static VecDesc desc_of(const sp_dense *d, int32_t col0) {
    VecDesc v;
    size_t es = dtype_size(d->dtype);
    if (d->layout == SP_ROW_MAJOR) {
        v.rs = d->ld;
        v.cs = 1;
    } else {
        v.rs = 1;
        v.cs = d->ld;
    }
    v.ptr = (const char *)d->ptr + (size_t)(col0 * v.cs) * es;
    return v;
}

// [first byte, last byte] touched by a block vector
static void extent(const sp_dense *d, uintptr_t *lo, uintptr_t *hi) {
    size_t es = dtype_size(d->dtype);
    int64_t last;
    if (d->layout == SP_ROW_MAJOR)
        last = (d->nrows - 1) * d->ld + (d->ncols - 1);
    else
        last = (int64_t)(d->ncols - 1) * d->ld + (d->nrows - 1);
    *lo = (uintptr_t)d->ptr;
    *hi = (uintptr_t)d->ptr + (uintptr_t)(last * es + es - 1);
}

static bool overlap(const sp_dense *a, const sp_dense *b) {
    if (a->nrows == 0 || b->nrows == 0 || a->ncols == 0 || b->ncols == 0) return false;
    uintptr_t a0, a1, b0, b1;
    extent(a, &a0, &a1);
    extent(b, &b0, &b1);
    return a0 <= b1 && b0 <= a1;
}

static bool valid_vec_dtype(sp_dtype t) { return t == SP_F64 || t == SP_F32; }
static bool valid_val_dtype(sp_dtype t) { return t == SP_F64 || t == SP_F32 || t == SP_BF16; }

}  // namespace sp

using namespace sp;

extern "C" {

const char *sp_error_string(int code) {
    switch (code) {
        case SP_OK: return "ok";
        case SP_ERR_ARG: return "invalid argument";
        case SP_ERR_DIM: return "dimension mismatch";
        case SP_ERR_DTYPE: return "unsupported precision";
        case SP_ERR_CUDA: return "CUDA error";
        case SP_ERR_OOM: return "out of device memory";
        case SP_ERR_TIMEOUT: return "device wait timed out";
        case SP_ERR_FORMAT: return "malformed CSR input";
        case SP_ERR_UNSUPPORTED: return "unsupported request";
        default: return "unknown error";
    }
}

const char *sp_last_error_detail(void) { return g_detail; }

int sp_device_sm_count(int *count) {
    if (!count) return SP_ERR_ARG;
    return device_sm_count(count);
}

int sp_mat_create_csr(sp_mat **out, int64_t nrows, int64_t ncols, const int64_t *rowptr, const int32_t *col,
                      const void *val, int C, int64_t sigma, sp_dtype val_dtype, unsigned flags, void *stream) {
    if (!out || !rowptr) return SP_ERR_ARG;
    *out = nullptr;
    if (nrows < 0 || ncols < 0 || nrows >= (1LL << 31) || ncols >= (1LL << 31)) return SP_ERR_DIM;
    if (C < 1 || C > 1024 || sigma < 1) return SP_ERR_ARG;
    if (!valid_val_dtype(val_dtype)) return SP_ERR_DTYPE;
    if (flags & ~(SP_MAT_CSR_ON_DEVICE | SP_MAT_VAL_F32 | SP_MAT_WITH_TRANSPOSE | SP_MAT_ORDER_FRONT |
                  SP_MAT_ORDER_RANGES | SP_MAT_PERMUTED_SPACE))
        return SP_ERR_ARG;
    if ((flags & SP_MAT_ORDER_FRONT) && (flags & SP_MAT_ORDER_RANGES)) return SP_ERR_ARG;
    if ((flags & SP_MAT_PERMUTED_SPACE) && (flags & SP_MAT_WITH_TRANSPOSE)) return SP_ERR_ARG;
    if ((flags & SP_MAT_PERMUTED_SPACE) && nrows != ncols) return SP_ERR_DIM;
    cudaStream_t s = (cudaStream_t)stream;
    bool on_dev = flags & SP_MAT_CSR_ON_DEVICE;
    bool f32 = flags & SP_MAT_VAL_F32;
    size_t vs = f32 ? 4 : 8;
    int64_t nnz = 0;
    if (on_dev) {
        // on the caller's stream, so that a row pointer array written there is complete
        SP_CUDA(cudaMemcpyAsync(&nnz, rowptr + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
    }
    else
        nnz = rowptr[nrows];
    if (nnz < 0) return SP_ERR_FORMAT;
    if (nnz > 0 && (!col || !val)) return SP_ERR_ARG;
    if (nrows > 0 && ncols == 0 && nnz > 0) return SP_ERR_FORMAT;

    DevBufPtr drp, dcol, dval;
    const int64_t *prp = rowptr;
    const int32_t *pcol = col;
    const void *pval = val;
    if (!on_dev) {
        SP_TRY(dev_alloc(drp, (nrows + 1) * sizeof(int64_t), s));
        SP_TRY(dev_alloc(dcol, std::max<int64_t>(nnz, 1) * sizeof(int32_t), s));
        SP_TRY(dev_alloc(dval, std::max<int64_t>(nnz, 1) * vs, s));
        SP_CUDA(cudaMemcpyAsync(drp->ptr, rowptr, (nrows + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if (nnz) {
            SP_CUDA(cudaMemcpyAsync(dcol->ptr, col, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            SP_CUDA(cudaMemcpyAsync(dval->ptr, val, nnz * vs, cudaMemcpyHostToDevice, s));
        }
        prp = (const int64_t *)drp->ptr;
        pcol = (const int32_t *)dcol->ptr;
        pval = dval->ptr;
    }
    sp_mat *A = new sp_mat();
    A->vdt = val_dtype;
    int rc = build_pattern_and_values(A, nrows, ncols, prp, pcol, pval, f32, C, sigma, s,
                                      (flags & SP_MAT_PERMUTED_SPACE) != 0);
    if (rc == SP_OK && (flags & SP_MAT_WITH_TRANSPOSE)) rc = build_transpose(A, prp, pcol, pval, f32, s);
    if (rc == SP_OK) {
        const int order = (flags & SP_MAT_ORDER_FRONT) ? 1 : (flags & SP_MAT_ORDER_RANGES) ? 2 : 0;
        A->pat->order = order;
        if (A->transpose) A->transpose->pat->order = order;
    }
    if (rc == SP_OK) rc = ensure_scratch(A, s);
    if (rc == SP_OK && A->transpose) rc = ensure_scratch(A->transpose, s);
    if (rc == SP_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            sp_internal_note_cuda_error(e, "create sync", __FILE__, __LINE__);
            rc = SP_ERR_CUDA;
        }
    }
    if (rc != SP_OK) {
        cudaStreamSynchronize(s);
        delete A->transpose;
        delete A;
        return rc;
    }
    *out = A;
    return SP_OK;
}

int sp_mat_update_values(sp_mat *A, const void *val, unsigned flags, void *stream) {
    if (!A || (!val && A->pat->nnz > 0)) return SP_ERR_ARG;
    if (flags & ~(SP_MAT_CSR_ON_DEVICE | SP_MAT_VAL_F32)) return SP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    bool f32 = flags & SP_MAT_VAL_F32;
    size_t vs = f32 ? 4 : 8;
    int64_t nnz = A->pat->nnz;
    DevBufPtr tmp;
    const void *pv = val;
    if (!(flags & SP_MAT_CSR_ON_DEVICE)) {
        SP_TRY(dev_alloc(tmp, std::max<int64_t>(nnz, 1) * vs, s));
        SP_CUDA(cudaMemcpyAsync(tmp->ptr, val, nnz * vs, cudaMemcpyHostToDevice, s));
        pv = tmp->ptr;
    }
    SP_TRY(fill_values_from_csr(*A->pat, A->vdt, A->val->ptr, pv, f32, s));
    if (A->transpose) {
        const Pattern &T = *A->transpose->pat;
        DevBufPtr tv;
        SP_TRY(dev_alloc(tv, std::max<int64_t>(nnz, 1) * vs, s));
        SP_TRY(gather_values(pv, f32, (const int64_t *)T.src_index->ptr, nnz, tv->ptr, f32, s));
        SP_TRY(fill_values_from_csr(T, A->transpose->vdt, A->transpose->val->ptr, tv->ptr, f32, s));
        // keep the temporary alive until the gather has run
        SP_CUDA(cudaStreamSynchronize(s));
    } else if (tmp) {
        SP_CUDA(cudaStreamSynchronize(s));
    }
    return SP_OK;
}

static int clone_one(sp_mat **out, const sp_mat *A, sp_dtype vdt, cudaStream_t s) {
    sp_mat *B = new sp_mat();
    B->pat = A->pat;
    B->vdt = vdt;
    int rc = dev_alloc(B->val, A->pat->nstored * dtype_size(vdt), s);
    if (rc == SP_OK) rc = convert_values(A->val->ptr, A->vdt, B->val->ptr, vdt, A->pat->nstored, s);
    if (rc == SP_OK) rc = ensure_scratch(B, s);
    if (rc != SP_OK) {
        delete B;
        return rc;
    }
    *out = B;
    return SP_OK;
}

int sp_mat_clone_values(sp_mat **out, const sp_mat *A, sp_dtype val_dtype, void *stream) {
    if (!out || !A) return SP_ERR_ARG;
    if (!valid_val_dtype(val_dtype)) return SP_ERR_DTYPE;
    cudaStream_t s = (cudaStream_t)stream;
    sp_mat *B = nullptr;
    SP_TRY(clone_one(&B, A, val_dtype, s));
    if (A->transpose) {
        int rc = clone_one(&B->transpose, A->transpose, val_dtype, s);
        if (rc != SP_OK) {
            delete B;
            return rc;
        }
    }
    *out = B;
    return SP_OK;
}

int sp_mat_info(const sp_mat *A, sp_mat_info_t *info) {
    if (!A || !info) return SP_ERR_ARG;
    const Pattern &P = *A->pat;
    info->nrows = P.nrows;
    info->ncols = P.ncols;
    info->nnz = P.nnz;
    info->nchunks = P.nchunks;
    info->nstored = P.nstored;
    info->C = P.C;
    info->maxrowlen = P.maxrowlen;
    info->sigma = P.sigma;
    info->val_dtype = A->vdt;
    info->has_transpose = A->transpose != nullptr;
    return SP_OK;
}

static int export_sell(const sp_mat *A, int64_t *chunkptr, int32_t *chunklen, int32_t *slotlen, int32_t *perm,
                       int32_t *col, double *val, cudaStream_t s) {
    const Pattern &P = *A->pat;
    if (chunkptr)
        SP_CUDA(cudaMemcpyAsync(chunkptr, P.chunkptr->ptr, (P.nchunks + 1) * 8, cudaMemcpyDeviceToHost, s));
    if (chunklen && P.nchunks)
        SP_CUDA(cudaMemcpyAsync(chunklen, P.chunklen->ptr, P.nchunks * 4, cudaMemcpyDeviceToHost, s));
    if (slotlen && P.nslots)
        SP_CUDA(cudaMemcpyAsync(slotlen, P.slotlen->ptr, P.nslots * 4, cudaMemcpyDeviceToHost, s));
    if (perm && P.nslots) SP_CUDA(cudaMemcpyAsync(perm, P.perm->ptr, P.nslots * 4, cudaMemcpyDeviceToHost, s));
    if (col && P.nstored) SP_CUDA(cudaMemcpyAsync(col, P.col->ptr, P.nstored * 4, cudaMemcpyDeviceToHost, s));
    if (val && P.nstored) {
        DevBufPtr w;
        SP_TRY(dev_alloc(w, P.nstored * 8, s));
        SP_TRY(widen_values(A->val->ptr, A->vdt, (double *)w->ptr, P.nstored, s));
        SP_CUDA(cudaMemcpyAsync(val, w->ptr, P.nstored * 8, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
    }
    SP_CUDA(cudaStreamSynchronize(s));
    return SP_OK;
}

int sp_mat_export_sell(const sp_mat *A, int64_t *chunkptr, int32_t *chunklen, int32_t *slotlen, int32_t *perm,
                       int32_t *col, double *val, void *stream) {
    if (!A) return SP_ERR_ARG;
    return export_sell(A, chunkptr, chunklen, slotlen, perm, col, val, (cudaStream_t)stream);
}

int sp_mat_export_sell_transpose(const sp_mat *A, int64_t *chunkptr, int32_t *chunklen, int32_t *slotlen,
                                 int32_t *perm, int32_t *col, double *val, void *stream) {
    if (!A || !A->transpose) return SP_ERR_ARG;
    return export_sell(A->transpose, chunkptr, chunklen, slotlen, perm, col, val, (cudaStream_t)stream);
}

}  // extern "C"

namespace sp {
// SELL -> CSR on the device (inverse of the scatter).
// colmap (may be null): map from stored indices back to the user's columns
__global__ void k_sell_to_csr(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ perm,
                              const int32_t *__restrict__ slotlen, const int64_t *__restrict__ chunkptr,
                              const int32_t *__restrict__ col_sell, const double *__restrict__ val_sell,
                              int64_t nslots, int C, const int32_t *__restrict__ colmap, int32_t *__restrict__ col,
                              double *__restrict__ val) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslots;
         s += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = perm[s];
        if (i < 0) continue;
        int64_t c = s / C, r = s - c * C;
        int64_t src = chunkptr[c] + r, dst = rowptr[i];
        for (int32_t j = 0; j < slotlen[s]; ++j) {
            const int32_t cs = col_sell[src + (int64_t)j * C];
            col[dst + j] = colmap ? colmap[cs] : cs;
            val[dst + j] = val_sell[src + (int64_t)j * C];
        }
    }
}
}  // namespace sp

extern "C" {

int sp_mat_to_csr(const sp_mat *A, int64_t *rowptr, int32_t *col, double *val, void *stream) {
    if (!A || !rowptr) return SP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const Pattern &P = *A->pat;
    SP_CUDA(cudaMemcpyAsync(rowptr, P.rowptr->ptr, (P.nrows + 1) * 8, cudaMemcpyDeviceToHost, s));
    if (P.nnz > 0) {
        if (!col || !val) return SP_ERR_ARG;
        DevBufPtr wv, dc, dv;
        SP_TRY(dev_alloc(wv, P.nstored * 8, s));
        SP_TRY(dev_alloc(dc, P.nnz * 4, s));
        SP_TRY(dev_alloc(dv, P.nnz * 8, s));
        SP_TRY(widen_values(A->val->ptr, A->vdt, (double *)wv->ptr, P.nstored, s));
        int g = (int)std::min<int64_t>((P.nslots + 255) / 256, 65535 * 16);
        k_sell_to_csr<<<std::max(g, 1), 256, 0, s>>>((const int64_t *)P.rowptr->ptr, (const int32_t *)P.perm->ptr,
                                                     (const int32_t *)P.slotlen->ptr,
                                                     (const int64_t *)P.chunkptr->ptr, (const int32_t *)P.col->ptr,
                                                     (const double *)wv->ptr, P.nslots, P.C,
                                                     P.permuted_space ? (const int32_t *)P.perm->ptr : nullptr,
                                                     (int32_t *)dc->ptr,
                                                     (double *)dv->ptr);
        SP_CUDA(cudaGetLastError());
        SP_CUDA(cudaMemcpyAsync(col, dc->ptr, P.nnz * 4, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaMemcpyAsync(val, dv->ptr, P.nnz * 8, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
    }
    SP_CUDA(cudaStreamSynchronize(s));
    return SP_OK;
}

int sp_mat_destroy(sp_mat *A, void *stream) {
    if (!A) return SP_ERR_ARG;
    cudaStreamSynchronize((cudaStream_t)stream);
    delete A->transpose;
    delete A;
    return SP_OK;
}

// ------------------------------------------------------------------ dense

int sp_dense_create(sp_dense **out, int64_t nrows, int32_t ncols, sp_dtype dtype, sp_layout layout, void *stream) {
    if (!out) return SP_ERR_ARG;
    *out = nullptr;
    if (nrows < 0 || ncols < 0) return SP_ERR_DIM;
    if (!valid_vec_dtype(dtype)) return SP_ERR_DTYPE;
    if (layout != SP_ROW_MAJOR && layout != SP_COL_MAJOR) return SP_ERR_ARG;
    sp_dense *d = new sp_dense();
    d->nrows = nrows;
    d->ncols = ncols;
    d->dtype = dtype;
    d->layout = layout;
    d->ld = layout == SP_ROW_MAJOR ? ncols : nrows;
    size_t bytes = (size_t)nrows * ncols * dtype_size(dtype);
    int rc = dev_alloc(d->owner, bytes, (cudaStream_t)stream);
    if (rc != SP_OK) {
        delete d;
        return rc;
    }
    d->ptr = d->owner->ptr;
    if (bytes) {
        cudaError_t e = cudaMemsetAsync(d->ptr, 0, bytes, (cudaStream_t)stream);
        if (e != cudaSuccess) {
            delete d;
            return SP_ERR_CUDA;
        }
    }
    *out = d;
    return SP_OK;
}

int sp_dense_view(sp_dense **out, void *dev_ptr, int64_t nrows, int32_t ncols, int64_t ld, sp_dtype dtype,
                  sp_layout layout) {
    if (!out) return SP_ERR_ARG;
    *out = nullptr;
    if (nrows < 0 || ncols < 0) return SP_ERR_DIM;
    if (!valid_vec_dtype(dtype)) return SP_ERR_DTYPE;
    if (layout != SP_ROW_MAJOR && layout != SP_COL_MAJOR) return SP_ERR_ARG;
    if (!dev_ptr && nrows > 0 && ncols > 0) return SP_ERR_ARG;
    if (layout == SP_ROW_MAJOR ? ld < ncols : ld < nrows) return SP_ERR_DIM;
    sp_dense *d = new sp_dense();
    d->ptr = dev_ptr;
    d->nrows = nrows;
    d->ncols = ncols;
    d->ld = ld;
    d->dtype = dtype;
    d->layout = layout;
    *out = d;
    return SP_OK;
}

int sp_dense_view_cols(sp_dense **out, const sp_dense *src, int32_t col0, int32_t ncols) {
    if (!out || !src) return SP_ERR_ARG;
    *out = nullptr;
    if (col0 < 0 || ncols < 0 || col0 + ncols > src->ncols) return SP_ERR_DIM;
    sp_dense *d = new sp_dense();
    *d = *src;
    d->owner.reset();
    d->ncols = ncols;
    if (src->cols) {
        // a run of a scattered view's columns is scattered too
        d->cols = std::make_shared<const std::vector<int32_t>>(src->cols->begin() + col0,
                                                               src->cols->begin() + col0 + ncols);
    } else {
        size_t es = dtype_size(src->dtype);
        d->ptr = (char *)src->ptr + (size_t)col0 * (src->layout == SP_ROW_MAJOR ? 1 : src->ld) * es;
    }
    *out = d;
    return SP_OK;
}

int sp_dense_data(const sp_dense *d, void **ptr, int64_t *nrows, int32_t *ncols, int64_t *ld, sp_dtype *dtype,
                  sp_layout *layout) {
    if (!d) return SP_ERR_ARG;
    if (ptr) *ptr = d->ptr;
    if (nrows) *nrows = d->nrows;
    if (ncols) *ncols = d->ncols;
    if (ld) *ld = d->ld;
    if (dtype) *dtype = d->dtype;
    if (layout) *layout = d->layout;
    return SP_OK;
}

int sp_dense_destroy(sp_dense *d, void *stream) {
    if (!d) return SP_ERR_ARG;
    if (d->owner) cudaStreamSynchronize((cudaStream_t)stream);
    delete d;
    return SP_OK;
}

// ------------------------------------------------------------------ spmv

int sp_spmv(sp_dense *y, const sp_mat *A, const sp_dense *x, const sp_spmv_opts *opts, void *stream) {
    static const sp_spmv_opts defaults = SP_SPMV_OPTS_INIT;
    if (!y || !A || !x) return SP_ERR_ARG;
    const sp_spmv_opts &o = opts ? *opts : defaults;
    // scattered views: the product runs on compact clones, copied back
    if (dense_scattered(x) || dense_scattered(y) || ((o.flags & SP_SPMV_CHAIN_AXPBY) && dense_scattered(o.z)))
        return spmv_scattered(y, A, x, o, stream);
    const uint32_t known = SP_SPMV_SCALE | SP_SPMV_SHIFT | SP_SPMV_VSHIFT | SP_SPMV_AXPBY | SP_SPMV_DOT_ANY |
                           SP_SPMV_CHAIN_AXPBY | SP_SPMV_DOT_HOST;
    uint32_t f = o.flags;
    if (f & ~known) return SP_ERR_ARG;
    const Pattern &P = *A->pat;
    if (x->nrows != P.ncols || y->nrows != P.nrows || x->ncols != y->ncols) return SP_ERR_DIM;
    if (x->dtype != y->dtype) return SP_ERR_DTYPE;
    if (!valid_vec_dtype(x->dtype)) return SP_ERR_DTYPE;
    if (A->vdt == SP_F64 && x->dtype != SP_F64) return SP_ERR_DTYPE;
    const int w = x->ncols;
    bool shift = f & (SP_SPMV_SHIFT | SP_SPMV_VSHIFT);
    if ((f & SP_SPMV_SHIFT) && (f & SP_SPMV_VSHIFT)) return SP_ERR_ARG;
    if (shift && !o.gamma) return SP_ERR_ARG;
    if ((f & SP_SPMV_VSHIFT) && w > SP_MAX_VSHIFT) return SP_ERR_ARG;
    // the identity of the shift (and x_i in the dots) is the leading nrows x nrows
    // block: x's first nrows rows (a square A, or a process's rows [A_loc | A_rem]
    // over x extended by its halo)
    if ((shift || (f & (SP_SPMV_DOT_XY | SP_SPMV_DOT_XX))) && P.ncols < P.nrows) return SP_ERR_DIM;
    if ((f & SP_SPMV_DOT_ANY) && !o.dot) return SP_ERR_ARG;
    bool chain = f & SP_SPMV_CHAIN_AXPBY;
    if (chain) {
        if (!o.z) return SP_ERR_ARG;
        if (o.z->nrows != y->nrows || o.z->ncols != y->ncols) return SP_ERR_DIM;
        if (o.z->dtype != y->dtype) return SP_ERR_DTYPE;
        if (overlap(o.z, x) || overlap(o.z, y)) return SP_ERR_ARG;
    }
    if (overlap(x, y)) return SP_ERR_ARG;
    if (w == 0) return SP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (!A->scratch) return SP_ERR_ARG;

    std::vector<double> gam(w, 0.0);
    if (f & SP_SPMV_SHIFT)
        std::fill(gam.begin(), gam.end(), o.gamma[0]);
    else if (f & SP_SPMV_VSHIFT)
        std::copy(o.gamma, o.gamma + w, gam.begin());

    bool host_dot = (f & SP_SPMV_DOT_HOST) && (f & SP_SPMV_DOT_ANY);
    Tmp ddot(s);  // stream-ordered
    double *dot = o.dot;
    if (host_dot) {
        SP_TRY(ddot.alloc(3 * (size_t)w * sizeof(double)));
        dot = ddot.as<double>();
    }
    SpmvLaunch L;
    L.P = &P;
    L.val = A->val->ptr;
    L.vdt = A->vdt;
    L.xdt = x->dtype;
    L.flags = f & ~SP_SPMV_DOT_HOST;
    L.alpha = o.alpha;
    L.beta = o.beta;
    L.delta = o.delta;
    L.eta = o.eta;
    L.dot = dot;
    L.dot_stride = w;
    L.partials = (double *)A->scratch->ptr;
    L.ticket = (unsigned *)((char *)A->scratch->ptr + A->scratch_bytes - 256);
    L.max_blocks = max_blocks_of(A);
    for (int c0 = 0; c0 < w; c0 += kMaxTileW) {
        int wt = std::min(kMaxTileW, w - c0);
        L.w = wt;
        L.x = desc_of(x, c0);
        L.y = desc_of(y, c0);
        L.z = chain ? desc_of(o.z, c0) : VecDesc{nullptr, 0, 0};
        L.gamma = gam.data() + c0;
        L.dot_off = c0;
        SP_TRY(launch_spmv(L, s));
    }
    if (host_dot) {
        for (int q = 0; q < 3; ++q)
            if (f & (SP_SPMV_DOT_YY << q))
                SP_CUDA(cudaMemcpyAsync(o.dot + (size_t)q * w, dot + (size_t)q * w, w * sizeof(double),
                                        cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
    }
    return SP_OK;
}

int sp_spmv_vty(sp_dense *y, const sp_mat *A, const sp_dense *x, const sp_spmv_opts *opts, const sp_dense *V,
                double *C, int64_t ldc, void *stream) {
    static const sp_spmv_opts defaults = SP_SPMV_OPTS_INIT;
    if (!y || !A || !x || !V || !C) return SP_ERR_ARG;
    const sp_spmv_opts &o = opts ? *opts : defaults;
    const uint32_t f = o.flags;
    const uint32_t known = SP_SPMV_SCALE | SP_SPMV_SHIFT | SP_SPMV_VSHIFT | SP_SPMV_AXPBY | SP_SPMV_CHAIN_AXPBY;
    if (f & ~known) return SP_ERR_ARG;  // the fused dots are not combined with V^T y here
    if (dense_scattered(x) || dense_scattered(y) || dense_scattered(V) ||
        ((f & SP_SPMV_CHAIN_AXPBY) && dense_scattered(o.z)))
        return scattered_refused("sp_spmv_vty");
    const Pattern &P = *A->pat;
    if (P.permuted_space) return SP_ERR_ARG;
    if (A->vdt != SP_F64 || x->dtype != SP_F64 || y->dtype != SP_F64 || V->dtype != SP_F64) return SP_ERR_DTYPE;
    if (x->layout != SP_ROW_MAJOR || y->layout != SP_ROW_MAJOR || V->layout != SP_ROW_MAJOR) return SP_ERR_ARG;
    if (x->nrows != P.ncols || y->nrows != P.nrows || x->ncols != y->ncols || V->nrows != y->nrows)
        return SP_ERR_DIM;
    const int w = x->ncols, m = V->ncols;
    if (w < 1 || w > 8 || m < 1 || m > 8) return SP_ERR_UNSUPPORTED;
    if (ldc < w) return SP_ERR_DIM;
    const bool shift = f & (SP_SPMV_SHIFT | SP_SPMV_VSHIFT);
    if ((f & SP_SPMV_SHIFT) && (f & SP_SPMV_VSHIFT)) return SP_ERR_ARG;
    if (shift && !o.gamma) return SP_ERR_ARG;
    if (shift && P.ncols < P.nrows) return SP_ERR_DIM;
    const bool chain = f & SP_SPMV_CHAIN_AXPBY;
    if (chain) {
        if (!o.z) return SP_ERR_ARG;
        if (o.z->nrows != y->nrows || o.z->ncols != w) return SP_ERR_DIM;
        if (o.z->dtype != SP_F64 || o.z->layout != SP_ROW_MAJOR) return SP_ERR_ARG;
        if (overlap(o.z, x) || overlap(o.z, y) || overlap(o.z, V)) return SP_ERR_ARG;
    }
    if (overlap(x, y) || overlap(V, y)) return SP_ERR_ARG;
    // vector loads of whole rows: rows a multiple of the lane vector, aligned
    const int cpl = host_cols_per_lane(8, w);
    const size_t align = std::min<size_t>(16, (size_t)cpl * 8);
    auto ok = [&](const sp_dense *d) { return ((uintptr_t)d->ptr % align) == 0 && ((size_t)d->ld * 8) % align == 0; };
    if (w % cpl != 0 || !ok(x) || !ok(y) || (chain && !ok(o.z))) return SP_ERR_UNSUPPORTED;
    int wp = 1;
    while (wp < w) wp <<= 1;
    if (host_log2_tpr(P.C, wp / cpl) != 0) return SP_ERR_UNSUPPORTED;  // rows split over lanes: not here
    if (!A->scratch) return SP_ERR_ARG;
    SpmvArgs a{};
    a.val = A->val->ptr;
    a.col = (const int32_t *)P.col->ptr;
    a.chunkptr = (const int64_t *)P.chunkptr->ptr;
    a.chunklen = (const int32_t *)P.chunklen->ptr;
    a.slotlen = (const int32_t *)P.slotlen->ptr;
    a.perm = P.sigma == 1 ? nullptr : (const int32_t *)P.perm->ptr;
    a.nrows = P.nrows;
    a.nslots = P.nslots;
    a.C = P.C;
    a.w = w;
    a.x = x->ptr;
    a.xrs = x->ld;
    a.xcs = 1;
    a.y = y->ptr;
    a.yrs = y->ld;
    a.ycs = 1;
    a.z = chain ? o.z->ptr : nullptr;
    a.zrs = chain ? o.z->ld : 0;
    a.zcs = 1;
    a.flags = f;
    a.alpha = o.alpha;
    a.beta = o.beta;
    a.delta = o.delta;
    a.eta = o.eta;
    a.partials = (double *)A->scratch->ptr;
    a.ticket = (unsigned *)((char *)A->scratch->ptr + A->scratch_bytes - 256);
    a.wbounds_src = &P;
    a.vty_V = (const double *)V->ptr;
    a.vty_ldv = V->ld;
    a.vty_m = m;
    a.vty_vec2 = ((uintptr_t)V->ptr % 16 == 0 && V->ld % 2 == 0) ? 1 : 0;
    a.vty_C = C;
    a.vty_ldc = ldc;
    for (int k = 0; k < kMaxTileW; ++k)
        a.gamma[k] = !shift || k >= w ? 0.0 : ((f & SP_SPMV_SHIFT) ? o.gamma[0] : o.gamma[k]);
    if (P.nrows == 0) {
        SP_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * (size_t)ldc * m, (cudaStream_t)stream));
        return SP_OK;
    }
    return launch_spmv_vty(a, max_blocks_of(A), (cudaStream_t)stream);
}

int sp_spmv_adjoint(sp_dense *dx, void *dvals, const sp_mat *A, const sp_dense *x, const sp_dense *g,
                    void *stream) {
    if (A && A->pat->permuted_space) return SP_ERR_ARG;  // the adjoint works in the user's order
    if (!A || !g) return SP_ERR_ARG;
    if (dense_scattered(dx) || dense_scattered(x) || dense_scattered(g)) return sp::scattered_refused("sp_spmv_adjoint");
    const Pattern &P = *A->pat;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->nrows != P.nrows) return SP_ERR_DIM;
    if (!valid_vec_dtype(g->dtype)) return SP_ERR_DTYPE;
    if (dx) {
        if (!A->transpose) return SP_ERR_ARG;
        if (dx->nrows != P.ncols || dx->ncols != g->ncols) return SP_ERR_DIM;
        if (dx->dtype != g->dtype) return SP_ERR_DTYPE;
        sp_spmv_opts o = SP_SPMV_OPTS_INIT;
        SP_TRY(sp_spmv(dx, A->transpose, g, &o, stream));
    }
    if (dvals) {
        if (!x) return SP_ERR_ARG;
        if (x->nrows != P.ncols || x->ncols != g->ncols) return SP_ERR_DIM;
        if (x->dtype != g->dtype) return SP_ERR_DTYPE;
        if (x->layout != SP_ROW_MAJOR || g->layout != SP_ROW_MAJOR || x->ld != x->ncols || g->ld != g->ncols)
            return SP_ERR_UNSUPPORTED;
        if (P.nnz > 0) SP_TRY(launch_sampled(P, x->dtype, x->ncols, x->ptr, g->ptr, dvals, s));
    }
    return SP_OK;
}

}  // extern "C"

namespace sp {
// row permutation of a block vector between the user's and the SELL row order
template <class T>
__global__ void k_permute_rows(const int32_t *__restrict__ perm, int64_t nrows, int w, const T *__restrict__ in,
                               int64_t ldi, T *__restrict__ out, int64_t ldo, int to_sell) {
    const int64_t total = nrows * w;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t / w;
        const int k = (int)(t - s * w);
        const int64_t i = perm[s];
        if (to_sell)
            out[s * ldo + k] = in[i * ldi + k];
        else
            out[i * ldo + k] = in[s * ldi + k];
    }
}
}  // namespace sp

extern "C" int sp_mat_permute(const sp_mat *A, sp_dense *out, const sp_dense *in, int to_sell, void *stream) {
    if (!A || !out || !in) return SP_ERR_ARG;
    if (sp::dense_scattered(out) || sp::dense_scattered(in)) return sp::scattered_refused("sp_mat_permute");
    const sp::Pattern &P = *A->pat;
    if (in->nrows != P.nrows || out->nrows != P.nrows || in->ncols != out->ncols) return SP_ERR_DIM;
    if (in->dtype != out->dtype || (in->dtype != SP_F64 && in->dtype != SP_F32)) return SP_ERR_DTYPE;
    if (in->layout != SP_ROW_MAJOR || out->layout != SP_ROW_MAJOR) return SP_ERR_ARG;
    const size_t xs = in->dtype == SP_F64 ? 8 : 4;
    const char *ib = (const char *)in->ptr, *ob = (const char *)out->ptr;
    const size_t ispan = (size_t)in->ld * in->nrows * xs, ospan = (size_t)out->ld * out->nrows * xs;
    if (ib < ob + ospan && ob < ib + ispan) return SP_ERR_ARG;  // overlap
    const int64_t total = P.nrows * (int64_t)in->ncols;
    if (total == 0) return SP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 65535 * 16);
    const int32_t *perm = (const int32_t *)P.perm->ptr;
    if (in->dtype == SP_F64)
        sp::k_permute_rows<double><<<grid, 256, 0, s>>>(perm, P.nrows, in->ncols, (const double *)in->ptr, in->ld,
                                                         (double *)out->ptr, out->ld, to_sell);
    else
        sp::k_permute_rows<float><<<grid, 256, 0, s>>>(perm, P.nrows, in->ncols, (const float *)in->ptr, in->ld,
                                                        (float *)out->ptr, out->ld, to_sell);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}
