// Pipelined augmented product over block vectors in HOST memory.
//
// A plan owns kSets sets of device buffers (x, y, z, dots) and three streams:
// copy-in, product, copy-out.  Call k uses set k mod kSets: its copy-in waits
// until the copy-out of call k - kSets (the last user of that set) is done,
// the product waits for its copy-in, the copy-out for its product.  So the
// copy-in of call k + 1 and the copy-out of call k - 1 run while the product
// of call k runs, in both directions of the host link at once.  The product
// is sp_spmv itself, so the results are those of sp_spmv on the same inputs.
#include <algorithm>

#include "common.cuh"

using sp::DevBufPtr;

#ifndef SP_HOST_PLAN_SETS
#define SP_HOST_PLAN_SETS 3
#endif
constexpr int kSets = SP_HOST_PLAN_SETS;

struct sp_host_plan {
    const sp_mat *A = nullptr;
    int w = 0;
    sp_dtype xdt = SP_F64;
    size_t xs = 8;
    sp_dense *dx[kSets] = {}, *dy[kSets] = {}, *dz[kSets] = {};
    DevBufPtr ddot[kSets];
    cudaStream_t in = nullptr, comp = nullptr, out = nullptr;
    cudaEvent_t in_done[kSets] = {}, comp_done[kSets] = {}, out_done[kSets] = {};
    bool used[kSets] = {};
    int next = 0;
};

static void plan_free(sp_host_plan *p) {
    if (!p) return;
    if (p->in) cudaStreamSynchronize(p->in);
    if (p->comp) cudaStreamSynchronize(p->comp);
    if (p->out) cudaStreamSynchronize(p->out);
    for (int b = 0; b < kSets; ++b) {
        if (p->dx[b]) sp_dense_destroy(p->dx[b], nullptr);
        if (p->dy[b]) sp_dense_destroy(p->dy[b], nullptr);
        if (p->dz[b]) sp_dense_destroy(p->dz[b], nullptr);
        if (p->in_done[b]) cudaEventDestroy(p->in_done[b]);
        if (p->comp_done[b]) cudaEventDestroy(p->comp_done[b]);
        if (p->out_done[b]) cudaEventDestroy(p->out_done[b]);
    }
    if (p->in) cudaStreamDestroy(p->in);
    if (p->comp) cudaStreamDestroy(p->comp);
    if (p->out) cudaStreamDestroy(p->out);
    delete p;
}

int sp_host_plan_create(sp_host_plan **out, const sp_mat *A, int32_t w, sp_dtype vec_dtype) {
    if (!out || !A) return SP_ERR_ARG;
    *out = nullptr;
    if (w < 1) return SP_ERR_ARG;
    if (vec_dtype != SP_F64 && vec_dtype != SP_F32) return SP_ERR_DTYPE;
    if (A->vdt == SP_F64 && vec_dtype != SP_F64) return SP_ERR_DTYPE;
    const sp::Pattern &P = *A->pat;
    sp_host_plan *p = new sp_host_plan();
    p->A = A;
    p->w = w;
    p->xdt = vec_dtype;
    p->xs = vec_dtype == SP_F64 ? 8 : 4;
    int rc = SP_OK;
    for (int b = 0; b < kSets && rc == SP_OK; ++b) {
        rc = sp_dense_create(&p->dx[b], P.ncols, w, vec_dtype, SP_ROW_MAJOR, nullptr);
        if (rc == SP_OK) rc = sp_dense_create(&p->dy[b], P.nrows, w, vec_dtype, SP_ROW_MAJOR, nullptr);
        if (rc == SP_OK) rc = sp_dense_create(&p->dz[b], P.nrows, w, vec_dtype, SP_ROW_MAJOR, nullptr);
        if (rc == SP_OK) rc = sp::dev_alloc(p->ddot[b], 3 * (size_t)w * sizeof(double), nullptr);
    }
    cudaError_t e = cudaSuccess;
    if (rc == SP_OK) e = cudaStreamCreateWithFlags(&p->in, cudaStreamNonBlocking);
    if (rc == SP_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->comp, cudaStreamNonBlocking);
    if (rc == SP_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->out, cudaStreamNonBlocking);
    for (int b = 0; b < kSets && rc == SP_OK && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&p->in_done[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->comp_done[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->out_done[b], cudaEventDisableTiming);
    }
    if (rc == SP_OK && e == cudaSuccess) e = cudaDeviceSynchronize();
    if (rc == SP_OK && e != cudaSuccess) {
        sp_internal_note_cuda_error(e, "host plan create", __FILE__, __LINE__);
        rc = SP_ERR_CUDA;
    }
    if (rc != SP_OK) {
        plan_free(p);
        return rc;
    }
    *out = p;
    return SP_OK;
}

int sp_spmv_host(sp_host_plan *p, const void *x, const void *y_in, void *y_out, const void *z_in, void *z_out,
                 double *dot, const sp_spmv_opts *opts) {
    static const sp_spmv_opts defaults = SP_SPMV_OPTS_INIT;
    if (!p || !x || !y_out) return SP_ERR_ARG;
    const sp_spmv_opts &o = opts ? *opts : defaults;
    const uint32_t f = o.flags & ~SP_SPMV_DOT_HOST;
    const bool axpby = f & SP_SPMV_AXPBY, chain = f & SP_SPMV_CHAIN_AXPBY, dots = f & SP_SPMV_DOT_ANY;
    if (axpby && !y_in) return SP_ERR_ARG;
    if (chain && (!z_in || !z_out)) return SP_ERR_ARG;
    if (dots && !dot) return SP_ERR_ARG;
    const sp::Pattern &P = *p->A->pat;
    const size_t xbytes = (size_t)P.ncols * p->w * p->xs, ybytes = (size_t)P.nrows * p->w * p->xs;
    const int b = p->next;
    p->next = (p->next + 1) % kSets;
    int rc = SP_OK;
    // copy-in (after the copy-out of the last call that used this buffer set)
    if (p->used[b]) SP_CUDA(cudaStreamWaitEvent(p->in, p->out_done[b], 0));
    SP_CUDA(cudaMemcpyAsync(p->dx[b]->ptr, x, xbytes, cudaMemcpyHostToDevice, p->in));
    if (axpby) SP_CUDA(cudaMemcpyAsync(p->dy[b]->ptr, y_in, ybytes, cudaMemcpyHostToDevice, p->in));
    if (chain) SP_CUDA(cudaMemcpyAsync(p->dz[b]->ptr, z_in, ybytes, cudaMemcpyHostToDevice, p->in));
    SP_CUDA(cudaEventRecord(p->in_done[b], p->in));
    // the product, exactly sp_spmv's
    SP_CUDA(cudaStreamWaitEvent(p->comp, p->in_done[b], 0));
    sp_spmv_opts o2 = o;
    o2.flags = f;
    o2.z = chain ? p->dz[b] : nullptr;
    o2.dot = dots ? (double *)p->ddot[b]->ptr : nullptr;
    rc = sp_spmv(p->dy[b], p->A, p->dx[b], &o2, p->comp);
    if (rc != SP_OK) return rc;
    SP_CUDA(cudaEventRecord(p->comp_done[b], p->comp));
    // copy-out of y, z and the requested dot products
    SP_CUDA(cudaStreamWaitEvent(p->out, p->comp_done[b], 0));
    SP_CUDA(cudaMemcpyAsync(y_out, p->dy[b]->ptr, ybytes, cudaMemcpyDeviceToHost, p->out));
    if (chain) SP_CUDA(cudaMemcpyAsync(z_out, p->dz[b]->ptr, ybytes, cudaMemcpyDeviceToHost, p->out));
    for (int q = 0; q < 3; ++q)
        if (f & (SP_SPMV_DOT_YY << q))
            SP_CUDA(cudaMemcpyAsync(dot + (size_t)q * p->w, (const double *)p->ddot[b]->ptr + (size_t)q * p->w,
                                    p->w * sizeof(double), cudaMemcpyDeviceToHost, p->out));
    SP_CUDA(cudaEventRecord(p->out_done[b], p->out));
    p->used[b] = true;
    return SP_OK;
}

int sp_host_plan_sync(sp_host_plan *p) {
    if (!p) return SP_ERR_ARG;
    SP_CUDA(cudaStreamSynchronize(p->in));
    SP_CUDA(cudaStreamSynchronize(p->comp));
    SP_CUDA(cudaStreamSynchronize(p->out));
    return SP_OK;
}

int sp_host_plan_destroy(sp_host_plan *p) {
    if (!p) return SP_ERR_ARG;
    plan_free(p);
    return SP_OK;
}
