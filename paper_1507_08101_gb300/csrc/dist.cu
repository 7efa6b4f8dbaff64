// Row-partitioned product (GHOST, Sec. "Data parallelism" and "Heterogeneous
// execution"): the matrix is split row-wise into contiguous blocks, one per
// process, weighted by rows or nonzeros and by a per-process share; each
// process keeps its rows with the columns split into a local part (columns it
// owns) and a remote part whose column indices are compressed into a halo
// numbered after the local rows (the figure of the row-wise distribution,
// steps 1-3).  The remote x entries arrive in that halo; the product then
// runs as two passes so that the local pass overlaps the halo exchange (the
// task-mode SpMV of Sec. "Resource management", on CUDA streams).
//
// Everything here except sp_dist_pack and sp_dist_spmv is host code: the
// plans can be built and checked without a GPU.
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

struct sp_dist_plan {
    int64_t nglobal = 0;
    int nranks = 0, rank = 0;
    std::vector<int64_t> bounds;    // nranks + 1
    int64_t r0 = 0, nloc = 0;       // own rows [r0, r0 + nloc)
    std::vector<int64_t> rowptr;    // nloc + 1 (the caller's rows)
    std::vector<int32_t> newcol;    // per entry: local column in [0, nloc + nhalo)
    std::vector<int64_t> halo;      // global index of each halo entry, ascending
    std::vector<int64_t> recv_counts;  // per rank: halo entries it owns
    int64_t nnz_loc = 0, nnz_rem = 0;
    bool sends_set = false;
    std::vector<int64_t> send_counts;  // per rank: rows sent to it
    std::vector<int32_t> send_local;   // local row of each sent row, by destination rank
    int32_t *d_send = nullptr;         // device copy of send_local (uploaded by the first pack)
    int dev = -1;
};

namespace {

int fail(const char *why) {
    sp_internal_set_detail("sp_dist", why);
    return SP_ERR_ARG;
}

}  // namespace

int sp_dist_partition(int64_t nrows, const int64_t *rowptr, int nparts, const double *share, int by_nnz,
                      int64_t *bounds) {
    if (nrows < 0 || nparts < 1 || !bounds || (by_nnz && !rowptr)) return SP_ERR_ARG;
    std::vector<double> cum(nparts + 1, 0.0);
    for (int p = 0; p < nparts; ++p) {
        const double s = share ? share[p] : 1.0;
        if (!(s >= 0.0) || s > 1e300) return fail("shares must be finite and >= 0");
        cum[p + 1] = cum[p] + s;
    }
    if (!(cum[nparts] > 0.0)) return fail("at least one share must be positive");
    // work done by rows [0, r): r, or the nonzeros of those rows
    auto work = [&](int64_t r) -> double { return by_nnz ? (double)rowptr[r] : (double)r; };
    if (by_nnz) {
        if (rowptr[0] != 0) return SP_ERR_FORMAT;
        for (int64_t r = 0; r < nrows; ++r)
            if (rowptr[r + 1] < rowptr[r]) return SP_ERR_FORMAT;
    }
    const double total = work(nrows);
    bounds[0] = 0;
    for (int p = 1; p < nparts; ++p) {
        const double target = total * (cum[p] / cum[nparts]);
        // first row boundary whose work reaches the target, then the nearer of
        // it and the boundary before it
        int64_t lo = bounds[p - 1], hi = nrows;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (work(mid) < target) lo = mid + 1;
            else hi = mid;
        }
        int64_t b = lo;
        if (b > bounds[p - 1] && target - work(b - 1) < work(b) - target) --b;
        bounds[p] = b;
    }
    bounds[nparts] = nrows;
    return SP_OK;
}

int sp_dist_plan_create(sp_dist_plan **out, int64_t nglobal, int nranks, const int64_t *bounds, int rank,
                        const int64_t *rowptr, const int64_t *gcol) {
    if (!out || !bounds || !rowptr || nranks < 1 || rank < 0 || rank >= nranks || nglobal < 0) return SP_ERR_ARG;
    *out = nullptr;
    if (bounds[0] != 0 || bounds[nranks] != nglobal) return SP_ERR_DIM;
    for (int q = 0; q < nranks; ++q)
        if (bounds[q + 1] < bounds[q]) return SP_ERR_DIM;
    const int64_t r0 = bounds[rank], nloc = bounds[rank + 1] - r0;
    if (rowptr[0] != 0) return SP_ERR_FORMAT;
    for (int64_t r = 0; r < nloc; ++r)
        if (rowptr[r + 1] < rowptr[r]) return SP_ERR_FORMAT;
    const int64_t nnz = rowptr[nloc];
    if (nnz > 0 && !gcol) return SP_ERR_ARG;
    for (int64_t e = 0; e < nnz; ++e)
        if (gcol[e] < 0 || gcol[e] >= nglobal) return SP_ERR_FORMAT;

    sp_dist_plan *p = new sp_dist_plan;
    p->nglobal = nglobal;
    p->nranks = nranks;
    p->rank = rank;
    p->bounds.assign(bounds, bounds + nranks + 1);
    p->r0 = r0;
    p->nloc = nloc;
    p->rowptr.assign(rowptr, rowptr + nloc + 1);
    // remote columns, compressed: the distinct ones in ascending global order
    for (int64_t e = 0; e < nnz; ++e)
        if (gcol[e] < r0 || gcol[e] >= r0 + nloc) p->halo.push_back(gcol[e]);
    std::sort(p->halo.begin(), p->halo.end());
    p->halo.erase(std::unique(p->halo.begin(), p->halo.end()), p->halo.end());
    const int64_t nhalo = (int64_t)p->halo.size();
    if (nloc + nhalo >= (1LL << 31)) {
        delete p;
        sp_internal_set_detail("sp_dist_plan_create", "local rows + halo exceed 32-bit local indices");
        return SP_ERR_DIM;
    }
    p->newcol.resize(nnz);
    for (int64_t e = 0; e < nnz; ++e) {
        const int64_t c = gcol[e];
        if (c >= r0 && c < r0 + nloc) {
            p->newcol[e] = (int32_t)(c - r0);
            ++p->nnz_loc;
        } else {
            const int64_t h = std::lower_bound(p->halo.begin(), p->halo.end(), c) - p->halo.begin();
            p->newcol[e] = (int32_t)(nloc + h);
            ++p->nnz_rem;
        }
    }
    // ranks own contiguous, ascending row ranges, so the sorted halo is
    // grouped by owner in rank order
    p->recv_counts.assign(nranks, 0);
    for (int q = 0; q < nranks; ++q) {
        auto a = std::lower_bound(p->halo.begin(), p->halo.end(), bounds[q]);
        auto b = std::lower_bound(p->halo.begin(), p->halo.end(), bounds[q + 1]);
        p->recv_counts[q] = (int64_t)(b - a);
    }
    *out = p;
    return SP_OK;
}

int sp_dist_plan_info(const sp_dist_plan *p, int64_t *nloc, int64_t *nhalo, int64_t *nnz_local,
                      int64_t *nnz_remote, int64_t *nsend) {
    if (!p) return SP_ERR_ARG;
    if (nloc) *nloc = p->nloc;
    if (nhalo) *nhalo = (int64_t)p->halo.size();
    if (nnz_local) *nnz_local = p->nnz_loc;
    if (nnz_remote) *nnz_remote = p->nnz_rem;
    if (nsend) *nsend = p->sends_set ? (int64_t)p->send_local.size() : -1;
    return SP_OK;
}

int sp_dist_plan_halo(const sp_dist_plan *p, int64_t *halo_gidx, int64_t *recv_counts) {
    if (!p) return SP_ERR_ARG;
    if (halo_gidx && !p->halo.empty()) std::copy(p->halo.begin(), p->halo.end(), halo_gidx);
    if (recv_counts) std::copy(p->recv_counts.begin(), p->recv_counts.end(), recv_counts);
    return SP_OK;
}

int sp_dist_plan_columns(const sp_dist_plan *p, int32_t *col_ext) {
    if (!p || (!col_ext && !p->newcol.empty())) return SP_ERR_ARG;
    std::copy(p->newcol.begin(), p->newcol.end(), col_ext);
    return SP_OK;
}

int sp_dist_plan_split(const sp_dist_plan *p, const double *val, int64_t *rowptr_loc, int32_t *col_loc,
                       double *val_loc, int64_t *rowptr_rem, int32_t *col_rem, double *val_rem) {
    if (!p || !rowptr_loc || !rowptr_rem) return SP_ERR_ARG;
    const int64_t nnz = p->rowptr[p->nloc];
    if (nnz > 0 && !val) return SP_ERR_ARG;
    if ((p->nnz_loc > 0 && (!col_loc || !val_loc)) || (p->nnz_rem > 0 && (!col_rem || !val_rem)))
        return SP_ERR_ARG;
    int64_t nl = 0, nr = 0;
    rowptr_loc[0] = 0;
    rowptr_rem[0] = 0;
    for (int64_t r = 0; r < p->nloc; ++r) {
        for (int64_t e = p->rowptr[r]; e < p->rowptr[r + 1]; ++e) {
            const int32_t c = p->newcol[e];
            if (c < p->nloc) {
                col_loc[nl] = c;
                val_loc[nl++] = val[e];
            } else {
                col_rem[nr] = c;
                val_rem[nr++] = val[e];
            }
        }
        rowptr_loc[r + 1] = nl;
        rowptr_rem[r + 1] = nr;
    }
    return SP_OK;
}

int sp_dist_plan_set_sends(sp_dist_plan *p, const int64_t *send_counts, const int64_t *send_gidx) {
    if (!p || !send_counts) return SP_ERR_ARG;
    int64_t total = 0;
    for (int q = 0; q < p->nranks; ++q) {
        if (send_counts[q] < 0) return fail("negative send count");
        if (q == p->rank && send_counts[q] != 0) return fail("a rank sends nothing to itself");
        total += send_counts[q];
    }
    if (total > 0 && !send_gidx) return SP_ERR_ARG;
    std::vector<int32_t> loc(total);
    int64_t k = 0;
    for (int q = 0; q < p->nranks; ++q) {
        for (int64_t i = 0; i < send_counts[q]; ++i, ++k) {
            const int64_t g = send_gidx[k];
            if (g < p->r0 || g >= p->r0 + p->nloc) return fail("requested row is not owned by this rank");
            if (i > 0 && g <= send_gidx[k - 1]) return fail("each peer's request must be strictly ascending");
            loc[k] = (int32_t)(g - p->r0);
        }
    }
    p->send_counts.assign(send_counts, send_counts + p->nranks);
    p->send_local.swap(loc);
    p->sends_set = true;
    if (p->d_send) {  // a new list: the next pack uploads it again
        cudaFree(p->d_send);
        p->d_send = nullptr;
    }
    return SP_OK;
}

int sp_dist_plan_sends(const sp_dist_plan *p, int64_t *send_counts, int32_t *send_local) {
    if (!p || !p->sends_set) return SP_ERR_ARG;
    if (send_counts) std::copy(p->send_counts.begin(), p->send_counts.end(), send_counts);
    if (send_local && !p->send_local.empty()) std::copy(p->send_local.begin(), p->send_local.end(), send_local);
    return SP_OK;
}

int sp_dist_split_opts(const sp_spmv_opts *in, sp_spmv_opts *pass1, sp_spmv_opts *pass2) {
    static const sp_spmv_opts defaults = SP_SPMV_OPTS_INIT;
    if (!pass1 || !pass2) return SP_ERR_ARG;
    const sp_spmv_opts &o = in ? *in : defaults;
    const uint32_t f = o.flags;
    const uint32_t late = SP_SPMV_DOT_ANY | SP_SPMV_DOT_HOST | SP_SPMV_CHAIN_AXPBY;
    // pass 1 (local columns): the whole augmentation except what needs the
    // final y: y = alpha (A_loc x - gamma x) + beta y
    *pass1 = o;
    pass1->flags = f & ~late;
    pass1->z = nullptr;
    pass1->dot = nullptr;
    // pass 2 (halo columns): y = alpha A_rem x + 1 * y, then the dots of the
    // final y and the chain
    *pass2 = defaults;
    pass2->flags = SP_SPMV_AXPBY | (f & (SP_SPMV_SCALE | late));
    pass2->alpha = o.alpha;
    pass2->beta = 1.0;
    pass2->delta = o.delta;
    pass2->eta = o.eta;
    pass2->z = o.z;
    pass2->dot = o.dot;
    return SP_OK;
}

namespace sp {

template <class T>
__global__ void k_halo_pack(const int32_t *__restrict__ idx, int64_t nsend, int w, const T *__restrict__ x,
                            int64_t rs, int64_t cs, T *__restrict__ out) {
    const int64_t n = nsend * w;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / w;
        const int c = (int)(t - k * w);
        out[t] = x[(int64_t)idx[k] * rs + (int64_t)c * cs];
    }
}

}  // namespace sp

int sp_dist_pack(sp_dist_plan *p, const sp_dense *x, void *send_buf, void *stream) {
    if (sp::dense_scattered(x)) return sp::scattered_refused("sp_dist_pack");
    if (!p || !x || !p->sends_set) return SP_ERR_ARG;
    void *xp = nullptr;
    int64_t nrows = 0, ld = 0;
    int32_t w = 0;
    sp_dtype dt;
    sp_layout lay;
    SP_TRY(sp_dense_data(x, &xp, &nrows, &w, &ld, &dt, &lay));
    if (nrows < p->nloc) return SP_ERR_DIM;
    const int64_t nsend = (int64_t)p->send_local.size();
    if (nsend == 0 || w == 0) return SP_OK;
    if (!send_buf) return SP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    SP_CUDA(cudaGetDevice(&dev));
    if (p->d_send && p->dev != dev) return fail("plan used on a second device");
    if (!p->d_send) {
        SP_CUDA(cudaMalloc(&p->d_send, nsend * sizeof(int32_t)));
        p->dev = dev;
        SP_CUDA(cudaMemcpyAsync(p->d_send, p->send_local.data(), nsend * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        // the host vector must outlive the copy: keep the stream ordered here once
        SP_CUDA(cudaStreamSynchronize(s));
    }
    const int64_t rs = lay == SP_ROW_MAJOR ? ld : 1, cs = lay == SP_ROW_MAJOR ? 1 : ld;
    int sms = 1;
    SP_TRY(sp::device_sm_count(&sms));
    const int64_t n = nsend * w;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
    if (dt == SP_F64)
        sp::k_halo_pack<double><<<(unsigned)blocks, 256, 0, s>>>(p->d_send, nsend, w, (const double *)xp, rs, cs,
                                                                  (double *)send_buf);
    else if (dt == SP_F32)
        sp::k_halo_pack<float><<<(unsigned)blocks, 256, 0, s>>>(p->d_send, nsend, w, (const float *)xp, rs, cs,
                                                                 (float *)send_buf);
    else
        return SP_ERR_DTYPE;
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

int sp_dist_spmv(sp_dense *y, const sp_mat *A_loc, const sp_mat *A_rem, const sp_dense *x, const sp_spmv_opts *opts,
                 void *halo_ready, void *stream) {
    if (!y || !A_loc || !A_rem || !x) return SP_ERR_ARG;
    if (sp::dense_scattered(x) || sp::dense_scattered(y)) return sp::scattered_refused("sp_dist_spmv");
    sp_spmv_opts o1, o2;
    SP_TRY(sp_dist_split_opts(opts, &o1, &o2));
    // pass 1 reads only the first nloc rows of x (its own rows)
    void *xp = nullptr;
    int64_t nrows = 0, ld = 0, ylen = 0;
    int32_t w = 0;
    sp_dtype dt;
    sp_layout lay;
    SP_TRY(sp_dense_data(x, &xp, &nrows, &w, &ld, &dt, &lay));
    SP_TRY(sp_dense_data(y, nullptr, &ylen, nullptr, nullptr, nullptr, nullptr));
    if (lay != SP_ROW_MAJOR) return fail("the halo form needs a row-major x");
    if (nrows < ylen) return SP_ERR_DIM;
    sp_dense *xo = nullptr;
    SP_TRY(sp_dense_view(&xo, xp, ylen, w, ld, dt, lay));
    int rc = sp_spmv(y, A_loc, xo, &o1, stream);
    sp_dense_destroy(xo, nullptr);
    if (rc != SP_OK) return rc;
    if (halo_ready) SP_CUDA(cudaStreamWaitEvent((cudaStream_t)stream, (cudaEvent_t)halo_ready, 0));
    return sp_spmv(y, A_rem, x, &o2, stream);
}

int sp_dist_plan_destroy(sp_dist_plan *p) {
    if (!p) return SP_ERR_ARG;
    if (p->d_send) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != p->dev) cudaSetDevice(p->dev);
        cudaDeviceSynchronize();
        cudaFree(p->d_send);
        if (cur != p->dev) cudaSetDevice(cur);
    }
    delete p;
    return SP_OK;
}
