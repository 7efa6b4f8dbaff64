// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <vector>

#include "../../include/sellcs.h"

#define SP_TRY(expr)                      \
    do {                                  \
        int _e = (expr);                  \
        if (_e != SP_OK) return _e;       \
    } while (0)

#define SP_CUDA(expr)                                                     \
    do {                                                                  \
        cudaError_t _c = (expr);                                          \
        if (_c != cudaSuccess) {                                          \
            sp_internal_note_cuda_error(_c, #expr, __FILE__, __LINE__);   \
            return _c == cudaErrorMemoryAllocation ? SP_ERR_OOM : SP_ERR_CUDA; \
        }                                                                 \
    } while (0)

void sp_internal_note_cuda_error(cudaError_t e, const char *what, const char *file, int line);
// Records "prefix: why" as the calling thread's sp_last_error_detail().
void sp_internal_set_detail(const char *prefix, const char *why);

namespace sp {

// ------------------------------------------------------------------ device buffers

// Stream-ordered device allocation owned by a shared_ptr so that patterns can
// be shared between a matrix and its value clones.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    ~DevBuf();
};
using DevBufPtr = std::shared_ptr<DevBuf>;
int dev_alloc(DevBufPtr &out, size_t bytes, cudaStream_t s);

// Temporary device buffer (stream-ordered allocation, freed on the stream).
// The device's default memory pool keeps what stream-ordered temporaries
// free (release threshold: unlimited) instead of returning it at every
// synchronisation, so the next call's temporaries need no new mapping.
// Set once per device (knob SP_POOL_KEEP).
#ifndef SP_POOL_KEEP
#define SP_POOL_KEEP 1
#endif
void pool_keep_memory();

struct Tmp {
    void *p = nullptr;
    cudaStream_t s;
    explicit Tmp(cudaStream_t st) : s(st) {}
    int alloc(size_t bytes) {
        if (!bytes) bytes = 16;
        if (SP_POOL_KEEP) pool_keep_memory();
        cudaError_t e = cudaMallocAsync(&p, bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return e == cudaErrorMemoryAllocation ? SP_ERR_OOM : SP_ERR_CUDA;
        }
        return SP_OK;
    }
    ~Tmp() {
        if (p) cudaFreeAsync(p, s);
    }
    template <class T>
    T *as() const { return (T *)p; }
};

// SELL-C-sigma pattern: everything except the values.
struct Pattern {
    int64_t nrows = 0, ncols = 0, nnz = 0;
    int64_t nchunks = 0, nslots = 0, nstored = 0;
    int32_t C = 1;
    int64_t sigma = 1;
    int32_t maxrowlen = 0;
    DevBufPtr chunkptr;  // int64[nchunks+1]
    DevBufPtr chunklen;  // int32[nchunks]
    DevBufPtr slotlen;   // int32[nslots]
    DevBufPtr perm;      // int32[nslots], -1 for padding rows
    DevBufPtr col;       // int32[nstored]
    DevBufPtr rowptr;    // int64[nrows+1], the CSR row pointers (original order)
    // for the transpose only: position in the parent's CSR of each of its own CSR entries
    DevBufPtr src_index; // int64[nnz]
    // Static work partition of the persistent kernels: for a grid of
    // SMs * b blocks (b = 1..kMaxOcc) of kPartWarps warps, warp t owns the
    // 32-slot blocks [bounds[off[b] + t], bounds[off[b] + t + 1]), chosen so
    // that every warp gets the same share of (stored entries + 2 per row).
    DevBufPtr bounds;    // int32
    int64_t bounds_off[9] = {0};
    int32_t bounds_sms = 0;
    // Moving-front schedule (same grids): round r, warp t of the grid takes the
    // 32-slot block sched[off[b] + r * warps + t] (-1: none).  In each round the
    // blocks of the grid cover the next run of adjacent 32-slot blocks, each CTA
    // a contiguous piece of it, assigned to the CTA's warps longest first to the
    // least loaded so far.
    DevBufPtr sched;     // int32
    int64_t sched_off[9] = {0};
    int32_t sched_rounds[9] = {0};
    // spread of the row lengths inside 32-slot blocks: sum over blocks of
    // (longest - shortest real row) / sum of the longest
    double lane_spread = 0.0;
    int order = 0;  // work order of the product: 0 by the size of x, 1 moving front, 2 contiguous ranges
    // vectors in SELL row order: column indices stored as slots (col' = slot of
    // row col), so the products read x and write y at the slot index
    bool permuted_space = false;
};
using PatternPtr = std::shared_ptr<Pattern>;

}  // namespace sp

struct sp_mat {
    sp::PatternPtr pat;
    sp_dtype vdt = SP_F64;
    sp::DevBufPtr val;           // vdt[nstored]
    sp_mat *transpose = nullptr; // owned
    // reduction scratch for the fused dot products (per-block partials + ticket)
    sp::DevBufPtr scratch;
    size_t scratch_bytes = 0;
};

struct sp_dense {
    void *ptr = nullptr;
    int64_t nrows = 0;
    int32_t ncols = 0;
    int64_t ld = 0;
    sp_dtype dtype = SP_F64;
    sp_layout layout = SP_ROW_MAJOR;
    sp::DevBufPtr owner;  // set when the library allocated the memory
    // scattered view: column c of the view is column cols[c] of the block at
    // ptr (null for a compact block or view)
    std::shared_ptr<const std::vector<int32_t>> cols;
};

namespace sp {

inline size_t dtype_size(sp_dtype t) { return t == SP_F64 ? 8 : (t == SP_F32 ? 4 : 2); }

// Scattered views are accepted by sp_spmv (through compact clones) and by the
// dense copy calls; the other entry points refuse them.
inline bool dense_scattered(const sp_dense *d) { return d && d->cols; }
inline int scattered_refused(const char *who) {
    sp_internal_set_detail(who, "a scattered view is not accepted here: make a compact clone (sp_dense_clone)");
    return SP_ERR_ARG;
}

inline int ilog2_exact(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return (int64_t(1) << l) == v ? l : -1;
}

// ------------------------------------------------------------------ conversion entry points
int build_pattern_and_values(sp_mat *A, int64_t nrows, int64_t ncols, const int64_t *d_rowptr,
                             const int32_t *d_col, const void *d_val, bool val_f32, int C,
                             int64_t sigma, cudaStream_t s, bool permuted = false);
int build_transpose(sp_mat *A, const int64_t *d_rowptr, const int32_t *d_col, const void *d_val,
                    bool val_f32, cudaStream_t s);
int fill_values_from_csr(const Pattern &P, sp_dtype vdt, void *val_sell, const void *d_val_csr,
                         bool val_f32, cudaStream_t s);
int gather_values(const void *src, bool src_f32, const int64_t *index, int64_t n, void *dst,
                  bool dst_f32, cudaStream_t s);
int convert_values(const void *src, sp_dtype sdt, void *dst, sp_dtype ddt, int64_t n, cudaStream_t s);
int widen_values(const void *src, sp_dtype sdt, double *dst, int64_t n, cudaStream_t s);


// ------------------------------------------------------------------ SpMMV launch
struct VecDesc {
    const void *ptr;
    int64_t rs, cs;  // element strides: (i,k) at ptr[i*rs + k*cs]
};

struct SpmvLaunch {
    const Pattern *P;
    const void *val;
    sp_dtype vdt, xdt;
    int w;
    VecDesc x, y, z;
    uint32_t flags;
    double alpha, beta, delta, eta;
    const double *gamma;  // host, w values (already expanded) or null
    double *dot;          // device, written at dot[q*dot_stride + dot_off + k]
    int dot_stride, dot_off;
    double *partials;     // device scratch
    unsigned *ticket;     // device scratch (zero between calls)
    int max_blocks;
};
int launch_spmv(const SpmvLaunch &L, cudaStream_t s);
int spmv_scratch_need(int sm_count, size_t *bytes, int *max_blocks);

int launch_sampled(const Pattern &P, sp_dtype xdt, int w, const void *x, const void *g, void *dvals,
                   cudaStream_t s);

int device_sm_count(int *n);
size_t device_l2_bytes();
int build_partition(Pattern &P, cudaStream_t s);
constexpr int kPartWarps = 8;  // warps per block of the partitioned kernels
constexpr int kSchedCtaWarps = 32;  // warps per CTA the front schedule is built for
constexpr int kSchedResidentCtas = 1;  // resident CTAs per SM the front schedule is built for
constexpr int kMaxOcc = 8;     // resident blocks per SM covered by the partition table
// Partition table for a grid of `warps` resident warps, or null when that is
// not kPartWarps * b * SMs for b <= kMaxOcc (then the kernels fall back to a
// block-strided loop).
inline const int32_t *partition_for(const Pattern &P, int64_t warps) {
    int64_t unit = (int64_t)kPartWarps * P.bounds_sms;
    if (!P.bounds || P.bounds_sms <= 0 || warps % unit) return nullptr;
    int64_t b = warps / unit;
    if (b < 1 || b > kMaxOcc) return nullptr;
    return (const int32_t *)P.bounds->ptr + P.bounds_off[b];
}
// Front schedule for a grid of `warps` resident warps in CTAs of kSchedCtaWarps, or null.
inline const int32_t *schedule_for(const Pattern &P, int64_t warps, int *rounds) {
    int64_t unit = (int64_t)kPartWarps * P.bounds_sms;
    if (!P.sched || P.bounds_sms <= 0 || warps % unit) return nullptr;
    int64_t b = warps / unit;
    if (b < 1 || b > kMaxOcc || P.sched_rounds[b] <= 0) return nullptr;
    *rounds = P.sched_rounds[b];
    return (const int32_t *)P.sched->ptr + P.sched_off[b];
}

}  // namespace sp
