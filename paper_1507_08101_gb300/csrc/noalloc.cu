// sp_spmv_noalloc: the augmented SpMMV for callers that cannot allocate device
// memory.  Such callers exist: a process whose device memory is already held
// by another allocator (a framework's caching pool that reserved the GPU), or
// a code path where cudaMalloc / cudaFree are not allowed because they
// synchronise the device or would break a stream capture.
//
// This entry point takes every input and output as a plain device pointer
// (the SELL-C-sigma arrays, x, y, z, the dot results) and allocates nothing:
// the scratch of the fused dot products (per-block partial sums and the
// arrival ticket) lives in the file-scope device arrays below, which every GPU
// that loads this library holds until the process exits.  It runs the same
// kernel as sp_spmv.
#include <stdio.h>

#include <mutex>

#include "common.cuh"
#include "spmv_kernel.cuh"

namespace sp {
template <class VT, class XT>
int launch_spmv_typed(const SpmvArgs &a, bool vec, int max_blocks, cudaStream_t s);
}

using namespace sp;

// Partial sums: one double per (dot kind, column, block).
static constexpr int kNoAllocBlocks = SP_NOALLOC_MAX_BLOCKS;
static __device__ __align__(256) double g_noalloc_partials[3 * SP_NOALLOC_MAX_W * SP_NOALLOC_MAX_BLOCKS];
static __device__ __align__(256) unsigned g_noalloc_ticket[64];

namespace {
// Device addresses of the arrays above, looked up once per device under a
// mutex, so that two host threads making their first call on one device at
// the same time both see a complete pair.
struct NoAllocAddr {
    double *partials = nullptr;
    unsigned *ticket = nullptr;
};
NoAllocAddr g_addr[64];
std::mutex g_addr_mutex;

int noalloc_setup(NoAllocAddr *out) {
    int dev = 0;
    SP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SP_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    NoAllocAddr &a = g_addr[dev];
    if (!a.partials) {
        void *p = nullptr, *t = nullptr;
        SP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_partials));
        SP_CUDA(cudaGetSymbolAddress(&t, g_noalloc_ticket));
        a.ticket = (unsigned *)t;
        a.partials = (double *)p;
    }
    *out = a;
    return SP_OK;
}

// Record why a call was rejected (the thread's sp_last_error_detail) and return the code.
int noalloc_reject(int code, const char *why) {
    sp_internal_set_detail("sp_spmv_noalloc", why);
    return code;
}
}  // namespace

extern "C" int sp_spmv_noalloc(const void *val, sp_dtype val_dtype, const int32_t *col, const int64_t *chunkptr,
                               const int32_t *slotlen, const int32_t *perm, int64_t nrows, int64_t ncols,
                               int32_t C, const void *x, int64_t ldx, void *y, int64_t ldy, void *z, int64_t ldz,
                               int32_t w, sp_dtype vec_dtype, uint32_t flags, double alpha, double beta,
                               const double *gamma, double delta, double eta, double *dot, void *stream) {
    const uint32_t known = SP_SPMV_SCALE | SP_SPMV_SHIFT | SP_SPMV_VSHIFT | SP_SPMV_AXPBY | SP_SPMV_DOT_ANY |
                           SP_SPMV_CHAIN_AXPBY;
    if (flags & ~known) return noalloc_reject(SP_ERR_ARG, "unknown flag (SP_SPMV_DOT_HOST is not available here)");
    if (w < 0 || w > SP_NOALLOC_MAX_W)
        return noalloc_reject(SP_ERR_UNSUPPORTED, "block width above SP_NOALLOC_MAX_W (32)");
    if (nrows < 0 || ncols < 0 || nrows >= (1LL << 31) || ncols >= (1LL << 31) || C < 1 || C > 1024)
        return noalloc_reject(SP_ERR_DIM, "matrix shape or chunk height out of range");
    if (!(val_dtype == SP_F64 || val_dtype == SP_F32 || val_dtype == SP_BF16) ||
        !(vec_dtype == SP_F64 || vec_dtype == SP_F32) || (val_dtype == SP_F64 && vec_dtype != SP_F64))
        return noalloc_reject(SP_ERR_DTYPE, "unsupported value / vector precision pair");
    if ((flags & SP_SPMV_SHIFT) && (flags & SP_SPMV_VSHIFT))
        return noalloc_reject(SP_ERR_ARG, "SHIFT and VSHIFT are exclusive");
    const bool shift = flags & (SP_SPMV_SHIFT | SP_SPMV_VSHIFT);
    if (shift && !gamma) return noalloc_reject(SP_ERR_ARG, "shift requested without gamma");
    if ((shift || (flags & (SP_SPMV_DOT_XY | SP_SPMV_DOT_XX))) && nrows != ncols)
        return noalloc_reject(SP_ERR_DIM, "shift and <x,y>, <x,x> need a square matrix");
    if ((flags & SP_SPMV_DOT_ANY) && !dot) return noalloc_reject(SP_ERR_ARG, "dots requested without dot");
    if ((flags & SP_SPMV_CHAIN_AXPBY) && !z) return noalloc_reject(SP_ERR_ARG, "chain requested without z");
    if (ldx < w || ldy < w || ((flags & SP_SPMV_CHAIN_AXPBY) && ldz < w))
        return noalloc_reject(SP_ERR_DIM, "leading dimension smaller than the block width");
    if (w == 0) return SP_OK;
    if (nrows > 0 && (!val || !col || !chunkptr || !slotlen || !x || !y))
        return noalloc_reject(SP_ERR_ARG, "null matrix or vector pointer");

    NoAllocAddr na;
    SP_TRY(noalloc_setup(&na));
    cudaStream_t s = (cudaStream_t)stream;
    // the ticket and the dynamic-order counters (words 0..2) must start at
    // zero; a call that did not finish could have left them set
    SP_CUDA(cudaMemsetAsync(na.ticket, 0, 3 * sizeof(unsigned), s));

    const int64_t nchunks = (nrows + C - 1) / C;
    SpmvArgs a{};
    a.val = val;
    a.col = col;
    a.chunkptr = chunkptr;
    a.chunklen = nullptr;  // chunk lengths are not among this entry point's arguments
    a.slotlen = slotlen;
    a.perm = perm;
    a.nrows = nrows;
    a.nslots = nchunks * C;
    a.C = C;
    a.w = w;
    a.x = x;
    a.xrs = ldx;
    a.xcs = 1;
    a.y = y;
    a.yrs = ldy;
    a.ycs = 1;
    a.z = z;
    a.zrs = ldz;
    a.zcs = 1;
    a.flags = flags;
    a.alpha = alpha;
    a.beta = beta;
    a.delta = delta;
    a.eta = eta;
    a.dot = dot;
    a.dot_stride = w;
    a.dot_off = 0;
    a.partials = na.partials;
    a.ticket = na.ticket;
    a.sched = nullptr;
    a.sched_rounds = 0;
    a.wbounds = nullptr;
    a.wbounds_src = nullptr;
    a.nsm = 0;
    for (int k = 0; k < kMaxTileW; ++k)
        a.gamma[k] = (k < w && (flags & SP_SPMV_VSHIFT)) ? gamma[k] : ((flags & SP_SPMV_SHIFT) ? gamma[0] : 0.0);
    // the grid may not need more partials than the array holds
    const int max_blocks = kNoAllocBlocks;
    const size_t xs = vec_dtype == SP_F64 ? 8 : 4;
    const int cpl = host_cols_per_lane(xs, w);
    const size_t align = cpl * xs < 16 ? cpl * xs : 16;
    auto ok = [&](const void *p, int64_t ld) { return ((uintptr_t)p % align == 0) && ((ld * xs) % align == 0); };
    const bool vec = (w % cpl == 0) && ok(x, ldx) && ok(y, ldy) && (!(flags & SP_SPMV_CHAIN_AXPBY) || ok(z, ldz));
    if (val_dtype == SP_F64) return launch_spmv_typed<double, double>(a, vec, max_blocks, s);
    if (val_dtype == SP_F32 && vec_dtype == SP_F64) return launch_spmv_typed<float, double>(a, vec, max_blocks, s);
    if (val_dtype == SP_F32) return launch_spmv_typed<float, float>(a, vec, max_blocks, s);
    if (vec_dtype == SP_F64) return launch_spmv_typed<__nv_bfloat16, double>(a, vec, max_blocks, s);
    return launch_spmv_typed<__nv_bfloat16, float>(a, vec, max_blocks, s);
}
