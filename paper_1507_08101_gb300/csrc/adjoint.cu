// Sampled product over the SELL pattern: the derivative of L(y), y = A x,
// with respect to the stored values,
//
//     dvals[p] = sum_k g[row(p), k] * x[col(p), k]      for every nonzero p,
//
// written in the caller's CSR order (entry j of row i is CSR position
// rowptr[i] + j, because a SELL row keeps the order of its CSR row).
//
// Same lane mapping as the SpMMV kernel: G lanes share one row and own CPL
// columns each; the row's g values stay in registers while its column
// indices stream past, the G partial products are combined by xor shuffles
// inside the row's lane group, and the group's first lane writes the result.
#include <algorithm>

#include "spmv_kernel.cuh"

namespace sp {

struct SampledArgs {
    const int32_t *col;
    const int64_t *chunkptr;
    const int32_t *slotlen;
    const int32_t *perm;
    const int64_t *rowptr;
    int64_t nrows, nslots;
    int32_t C, w;
    int32_t log2_tpr;  // threads per row (lanes splitting a row's entries)
    const int32_t *wbounds;  // partition of this grid into warp ranges (null: block-strided)
    const Pattern *pat;      // host side only: where the launcher finds the partition
    const void *x;  // ncols x w row-major (ld = w)
    const void *g;  // nrows x w row-major (ld = w)
    void *dvals;
};

template <class XT, int WP, bool VEC>
__global__ void __launch_bounds__(kSpmvThreads) k_sampled(const __grid_constant__ SampledArgs a) {
    constexpr int CPL = cols_per_lane<XT, WP>();
    constexpr int G = WP / CPL;
    constexpr int R = 32 / G;
    constexpr int U = CPL >= 4 ? 4 : 8 / CPL;  // column indices and x rows in flight per lane
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lt = a.log2_tpr;
    const int T = 1 << lt;
    const int gl = lane % G;
    const int tt = (lane / G) & (T - 1);
    const int rw = (lane / G) >> lt;
    const int Rr = R >> lt;
    const int k0 = gl * CPL;
    const int nvalid = a.w - k0 < CPL ? a.w - k0 : CPL;
    const XT *__restrict__ x = (const XT *)a.x + k0;
    const XT *__restrict__ g = (const XT *)a.g + k0;
    XT *__restrict__ out = (XT *)a.dvals;
    // one slot (s < 0 or beyond the matrix: no row); every lane of the warp
    // calls it the same number of times, so the shuffles see the full warp
    auto slot = [&](int64_t s) {
        int64_t i = -1;
        int len = 0;
        int64_t off = 0;
        if (s >= 0 && s < a.nslots) {
            i = a.perm ? (int64_t)a.perm[s] : (s < a.nrows ? s : -1);
            if (i >= 0) {
                uint32_t cidx = (uint32_t)s / (uint32_t)a.C;
                off = a.chunkptr[cidx] + ((uint32_t)s - cidx * (uint32_t)a.C);
                len = a.slotlen[s];
            }
        }
        XT gv[CPL];
        if (i >= 0 && nvalid > 0) load_cols<XT, CPL, VEC>(g + i * a.w, 1, nvalid, gv);
        else {
#pragma unroll
            for (int c = 0; c < CPL; ++c) gv[c] = XT(0);
        }
        const int64_t dst = i >= 0 ? a.rowptr[i] : 0;
        // this lane's entries of the row: j = tt, tt + T, ...
        const int len_t = len > tt ? (len - tt + T - 1) >> lt : 0;
        int maxlen = len_t;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) maxlen = max(maxlen, __shfl_xor_sync(0xffffffffu, maxlen, o));
        const int32_t *cp = a.col + off + (int64_t)tt * a.C;
        const int64_t step = (int64_t)a.C << lt;
        for (int q = 0; q < maxlen; q += U) {
            int32_t cc[U];
#pragma unroll
            for (int u = 0; u < U; ++u) cc[u] = (q + u < len_t && nvalid > 0) ? ld_stream(cp + (q + u) * step) : 0;
            XT sum[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                sum[u] = XT(0);
                if (q + u < len_t && nvalid > 0) {
                    XT xv[CPL];
                    load_cols<XT, CPL, VEC>(x + (int64_t)cc[u] * a.w, 1, nvalid, xv);
#pragma unroll
                    for (int c = 0; c < CPL; ++c) sum[u] = fma(gv[c], xv[c], sum[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int o = 1; o < G; o <<= 1) sum[u] += __shfl_xor_sync(0xffffffffu, sum[u], o);
                if (gl == 0 && q + u < len_t) out[dst + tt + (int64_t)(q + u) * T] = sum[u];
            }
        }
    };
    if (a.wbounds) {
        // the cost-balanced partition of the product kernels: a contiguous
        // range of 32-slot blocks per warp
        const int gw = blockIdx.x * kSpmvWarps + warp;
        const int64_t s0 = (int64_t)a.wbounds[gw] * 32;
        const int64_t s1e = (int64_t)a.wbounds[gw + 1] * 32;
        const int64_t s1 = s1e < a.nslots ? s1e : a.nslots;
        for (int64_t base = s0; base < s1; base += Rr) slot(base + rw < s1 ? base + rw : -1);
    } else {
        const int rows = Rr * kSpmvWarps;
        for (int64_t base = (int64_t)blockIdx.x * rows; base < a.nslots; base += (int64_t)gridDim.x * rows)
            slot(base + warp * Rr + rw);
    }
}

template <class XT, int WP, bool VEC>
static int launch_sampled_variant(const SampledArgs &a, cudaStream_t s) {
    constexpr int CPL = cols_per_lane<XT, WP>();
    constexpr int G = WP / CPL;
    constexpr int ROWS = (32 / G) * kSpmvWarps;
    SampledArgs b = a;
    b.log2_tpr = host_log2_tpr(a.C, G);
    static int occ = 0;
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sampled<XT, WP, VEC>, kSpmvThreads, 0) !=
                cudaSuccess || occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
    }
    int sms = 1;
    SP_TRY(device_sm_count(&sms));
    int64_t need = ((a.nslots << b.log2_tpr) + ROWS - 1) / ROWS;
    int64_t grid = (int64_t)sms * occ;
    // with a partition table the whole grid runs and each warp takes its range
    b.wbounds = a.pat ? partition_for(*a.pat, grid * kSpmvWarps) : nullptr;
    if (!b.wbounds && grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_sampled<XT, WP, VEC><<<(unsigned)grid, kSpmvThreads, 0, s>>>(b);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

template <class XT>
static int launch_sampled_typed(const SampledArgs &a, bool vec, cudaStream_t s) {
#define SP_SAMPLED_W(WPV)                                                                  \
    if (a.w <= WPV)                                                                        \
        return vec ? launch_sampled_variant<XT, WPV, true>(a, s)                           \
                   : launch_sampled_variant<XT, WPV, false>(a, s);
    SP_SAMPLED_W(1)
    SP_SAMPLED_W(2)
    SP_SAMPLED_W(4)
    SP_SAMPLED_W(8)
    SP_SAMPLED_W(16)
    SP_SAMPLED_W(32)
#undef SP_SAMPLED_W
    return SP_ERR_UNSUPPORTED;
}

int launch_sampled(const Pattern &P, sp_dtype xdt, int w, const void *x, const void *g, void *dvals,
                   cudaStream_t s) {
    if (w < 1 || w > kMaxTileW) return SP_ERR_UNSUPPORTED;
    SampledArgs a{};
    a.pat = &P;
    a.col = (const int32_t *)P.col->ptr;
    a.chunkptr = (const int64_t *)P.chunkptr->ptr;
    a.slotlen = (const int32_t *)P.slotlen->ptr;
    a.perm = P.sigma == 1 ? nullptr : (const int32_t *)P.perm->ptr;
    a.rowptr = (const int64_t *)P.rowptr->ptr;
    a.nrows = P.nrows;
    a.nslots = P.nslots;
    a.C = P.C;
    a.w = w;
    a.x = x;
    a.g = g;
    a.dvals = dvals;
    size_t xs = xdt == SP_F64 ? 8 : 4;
    int cpl = host_cols_per_lane(xs, w);
    int align = (int)std::min<size_t>(16, cpl * xs);
    bool vec = (w % cpl == 0) && ((w * xs) % align == 0) && ((uintptr_t)x % align == 0) &&
               ((uintptr_t)g % align == 0);
    if (xdt == SP_F64) return launch_sampled_typed<double>(a, vec, s);
    if (xdt == SP_F32) return launch_sampled_typed<float>(a, vec, s);
    return SP_ERR_DTYPE;
}

}  // namespace sp
