// Launch of the SpMMV kernel variants; included by the per-precision,
// per-width translation units (spmv_<pair>_<widths>.cu), which compile in
// parallel.  The block width is a compile-time constant of each kernel
// variant (the paper's fixed-loop-length code generation, Sec.
// "Implementation"), padded to a power of two; a variant exists for every
// width up to 32, so every width is served (the paper's always-correct
// fallback chain); wider blocks are processed in tiles of 32 columns.
#pragma once

#include <type_traits>

#include "spmv_kernel.cuh"

namespace sp {

// Row order of the product kernel: 0 = static cost-balanced contiguous range
// per warp; 1 = block-strided front (all warps near the same rows);
// 2 = moving front with a balanced assignment (falls back to 0 when the grid
// has no schedule).
#ifndef SP_ORDER
#define SP_ORDER 2
#endif

// The moving front is taken when x is larger than this fraction of L2.
#ifndef SP_FRONT_X_L2_FRAC
#define SP_FRONT_X_L2_FRAC 0.5
#endif

// Dynamic row order for products without fused reductions (knob) and the
// number of slot runs per warp it aims at.
#ifndef SP_DYN
#define SP_DYN 1
#endif
#ifndef SP_DYN_RUNS_PER_WARP
#define SP_DYN_RUNS_PER_WARP 16
#endif
#ifndef SP_DYN_MIN_WP
#define SP_DYN_MIN_WP 8
#endif

// Preferred shared-memory carveout (percent of the unified L1/shared array
// given to shared memory); negative: leave the CUDA default.
#ifndef SP_CARVEOUT
#define SP_CARVEOUT -1
#endif

template <class VT, class XT, int WP, bool VEC, int DM, bool MT, bool LS, int EPI, int MV = 0>
static int launch_spmv_variant(const SpmvArgs &a, int max_blocks, cudaStream_t s) {
    constexpr int CPL = cols_per_lane<XT, WP>();
    constexpr int G = WP / CPL;
    constexpr int ROWS = (32 / G) * kMainWarps;
    static int occ = 0;
    if (occ == 0) {
        if (SP_CARVEOUT >= 0)
            cudaFuncSetAttribute(k_spmmv<VT, XT, WP, VEC, DM, MT, LS, EPI, MV>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 SP_CARVEOUT);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmmv<VT, XT, WP, VEC, DM, MT, LS, EPI, MV>,
                                                                      kMainThreads, 0);
        if (e != cudaSuccess || occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
    }
    int sms = 1;
    SP_TRY(device_sm_count(&sms));
    const int lt = MT ? host_log2_tpr(a.C, G) : 0;
    int64_t need = ((a.nslots << lt) + ROWS - 1) / ROWS;
    int64_t grid = (int64_t)sms * occ;
    if (grid > max_blocks) grid = max_blocks;
    // with a partition table the whole persistent grid runs (idle warps exit at
    // once), so even a small matrix is spread over every SM
    const bool part = SP_ORDER != 1 && a.wbounds_src && partition_for(*a.wbounds_src, grid * kMainWarps);
    if (!part && grid > need) grid = need;
    if (grid < 1) grid = 1;
    SpmvArgs b = a;
    b.wbounds = part ? partition_for(*a.wbounds_src, grid * kMainWarps) : nullptr;
    b.sched = nullptr;
    b.sched_rounds = 0;
    // unless the matrix names an order: the moving front pays when x does not
    // fit in L2 (its reuse across rows must then come from L2); otherwise the
    // contiguous ranges keep more of x in L1
    if (SP_ORDER == 2 && part && kMainWarps == kSchedCtaWarps) {
        const int order = a.wbounds_src->order;
        const bool front = order == 1 || (order == 0 && (double)a.wbounds_src->ncols * a.w * sizeof(XT) >
                                                            SP_FRONT_X_L2_FRAC * (double)device_l2_bytes());
        if (front) b.sched = schedule_for(*a.wbounds_src, grid * kMainWarps, &b.sched_rounds);
    }
    b.nsm = sms;
    b.log2_tpr = lt;
    b.log2C = ilog2_exact(a.C);
    // products without fused reductions on wide row-major blocks take their
    // rows in dynamic order: runs of whole 32-slot blocks, about
    // SP_DYN_RUNS_PER_WARP runs per warp.  Measured faster for w = 8 and 16
    // (Anderson: float32 105 -> 85 and 179 -> 140 us, float64 274 -> 264 and
    // 540 -> 515 us) and slower where x is reused from L1 by the adjacent
    // ranges of one SM's warps (float32 w = 4: 46 -> 71 us; power-law forward
    // 63 -> 78 us).
    b.dyn_grab = 0;
    if constexpr (DM == 0 && MV == 0 && VEC && WP >= SP_DYN_MIN_WP) {
        if (SP_DYN != 0 && a.ticket) {
            const int64_t warps = grid * kMainWarps;
            int64_t g = (a.nslots + warps * SP_DYN_RUNS_PER_WARP - 1) / (warps * SP_DYN_RUNS_PER_WARP);
            g = (g + 31) / 32 * 32;
            b.dyn_grab = (int32_t)(g < 32 ? 32 : g);
        }
    }
    k_spmmv<VT, XT, WP, VEC, DM, MT, LS, EPI, MV><<<(unsigned)grid, kMainThreads, 0, s>>>(b);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

template <class VT, class XT, int WP, bool MT, bool LS>
static int launch_spmv_wml(const SpmvArgs &a, bool vec, int max_blocks, cudaStream_t s) {
    // dot set compiled in: none, <y,y> and <x,y>, or all three
    const uint32_t req = (a.flags & SP_SPMV_DOT_ANY) / SP_SPMV_DOT_YY;
    if constexpr (std::is_same<VT, double>::value && std::is_same<XT, double>::value) {
        // shift, scale and beta = 1 with fused dots: the two-fma epilogue
        const uint32_t need = SP_SPMV_SCALE | SP_SPMV_AXPBY;
        if (req && (a.flags & need) == need && (a.flags & (SP_SPMV_SHIFT | SP_SPMV_VSHIFT)) && a.beta == 1.0) {
            SpmvArgs b = a;  // the kernel takes alpha gamma in place of gamma
            for (int k = 0; k < kMaxTileW; ++k) b.gamma[k] = a.alpha * a.gamma[k];
            if (req & 4)
                return vec ? launch_spmv_variant<VT, XT, WP, true, 7, MT, LS, 3>(b, max_blocks, s)
                           : launch_spmv_variant<VT, XT, WP, false, 7, MT, LS, 3>(b, max_blocks, s);
            return vec ? launch_spmv_variant<VT, XT, WP, true, 3, MT, LS, 3>(b, max_blocks, s)
                       : launch_spmv_variant<VT, XT, WP, false, 3, MT, LS, 3>(b, max_blocks, s);
        }
    }
    if (req & 4)
        return vec ? launch_spmv_variant<VT, XT, WP, true, 7, MT, LS, 2>(a, max_blocks, s)
                   : launch_spmv_variant<VT, XT, WP, false, 7, MT, LS, 2>(a, max_blocks, s);
    if (req)
        return vec ? launch_spmv_variant<VT, XT, WP, true, 3, MT, LS, 2>(a, max_blocks, s)
                   : launch_spmv_variant<VT, XT, WP, false, 3, MT, LS, 2>(a, max_blocks, s);
    if constexpr (sizeof(XT) == 8) {
        // float64 vectors: the plain product and the Chebyshev step get
        // epilogues without runtime flags (no float64 work for flags that are off)
        const uint32_t ef = a.flags & (SP_SPMV_SHIFT | SP_SPMV_VSHIFT | SP_SPMV_SCALE | SP_SPMV_AXPBY |
                                       SP_SPMV_CHAIN_AXPBY);
        if (ef == 0)
            return vec ? launch_spmv_variant<VT, XT, WP, true, 0, MT, LS, 0>(a, max_blocks, s)
                       : launch_spmv_variant<VT, XT, WP, false, 0, MT, LS, 0>(a, max_blocks, s);
        if (ef == (SP_SPMV_SCALE | SP_SPMV_AXPBY))
            return vec ? launch_spmv_variant<VT, XT, WP, true, 0, MT, LS, 1>(a, max_blocks, s)
                       : launch_spmv_variant<VT, XT, WP, false, 0, MT, LS, 1>(a, max_blocks, s);
    }
    return vec ? launch_spmv_variant<VT, XT, WP, true, 0, MT, LS, 2>(a, max_blocks, s)
               : launch_spmv_variant<VT, XT, WP, false, 0, MT, LS, 2>(a, max_blocks, s);
}

// Lockstep row loop (row_product_ls) or per-lane loop: the lockstep form saves
// float64-pipe steps when lanes of a warp have rows of different lengths, and
// costs a few instructions per step; it is used only where the float64 pipe
// binds (float64 values and vectors).
template <class VT, class XT, int WP, bool MT>
static int launch_spmv_wm(const SpmvArgs &a, bool vec, int max_blocks, cudaStream_t s) {
    constexpr bool f64 = std::is_same<VT, double>::value && std::is_same<XT, double>::value;
    if constexpr (!f64 || SP_LOCKSTEP == 0) {
        return launch_spmv_wml<VT, XT, WP, MT, false>(a, vec, max_blocks, s);
    } else if constexpr (WP >= 2 || SP_LOCKSTEP == 2) {
        return launch_spmv_wml<VT, XT, WP, MT, true>(a, vec, max_blocks, s);
    } else {
        // the fused dots and the chain add float64 work per row, so the pipe
        // binds already at a smaller spread
        const double thr = (a.flags & (SP_SPMV_DOT_ANY | SP_SPMV_CHAIN_AXPBY)) ? SP_LS_SPREAD_DOTS : SP_LS_SPREAD;
        const bool ls = a.wbounds_src && a.wbounds_src->lane_spread > thr;
        return ls ? launch_spmv_wml<VT, XT, WP, MT, true>(a, vec, max_blocks, s)
                  : launch_spmv_wml<VT, XT, WP, MT, false>(a, vec, max_blocks, s);
    }
}

// Every kernel variant of one (value, vector) precision pair and one padded
// width.  Instantiated by the spmv_<pair>_<widths>.cu units, a few widths
// each, so that the variants compile in parallel; spmv_dispatch.cu picks the
// width at run time (launch_spmv_typed).
template <class VT, class XT, int WP>
int launch_spmv_width(const SpmvArgs &a, bool vec, int max_blocks, cudaStream_t s) {
    constexpr int CPL = cols_per_lane<XT, WP>();
    const bool mt = host_log2_tpr(a.C, WP / CPL) > 0;
    return mt ? launch_spmv_wm<VT, XT, WP, true>(a, vec, max_blocks, s)
              : launch_spmv_wm<VT, XT, WP, false>(a, vec, max_blocks, s);
}

#define SP_INSTANTIATE_WIDTH(VT, XT, WP) \
    template int launch_spmv_width<VT, XT, WP>(const SpmvArgs &, bool, int, cudaStream_t);

}  // namespace sp
