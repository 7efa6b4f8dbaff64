// Batched SpMMV over many SELL-C-sigma matrices of uneven size and block
// width in ONE persistent launch, and a mixed-precision CG with iterative
// refinement built on it (float64 residual and solution update, float32 inner
// solve), with the inner iterations captured in a CUDA graph.
//
// Work list.  Every matrix's row slots are cut into units of about equal
// cost (stored entries + 2 per row) at 32-slot granularity; unit u is owned by
// warp u mod (number of resident warps), so the assignment is static and the
// per-unit dot partials are summed per matrix in a fixed order: the results
// are deterministic.  A unit carries the lane layout chosen for its matrix
// (block width padded to WP in {1,2,4,8}, CPL columns per lane), so one launch
// serves matrices of different widths with the same row kernel as sp_spmv.
//
// Inner solver: the Chronopoulos-Gear form of CG (A. T. Chronopoulos and
// C. W. Gear, "s-step iterative methods for symmetric linear systems", J.
// Comput. Appl. Math. 25 (1989)), which needs per iteration one product
// s = A r and the two inner products <r,r>, <r,s> -- exactly the <x,x> and
// <x,y> that the augmented product fuses -- followed by one vector update:
//     beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old)
//     p = r + beta p,  q = s + beta q,  d = d + alpha p,  r = r - alpha q
// (alpha = gamma / delta, beta = 0 on the first iteration).
#include <algorithm>
#include <type_traits>
#include <vector>

#include "spmv_kernel.cuh"
#include "dotacc.cuh"

namespace sp {

constexpr int kBatchMaxW = SP_BATCH_MAX_W;
constexpr int kNumVariants = 10;
// (WP, CPL) of each lane-layout variant
__host__ __device__ constexpr int variant_wp(int v) { return v == 0 ? 1 : v <= 2 ? 2 : v <= 5 ? 4 : 8; }
__host__ __device__ constexpr int variant_cpl(int v) {
    return v == 0 ? 1 : v == 1 ? 1 : v == 2 ? 2 : v == 3 ? 1 : v == 4 ? 2 : v == 5 ? 4 : v == 6 ? 1 : v == 7 ? 2
                                                                                     : v == 8 ? 4 : 8;
}
static int variant_of(int wp, int cpl) {
    for (int v = 0; v < kNumVariants; ++v)
        if (variant_wp(v) == wp && variant_cpl(v) == cpl) return v;
    return -1;
}

struct BMat {
    const void *val;
    const int32_t *col;
    const int64_t *chunkptr;
    const int32_t *slotlen;
    const int32_t *perm;  // null: identity
    int64_t nrows;
    int32_t C, w;
    const void *x;   // ncols x w row-major, ld = w
    void *y;         // nrows x w
    const void *y0;  // beta term source (may equal y)
    int32_t unit0, unit1;
};

struct BUnit {
    int32_t m;
    int16_t variant, log2_tpr;  // lane layout and threads per row of matrix m
    int64_t s0, s1;
};

struct BatchArgs {
    const BMat *mats;
    const BUnit *units;
    int32_t nunits;
    uint32_t flags;
    double alpha, beta;
    double *partials;  // [unit][3][kBatchMaxW]
    unsigned *next;    // unit counter of the dynamic assignment (zero at launch)
};

// Units go to warps dynamically (each warp takes the next unit from a counter)
// when SP_BATCH_DYNAMIC is set, else statically (unit u to warp u mod warps).
// Either way a unit's partial sums land in the unit's own slot and are added
// in unit order, so the results do not depend on the assignment.
#ifndef SP_BATCH_DYNAMIC
#define SP_BATCH_DYNAMIC 1
#endif
// units per resident warp the work list is cut into: finer units balance the
// warps better, but every CG iteration sums the dot partials of all units of
// a matrix (64-system batch: 8 -> 16 took the float32 product from 367 to
// 352 us and the mixed-precision solve from 0.261 to 0.260 s; 32 made the
// solves slower, 0.278 s)
#ifndef SP_BATCH_UNITS_PER_WARP
#define SP_BATCH_UNITS_PER_WARP 16
#endif

// float32 inner CG: its two inner products accumulated in float per lane and
// unit (knob; float64 across lanes and units either way)
#ifndef SP_CG_PLAIN_DOTS
#define SP_CG_PLAIN_DOTS 1
#endif
// load the next slot's metadata while the current slot runs (knob; off: the
// registers it holds cost the kernel that carries every layout more than the
// latency it hides, 418 -> 376 us on the 64-system float32 product)
#ifndef SP_BATCH_PREFETCH
#define SP_BATCH_PREFETCH 0
#endif
// matrix loads: 1 always evict-first, 0 never, 2 only where a warp step reads
// whole sectors (knob)
#ifndef SP_BATCH_STREAM
#define SP_BATCH_STREAM 2
#endif
// unroll depth of the row loop for 4-column lanes (knob)
#ifndef SP_BATCH_UNROLL_WIDE
#define SP_BATCH_UNROLL_WIDE SP_UNROLL_WIDE
#endif

// DM: the dot products this kernel accumulates (bit 0 <y,y>, bit 1 <x,y>,
// bit 2 <x,x>), a compile-time set so that only their accumulators hold
// registers; the flags pick which of them are written.
template <class VT, class XT, int WP, int CPL, int DM>
__device__ __forceinline__ void batch_unit(const BatchArgs &a, const BMat *__restrict__ Mp, const BUnit &u, int lane,
                                           double *part) {
    using AT = typename AccOf<VT, XT>::T;
    constexpr int G = WP / CPL;
    constexpr int R = 32 / G;
    constexpr int U = CPL >= 4 ? SP_BATCH_UNROLL_WIDE : SP_UNROLL_NARROW / CPL;
    constexpr bool dots = (DM & 7) != 0;
    // evict-first matrix loads only where one warp step reads whole 32-byte
    // sectors of values and indices (R rows of a chunk column per step)
    constexpr bool stream = SP_BATCH_STREAM == 1 || (SP_BATCH_STREAM == 2 && R * sizeof(int32_t) >= 32 &&
                                                     R * sizeof(VT) >= 32);
    const int lt = u.log2_tpr;
    const int T = 1 << lt;
    const int gl = lane % G;
    const int tt = (lane / G) & (T - 1);
    const int rw = (lane / G) >> lt;
    const int Rr = R >> lt;
    const unsigned rowmask = (G * T == 32) ? 0xffffffffu : (((1u << (G * T)) - 1u) << (rw * G * T));
    const int w = Mp->w;
    const int k0 = gl * CPL;
    const int nvalid = w - k0 < CPL ? w - k0 : CPL;
    const uint32_t f = a.flags;
    const bool need_xi = (DM & 6) != 0;
    const VT *__restrict__ val = (const VT *)Mp->val;
    const int32_t *__restrict__ colp = Mp->col;
    const int64_t *__restrict__ chunkptr = Mp->chunkptr;
    const int32_t *__restrict__ slotlen = Mp->slotlen;
    const int32_t *__restrict__ perm = Mp->perm;
    const int64_t nrows = Mp->nrows;
    const uint32_t C = (uint32_t)Mp->C;
    const XT *__restrict__ xk = (const XT *)Mp->x + k0;
    const XT alpha = (XT)a.alpha, beta = (XT)a.beta;
    // DM bit 3: accumulate in the vector precision (the float32 inner CG)
    using Acc = typename std::conditional<(DM & 8) != 0, DotAccPlain<XT>, DotAcc<XT>>::type;
    Acc ayy[(DM & 1) ? CPL : 1], axy[(DM & 2) ? CPL : 1], axx[(DM & 4) ? CPL : 1];
    // where a slot's row lives; the next slot's is loaded while this one runs
    struct Meta {
        int64_t i, off;
        int len;
    };
    auto meta_of = [&](int64_t s) {
        Meta m;
        m.i = perm ? (int64_t)perm[s] : (s < nrows ? s : -1);
        const uint32_t cidx = (uint32_t)s / C;
        m.off = chunkptr[cidx] + ((uint32_t)s - cidx * C) + (int64_t)tt * C;
        m.len = slotlen[s];
        return m;
    };
    int64_t s = u.s0 + rw;
    Meta cur{-1, 0, 0};
    if (SP_BATCH_PREFETCH && s < u.s1) cur = meta_of(s);
    for (; s < u.s1; s += Rr) {
        Meta nxt{-1, 0, 0};
        if (SP_BATCH_PREFETCH) {
            if (s + Rr < u.s1) nxt = meta_of(s + Rr);
        } else {
            cur = meta_of(s);
        }
        const int64_t i = cur.i;
        if (i >= 0) {
            const int len_t = cur.len > tt ? (cur.len - tt + T - 1) >> lt : 0;
            AT acc[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) acc[c] = AT(0);
            int bad = 0;
            row_product<VT, XT, AT, CPL, true, U, false, stream>(val + cur.off, colp + cur.off, (int)C << lt, len_t,
                                                                 xk, w, 1, nvalid, acc, bad);
            if constexpr (std::is_same<AT, float>::value && std::is_same<XT, double>::value) {
                if (bad) {  // x outside the fast conversion's range: again with the conversion instruction
#pragma unroll
                    for (int c = 0; c < CPL; ++c) acc[c] = AT(0);
                    row_product<VT, XT, AT, CPL, true, U, true, stream>(val + cur.off, colp + cur.off, (int)C << lt,
                                                                        len_t, xk, w, 1, nvalid, acc, bad);
                }
            }
            bool epi = true;
            if (T > 1) {
#pragma unroll
                for (int c = 0; c < CPL; ++c)
                    for (int o = G; o < G * T; o <<= 1) acc[c] += __shfl_xor_sync(rowmask, acc[c], o);
                epi = tt == 0;
            }
            if (epi && nvalid > 0) {
                XT xi[CPL], yo[CPL], t[CPL];
                if (need_xi) load_cols<XT, CPL, true>(xk + i * w, 1, nvalid, xi);
                if (f & SP_SPMV_AXPBY) load_out<XT, CPL, true>((const XT *)Mp->y0 + i * w + k0, 1, nvalid, yo);
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    XT v = acc_to_x<XT, AT>(acc[c]);
                    if (f & SP_SPMV_SCALE) v = mul_rn(alpha, v);
                    if (f & SP_SPMV_AXPBY) v = fma_rn(beta, yo[c], v);
                    t[c] = v;
                }
                store_out<XT, CPL, true>((XT *)Mp->y + i * w + k0, 1, nvalid, t);
                if constexpr (dots) {
#pragma unroll
                    for (int c = 0; c < CPL; ++c) {
                        if constexpr ((DM & 1) != 0) ayy[c].add(t[c], t[c]);
                        if constexpr ((DM & 2) != 0) axy[c].add(xi[c], t[c]);
                        if constexpr ((DM & 4) != 0) axx[c].add(xi[c], xi[c]);
                    }
                }
            }
        }
        cur = nxt;
    }
    if constexpr (dots) {
        if constexpr ((DM & 8) != 0) {
            // plain accumulators: the xor tree across lanes in the vector
            // precision too (one conversion per unit instead of one per step)
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int o = G; o < 32; o <<= 1) {
                    if constexpr ((DM & 1) != 0) ayy[c].v += __shfl_xor_sync(0xffffffffu, ayy[c].v, o);
                    if constexpr ((DM & 2) != 0) axy[c].v += __shfl_xor_sync(0xffffffffu, axy[c].v, o);
                    if constexpr ((DM & 4) != 0) axx[c].v += __shfl_xor_sync(0xffffffffu, axx[c].v, o);
                }
        }
        double dyy[CPL], dxy[CPL], dxx[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            dyy[c] = (DM & 1) ? ayy[(DM & 1) ? c : 0].value() : 0.0;
            dxy[c] = (DM & 2) ? axy[(DM & 2) ? c : 0].value() : 0.0;
            dxx[c] = (DM & 4) ? axx[(DM & 4) ? c : 0].value() : 0.0;
#pragma unroll
            for (int o = G; o < 32 && (DM & 8) == 0; o <<= 1) {
                if constexpr ((DM & 1) != 0) dyy[c] += __shfl_xor_sync(0xffffffffu, dyy[c], o);
                if constexpr ((DM & 2) != 0) dxy[c] += __shfl_xor_sync(0xffffffffu, dxy[c], o);
                if constexpr ((DM & 4) != 0) dxx[c] += __shfl_xor_sync(0xffffffffu, dxx[c], o);
            }
        }
        if (lane < G) {
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                int k = k0 + c;
                if (k < w) {
                    part[0 * kBatchMaxW + k] = dyy[c];
                    part[1 * kBatchMaxW + k] = dxy[c];
                    part[2 * kBatchMaxW + k] = dxx[c];
                }
            }
        }
    }
}

// widest lane vector a batch may use: 2 doubles or 4 floats (wider blocks use
// more lanes per row); this bounds the registers of the one kernel that holds
// every layout
__host__ __device__ constexpr int batch_max_cpl(int xsize) { return xsize == 8 ? 2 : 4; }

// block size and minimum resident blocks per SM of the batched kernel (knobs)
#ifndef SP_BATCH_THREADS
#define SP_BATCH_THREADS 256
#endif
#ifndef SP_BATCH_MINB
#define SP_BATCH_MINB (1024 / SP_BATCH_THREADS)
#endif
constexpr int kBatchThreads = SP_BATCH_THREADS;
constexpr int kBatchWarps = kBatchThreads / 32;

template <class VT, class XT, int DM>
__global__ void __launch_bounds__(kBatchThreads, SP_BATCH_MINB) k_spmmv_batched(const __grid_constant__ BatchArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kBatchWarps + (threadIdx.x >> 5);
    const int T = gridDim.x * kBatchWarps;
    for (int u = gw;;) {
        if (SP_BATCH_DYNAMIC) {
            int t = 0;
            if (lane == 0) t = (int)atomicAdd(a.next, 1u);
            u = __shfl_sync(0xffffffffu, t, 0);
        }
        if (u >= a.nunits) break;
        const BUnit U = a.units[u];
        const BMat *__restrict__ M = a.mats + U.m;
        double *part = a.partials + (int64_t)u * 3 * kBatchMaxW;
        constexpr bool wide = batch_max_cpl(sizeof(XT)) >= 4;
        switch (U.variant) {
            case 0: batch_unit<VT, XT, 1, 1, DM>(a, M, U, lane, part); break;
            case 1: batch_unit<VT, XT, 2, 1, DM>(a, M, U, lane, part); break;
            case 2: batch_unit<VT, XT, 2, 2, DM>(a, M, U, lane, part); break;
            case 3: batch_unit<VT, XT, 4, 1, DM>(a, M, U, lane, part); break;
            case 4: batch_unit<VT, XT, 4, 2, DM>(a, M, U, lane, part); break;
            case 6: batch_unit<VT, XT, 8, 1, DM>(a, M, U, lane, part); break;
            case 7: batch_unit<VT, XT, 8, 2, DM>(a, M, U, lane, part); break;
            default:
                if constexpr (wide) {
                    if (U.variant == 5) batch_unit<VT, XT, 4, 4, DM>(a, M, U, lane, part);
                    else batch_unit<VT, XT, 8, 4, DM>(a, M, U, lane, part);
                }
                break;
        }
        if (!SP_BATCH_DYNAMIC) u += T;
    }
}

// Sum of one partial value over the units of a matrix, in unit order per lane
// and a fixed xor tree across lanes (same result in every block that asks).
__device__ __forceinline__ double sum_units(const double *partials, int u0, int u1, int q, int k, int lane) {
    double s = 0.0;
    for (int u = u0 + lane; u < u1; u += 32) s += __ldcg(partials + (int64_t)u * 3 * kBatchMaxW + q * kBatchMaxW + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// dots[m][q][k] for the requested q: one block per matrix, one warp per (q, k)
__global__ void k_batch_dots(const BMat *mats, const double *partials, uint32_t flags, double *dots) {
    const int m = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const BMat M = mats[m];
    for (int v = warp; v < 3 * M.w; v += blockDim.x / 32) {
        int q = v / M.w, k = v - q * M.w;
        if (!(flags & (SP_SPMV_DOT_YY << q))) continue;
        double s = sum_units(partials, M.unit0, M.unit1, q, k, lane);
        if (lane == 0) dots[(int64_t)m * 3 * kBatchMaxW + q * kBatchMaxW + k] = s;
    }
}

// ------------------------------------------------------------------ host side: batch objects

struct Batch {
    int count = 0;
    sp_dtype vdt = SP_F64, xdt = SP_F64;
    std::vector<sp_mat *> mats;       // not owned
    std::vector<BMat> hmats;
    std::vector<BUnit> hunits;
    DevBufPtr dmats, dunits, partials, next;
    int grid = 1;
};

// cost-balanced units of at most ~target cost, cut at 32-slot boundaries
static int make_units(Batch &B, int64_t target) {
    B.hunits.clear();
    for (int m = 0; m < B.count; ++m) {
        const Pattern &P = *B.mats[m]->pat;
        std::vector<int32_t> sl(P.nslots);
        if (P.nslots)
            SP_CUDA(cudaMemcpy(sl.data(), P.slotlen->ptr, P.nslots * sizeof(int32_t), cudaMemcpyDeviceToHost));
        int w = B.hmats[m].w;
        int v = B.hmats[m].unit0;  // holds the variant until units are made
        B.hmats[m].unit0 = (int32_t)B.hunits.size();
        int64_t s0 = 0, cost = 0;
        for (int64_t s = 0; s < P.nslots; ++s) {
            cost += (int64_t)(sl[s] + (s < P.nrows ? 2 : 0)) * std::max(1, w);
            bool cut = ((s + 1) % 32 == 0) && cost >= target;
            if (cut || s + 1 == P.nslots) {
                int G = variant_wp(v) / variant_cpl(v);
                B.hunits.push_back(BUnit{m, (int16_t)v, (int16_t)host_log2_tpr(P.C, G), s0, s + 1});
                s0 = s + 1;
                cost = 0;
            }
        }
        B.hmats[m].unit1 = (int32_t)B.hunits.size();
    }
    return SP_OK;
}

static size_t xsize(sp_dtype t) { return t == SP_F64 ? 8 : 4; }

// choose CPL for width w: the widest lane vector that divides w and keeps
// 16-byte (or 8-byte) alignment of every row
static int auto_cpl(int w, size_t xs) {
    int wp = 1;
    while (wp < w) wp <<= 1;
    int c = std::min(wp, batch_max_cpl((int)xs));
    while (c > 1 && (w % c != 0 || ((size_t)w * xs) % std::min<size_t>(16, c * xs) != 0)) c >>= 1;
    return c;
}

static int batch_init(Batch &B, int count, sp_mat *const *A, const int32_t *widths, const int32_t *cpl,
                      sp_dtype xdt) {
    if (count < 1 || !A || !widths) return SP_ERR_ARG;
    B.count = count;
    B.xdt = xdt;
    B.mats.assign(A, A + count);
    B.vdt = A[0]->vdt;
    B.hmats.resize(count);
    int64_t total_cost = 0;
    for (int m = 0; m < count; ++m) {
        if (!A[m]) return SP_ERR_ARG;
        if (A[m]->vdt != B.vdt) return SP_ERR_DTYPE;
        int w = widths[m];
        if (w < 1 || w > kBatchMaxW) return SP_ERR_ARG;
        int c = (cpl && cpl[m] > 0) ? cpl[m] : auto_cpl(w, xsize(xdt));
        int wp = 1;
        while (wp < w) wp <<= 1;
        if (c > wp || c > batch_max_cpl((int)xsize(xdt)) || (w % c) != 0 ||
            ((size_t)w * xsize(xdt)) % std::min<size_t>(16, c * xsize(xdt)) != 0)
            return SP_ERR_ARG;
        int v = variant_of(wp, c);
        if (v < 0) return SP_ERR_ARG;
        const Pattern &P = *A[m]->pat;
        BMat &M = B.hmats[m];
        M.val = A[m]->val->ptr;
        M.col = (const int32_t *)P.col->ptr;
        M.chunkptr = (const int64_t *)P.chunkptr->ptr;
        M.slotlen = (const int32_t *)P.slotlen->ptr;
        M.perm = (P.sigma == 1 || P.permuted_space) ? nullptr : (const int32_t *)P.perm->ptr;
        M.nrows = P.nrows;
        M.C = P.C;
        M.w = w;
        M.x = M.y = nullptr;
        M.y0 = nullptr;
        M.unit0 = v;
        total_cost += (P.nstored + 2 * P.nrows) * w;
    }
    int sms = 1;
    SP_TRY(device_sm_count(&sms));
    int occ = 1;
    if (B.vdt == SP_F64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmmv_batched<double, double, 7>, kBatchThreads, 0);
    else if (xdt == SP_F32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmmv_batched<float, float, 7>, kBatchThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmmv_batched<float, double, 7>, kBatchThreads, 0);
    cudaGetLastError();
    occ = std::max(1, occ);
    B.grid = sms * occ;
    int64_t warps = (int64_t)B.grid * kBatchWarps;
    // about 4 units per resident warp, at least 32 slots each
    int64_t target = std::max<int64_t>(1, total_cost / (warps * SP_BATCH_UNITS_PER_WARP));
    SP_TRY(make_units(B, target));
    SP_TRY(dev_alloc(B.dmats, count * sizeof(BMat), nullptr));
    SP_TRY(dev_alloc(B.dunits, std::max<size_t>(1, B.hunits.size()) * sizeof(BUnit), nullptr));
    SP_TRY(dev_alloc(B.partials, std::max<size_t>(1, B.hunits.size()) * 3 * kBatchMaxW * sizeof(double), nullptr));
    SP_TRY(dev_alloc(B.next, sizeof(unsigned), nullptr));
    SP_CUDA(cudaMemset(B.partials->ptr, 0, B.partials->bytes));
    SP_CUDA(cudaMemcpy(B.dunits->ptr, B.hunits.data(), B.hunits.size() * sizeof(BUnit), cudaMemcpyHostToDevice));
    return SP_OK;
}

static int batch_upload(Batch &B, cudaStream_t s) {
    SP_CUDA(cudaMemcpyAsync(B.dmats->ptr, B.hmats.data(), B.count * sizeof(BMat), cudaMemcpyHostToDevice, s));
    SP_CUDA(cudaStreamSynchronize(s));
    return SP_OK;
}

template <class VT, class XT>
static void launch_batched_dm(int dm, int grid, const BatchArgs &a, cudaStream_t s) {
    if (dm == 0)
        k_spmmv_batched<VT, XT, 0><<<grid, kBatchThreads, 0, s>>>(a);
    else if (dm == 6)
        k_spmmv_batched<VT, XT, 6><<<grid, kBatchThreads, 0, s>>>(a);
    else if (dm == 14)
        k_spmmv_batched<VT, XT, 14><<<grid, kBatchThreads, 0, s>>>(a);
    else
        k_spmmv_batched<VT, XT, 7><<<grid, kBatchThreads, 0, s>>>(a);
}

static int batch_launch(const Batch &B, uint32_t flags, double alpha, double beta, cudaStream_t s,
                        bool plain_dots = false) {
    BatchArgs a;
    a.mats = (const BMat *)B.dmats->ptr;
    a.units = (const BUnit *)B.dunits->ptr;
    a.nunits = (int32_t)B.hunits.size();
    a.flags = flags;
    a.alpha = alpha;
    a.beta = beta;
    a.partials = (double *)B.partials->ptr;
    a.next = (unsigned *)B.next->ptr;
    if (SP_BATCH_DYNAMIC) SP_CUDA(cudaMemsetAsync(B.next->ptr, 0, sizeof(unsigned), s));
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(B.grid, (a.nunits + kBatchWarps - 1) / kBatchWarps));
    // dot set compiled in: none, the CG pair <x,y>, <x,x>, or all three
    const int req = (int)((flags & SP_SPMV_DOT_ANY) / SP_SPMV_DOT_YY);
    int dm = req == 0 ? 0 : (req & 1) ? 7 : 6;
    if (dm == 6 && plain_dots && B.xdt == SP_F32) dm = 14;
    if (B.vdt == SP_F64 && B.xdt == SP_F64)
        launch_batched_dm<double, double>(dm, grid, a, s);
    else if (B.vdt == SP_F32 && B.xdt == SP_F32)
        launch_batched_dm<float, float>(dm, grid, a, s);
    else if (B.vdt == SP_F32 && B.xdt == SP_F64)
        launch_batched_dm<float, double>(dm, grid, a, s);
    else
        return SP_ERR_DTYPE;
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// ------------------------------------------------------------------ CG kernels

struct CGCol {
    double gamma_prev, alpha_prev, gamma0;
    int32_t it, active;
};
struct OuterCol {
    double bb, rel, scale, norm;  // norm = ||r|| = 1 / scale (0 when inactive)
    int32_t active, pad;
};
struct VUnit {
    int32_t m, w;
    int64_t e0, e1;  // element range of the row-major n x w vectors
};
struct CGVec {
    void *r, *s, *p, *q, *d;   // inner precision
    double *x, *r64, *b;       // outer (float64)
    int32_t w;
};

__global__ void k_cg_scalars(const BMat *mats, const double *partials, int count, double inner_tol2,
                             CGCol *st, double *coef, float2 *coef_f) {
    const int m = blockIdx.x, lane = threadIdx.x & 31, k = threadIdx.x >> 5;
    const BMat M = mats[m];
    if (k >= M.w) return;
    double gamma = sum_units(partials, M.unit0, M.unit1, 2, k, lane);  // <r, r>
    double delta = sum_units(partials, M.unit0, M.unit1, 1, k, lane);  // <r, A r>
    if (lane != 0) return;
    CGCol &c = st[m * kBatchMaxW + k];
    double alpha = 0.0, beta = 0.0;
    if (c.active) {
        if (c.it == 0) c.gamma0 = gamma;
        bool go = gamma > inner_tol2 * c.gamma0 && gamma > 0.0;
        if (go) {
            if (c.it == 0) {
                alpha = gamma / delta;
            } else {
                beta = gamma / c.gamma_prev;
                alpha = gamma / (delta - beta * gamma / c.alpha_prev);
            }
            if (!(isfinite(alpha) && isfinite(beta))) go = false;
        }
        if (go) {
            c.gamma_prev = gamma;
            c.alpha_prev = alpha;
            c.it += 1;
        } else {
            c.active = 0;
            alpha = beta = 0.0;
        }
    }
    coef[(m * kBatchMaxW + k) * 2 + 0] = alpha;
    coef[(m * kBatchMaxW + k) * 2 + 1] = beta;
    coef_f[m * kBatchMaxW + k] = make_float2((float)alpha, (float)beta);
}

// 16-byte vector of the inner precision
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
    using V = float4;
};
template <>
struct Vec16<double> {
    using V = double2;
};

template <class T>
__device__ __forceinline__ void cg_update_elem(T &re, T se, T &pe, T &qe, T &de, T alpha, T beta) {
    pe = re + beta * pe;
    qe = se + beta * qe;
    de = de + alpha * pe;
    re = re - alpha * qe;
}

// p = r + beta p, q = s + beta q, d = d + alpha p, r = r - alpha q with the
// (alpha, beta) of each element's column; 16-byte accesses (units start at a
// multiple of 16 bytes and of a row), the unit's last partial vector scalar.
template <class T>
__global__ void k_cg_update(const VUnit *units, int nunits, const CGVec *vec, const double *coef,
                            const float2 *coef_f) {
    constexpr int NV = 16 / sizeof(T);
    using V = typename Vec16<T>::V;
    auto ab_of = [&](int m, int k, T &alpha, T &beta) {
        if constexpr (sizeof(T) == 4) {
            const float2 ab = coef_f[m * kBatchMaxW + k];  // no float64 conversion per element
            alpha = ab.x;
            beta = ab.y;
        } else {
            alpha = coef[(m * kBatchMaxW + k) * 2];
            beta = coef[(m * kBatchMaxW + k) * 2 + 1];
        }
    };
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
        const VUnit U = units[u];
        const CGVec Vc = vec[U.m];
        T *r = (T *)Vc.r + U.e0, *s = (T *)Vc.s + U.e0, *p = (T *)Vc.p + U.e0, *q = (T *)Vc.q + U.e0,
          *d = (T *)Vc.d + U.e0;
        const int64_t n = U.e1 - U.e0;
        const int64_t nv = n / NV;
        for (int64_t t = threadIdx.x; t < nv; t += blockDim.x) {
            V rv = reinterpret_cast<const V *>(r)[t], sv = reinterpret_cast<const V *>(s)[t];
            V pv = reinterpret_cast<const V *>(p)[t], qv = reinterpret_cast<const V *>(q)[t];
            V dv = reinterpret_cast<const V *>(d)[t];
            T *re = reinterpret_cast<T *>(&rv), *se = reinterpret_cast<T *>(&sv), *pe = reinterpret_cast<T *>(&pv);
            T *qe = reinterpret_cast<T *>(&qv), *de = reinterpret_cast<T *>(&dv);
            int k = (int)((t * NV) % U.w);  // units start on a row boundary
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                T alpha, beta;
                ab_of(U.m, k, alpha, beta);
                cg_update_elem(re[j], se[j], pe[j], qe[j], de[j], alpha, beta);
                k = k + 1 == U.w ? 0 : k + 1;
            }
            reinterpret_cast<V *>(p)[t] = pv;
            reinterpret_cast<V *>(q)[t] = qv;
            reinterpret_cast<V *>(d)[t] = dv;
            reinterpret_cast<V *>(r)[t] = rv;
        }
        for (int64_t e = nv * NV + threadIdx.x; e < n; e += blockDim.x) {
            T alpha, beta;
            ab_of(U.m, (int)(e % U.w), alpha, beta);
            T re = r[e], pe = p[e], qe = q[e], de = d[e];
            cg_update_elem(re, s[e], pe, qe, de, alpha, beta);
            p[e] = pe;
            q[e] = qe;
            d[e] = de;
            r[e] = re;
        }
    }
}

__global__ void k_outer_scalars(const BMat *mats, const double *partials, int count, double tol, int first,
                                OuterCol *oc, CGCol *st) {
    const int m = blockIdx.x, lane = threadIdx.x & 31, k = threadIdx.x >> 5;
    const BMat M = mats[m];
    if (k >= M.w) return;
    double rr = sum_units(partials, M.unit0, M.unit1, 0, k, lane);  // <r64, r64>
    if (lane != 0) return;
    OuterCol &o = oc[m * kBatchMaxW + k];
    if (first) o.bb = rr;
    o.rel = o.bb > 0.0 ? sqrt(rr / o.bb) : 0.0;
    o.active = o.rel > tol;
    o.scale = (o.active && rr > 0.0) ? 1.0 / sqrt(rr) : 0.0;
    o.norm = o.scale != 0.0 ? sqrt(rr) : 0.0;
    CGCol &c = st[m * kBatchMaxW + k];
    c.it = 0;
    c.active = o.active;
    c.gamma_prev = c.alpha_prev = c.gamma0 = 0.0;
}

template <class T>
__global__ void k_start_inner(const VUnit *units, int nunits, const CGVec *vec, const OuterCol *oc) {
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
        const VUnit U = units[u];
        const CGVec V = vec[U.m];
        T *r = (T *)V.r, *p = (T *)V.p, *q = (T *)V.q, *d = (T *)V.d;
        for (int64_t e = U.e0 + threadIdx.x; e < U.e1; e += blockDim.x) {
            const int k = (int)(e - U.e0) % U.w;  // units start on a row boundary
            double sc = oc[U.m * kBatchMaxW + k].scale;
            r[e] = (T)(V.r64[e] * sc);
            p[e] = T(0);
            q[e] = T(0);
            d[e] = T(0);
        }
    }
}

template <class T>
__global__ void k_x_update(const VUnit *units, int nunits, const CGVec *vec, const OuterCol *oc) {
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
        const VUnit U = units[u];
        const CGVec V = vec[U.m];
        const T *d = (const T *)V.d;
        for (int64_t e = U.e0 + threadIdx.x; e < U.e1; e += blockDim.x) {
            const int k = (int)(e - U.e0) % U.w;  // units start on a row boundary
            const double nr = oc[U.m * kBatchMaxW + k].norm;
            V.x[e] = __fma_rn((double)d[e], nr, V.x[e]);  // x += ||r|| d
        }
    }
}

__global__ void k_copy_f64(const double *src, double *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

}  // namespace sp

using namespace sp;

struct sp_batch {
    Batch B;
};

struct sp_cg {
    int count = 0;
    std::vector<int32_t> widths;
    std::vector<int64_t> nrows;
    std::vector<sp_mat *> A64;   // caller's
    std::vector<sp_mat *> A32;   // owned clones
    Batch b64;                   // residual: x64 -> r64 (y0 = b)
    Batch b32, b64in;            // inner products (float32, or float64 when asked)
    std::vector<VUnit> hvunits;
    DevBufPtr dvunits, dvec32, dvec64, vecs, cgcol, outer, coef, coef_f;
    std::vector<CGVec> hvec32, hvec64;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [inner f32, inner f64]
    int graph_iters[2] = {0, 0};
    double graph_tol2[2] = {-1.0, -1.0};  // inner tolerance baked into each captured graph
    int grid_vec = 1;
};

extern "C" {

int sp_batch_create(sp_batch **out, int count, sp_mat *const *A, const int32_t *widths,
                    const int32_t *cols_per_lane, sp_dtype vec_dtype, void *stream) {
    if (!out) return SP_ERR_ARG;
    *out = nullptr;
    if (vec_dtype != SP_F64 && vec_dtype != SP_F32) return SP_ERR_DTYPE;
    sp_batch *b = new sp_batch();
    int rc = batch_init(b->B, count, A, widths, cols_per_lane, vec_dtype);
    if (rc == SP_OK && b->B.vdt == SP_BF16) rc = SP_ERR_DTYPE;
    if (rc == SP_OK && b->B.vdt == SP_F64 && vec_dtype != SP_F64) rc = SP_ERR_DTYPE;
    if (rc != SP_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return SP_OK;
}

int sp_batch_bind(sp_batch *b, const void *const *x, void *const *y, const void *const *y0, void *stream) {
    if (!b || !x || !y) return SP_ERR_ARG;
    for (int m = 0; m < b->B.count; ++m) {
        if (!x[m] || !y[m]) return SP_ERR_ARG;
        if (((uintptr_t)x[m] | (uintptr_t)y[m] | (y0 && y0[m] ? (uintptr_t)y0[m] : 0)) % 16) return SP_ERR_ARG;
        b->B.hmats[m].x = x[m];
        b->B.hmats[m].y = y[m];
        b->B.hmats[m].y0 = (y0 && y0[m]) ? y0[m] : y[m];
    }
    return batch_upload(b->B, (cudaStream_t)stream);
}

int sp_batch_spmv(sp_batch *b, uint32_t flags, double alpha, double beta, double *dots, void *stream) {
    if (!b) return SP_ERR_ARG;
    const uint32_t ok = SP_SPMV_SCALE | SP_SPMV_AXPBY | SP_SPMV_DOT_ANY;
    if (flags & ~ok) return SP_ERR_UNSUPPORTED;
    if ((flags & SP_SPMV_DOT_ANY) && !dots) return SP_ERR_ARG;
    if (!b->B.hmats[0].x) return SP_ERR_ARG;  // not bound
    if (flags & (SP_SPMV_DOT_XY | SP_SPMV_DOT_XX))
        for (int m = 0; m < b->B.count; ++m)
            if (b->B.mats[m]->pat->nrows != b->B.mats[m]->pat->ncols) return SP_ERR_DIM;
    cudaStream_t s = (cudaStream_t)stream;
    SP_TRY(batch_launch(b->B, flags, alpha, beta, s));
    if (flags & SP_SPMV_DOT_ANY) {
        k_batch_dots<<<b->B.count, 256, 0, s>>>((const BMat *)b->B.dmats->ptr, (const double *)b->B.partials->ptr,
                                                 flags, dots);
        SP_CUDA(cudaGetLastError());
    }
    return SP_OK;
}

int sp_batch_info(const sp_batch *b, int32_t *nunits, int32_t *grid, int32_t *cols_per_lane) {
    if (!b) return SP_ERR_ARG;
    if (nunits) *nunits = (int32_t)b->B.hunits.size();
    if (grid) *grid = b->B.grid;
    if (cols_per_lane)
        for (int m = 0; m < b->B.count; ++m) {
            int u = b->B.hmats[m].unit0;
            cols_per_lane[m] = u < (int)b->B.hunits.size() ? variant_cpl(b->B.hunits[u].variant) : 0;
        }
    return SP_OK;
}

int sp_batch_destroy(sp_batch *b, void *stream) {
    if (!b) return SP_ERR_ARG;
    cudaStreamSynchronize((cudaStream_t)stream);
    delete b;
    return SP_OK;
}

// ------------------------------------------------------------------ mixed-precision CG

int sp_cg_create(sp_cg **out, int count, sp_mat *const *A, const int32_t *widths, const int32_t *cpl64,
                 const int32_t *cpl32, void *stream) {
    if (!out || !A || !widths || count < 1) return SP_ERR_ARG;
    *out = nullptr;
    cudaStream_t cs = (cudaStream_t)stream;
    sp_cg *cg = new sp_cg();
    auto fail = [&](int rc) {
        for (sp_mat *m : cg->A32) sp_mat_destroy(m, stream);
        delete cg;
        return rc;
    };
    cg->count = count;
    cg->widths.assign(widths, widths + count);
    cg->A64.assign(A, A + count);
    for (int m = 0; m < count; ++m) {
        if (!A[m] || A[m]->vdt != SP_F64) return fail(SP_ERR_DTYPE);
        if (A[m]->pat->nrows != A[m]->pat->ncols) return fail(SP_ERR_DIM);
        cg->nrows.push_back(A[m]->pat->nrows);
        sp_mat *c = nullptr;
        int rc = sp_mat_clone_values(&c, A[m], SP_F32, stream);
        if (rc != SP_OK) return fail(rc);
        cg->A32.push_back(c);
    }
    int rc = batch_init(cg->b64, count, A, widths, cpl64, SP_F64);
    if (rc == SP_OK) rc = batch_init(cg->b64in, count, A, widths, cpl64, SP_F64);
    if (rc == SP_OK) rc = batch_init(cg->b32, count, cg->A32.data(), widths, cpl32, SP_F32);
    if (rc != SP_OK) return fail(rc);
    // vectors: per matrix 5 inner vectors in f32 and in f64, plus x, r64, b in f64
    size_t total = 0;
    for (int m = 0; m < count; ++m) {
        int64_t n = cg->nrows[m] * widths[m];
        total += 5 * ((n * 4 + 255) / 256) * 256 + 5 * ((n * 8 + 255) / 256) * 256 + 3 * ((n * 8 + 255) / 256) * 256;
    }
    rc = dev_alloc(cg->vecs, std::max<size_t>(total, 256), cs);
    if (rc != SP_OK) return fail(rc);
    char *cur = (char *)cg->vecs->ptr;
    cg->hvec32.resize(count);
    cg->hvec64.resize(count);
    for (int m = 0; m < count; ++m) {
        int64_t n = cg->nrows[m] * widths[m];
        size_t b4 = ((n * 4 + 255) / 256) * 256, b8 = ((n * 8 + 255) / 256) * 256;
        CGVec &V = cg->hvec32[m];
        CGVec &W = cg->hvec64[m];
        V.r = cur; cur += b4; V.s = cur; cur += b4; V.p = cur; cur += b4; V.q = cur; cur += b4; V.d = cur; cur += b4;
        W.r = cur; cur += b8; W.s = cur; cur += b8; W.p = cur; cur += b8; W.q = cur; cur += b8; W.d = cur; cur += b8;
        double *x = (double *)cur; cur += b8;
        double *r64 = (double *)cur; cur += b8;
        double *b = (double *)cur; cur += b8;
        V.x = W.x = x;
        V.r64 = W.r64 = r64;
        V.b = W.b = b;
        V.w = W.w = widths[m];
        cg->b32.hmats[m].x = V.r;
        cg->b32.hmats[m].y = V.s;
        cg->b32.hmats[m].y0 = V.s;
        cg->b64in.hmats[m].x = W.r;
        cg->b64in.hmats[m].y = W.s;
        cg->b64in.hmats[m].y0 = W.s;
        cg->b64.hmats[m].x = x;
        cg->b64.hmats[m].y = r64;
        cg->b64.hmats[m].y0 = b;
    }
    rc = batch_upload(cg->b32, cs);
    if (rc == SP_OK) rc = batch_upload(cg->b64in, cs);
    if (rc == SP_OK) rc = batch_upload(cg->b64, cs);
    // element units for the vector kernels (about 16K elements each)
    for (int m = 0; m < count && rc == SP_OK; ++m) {
        int64_t n = cg->nrows[m] * widths[m];
        // a multiple of the row width and of 4 elements: every unit starts on a
        // row and on a 16-byte boundary
        const int64_t step = 16384 / (4 * widths[m]) * (4 * widths[m]);
        for (int64_t e = 0; e < n; e += step) cg->hvunits.push_back(VUnit{m, widths[m], e, std::min(n, e + step)});
    }
    if (rc == SP_OK) rc = dev_alloc(cg->dvunits, std::max<size_t>(1, cg->hvunits.size()) * sizeof(VUnit), cs);
    if (rc == SP_OK) rc = dev_alloc(cg->dvec32, count * sizeof(CGVec), cs);
    if (rc == SP_OK) rc = dev_alloc(cg->dvec64, count * sizeof(CGVec), cs);
    if (rc == SP_OK) rc = dev_alloc(cg->cgcol, count * kBatchMaxW * sizeof(CGCol), cs);
    if (rc == SP_OK) rc = dev_alloc(cg->outer, count * kBatchMaxW * sizeof(OuterCol), cs);
    if (rc == SP_OK) rc = dev_alloc(cg->coef, count * kBatchMaxW * 2 * sizeof(double), cs);
    if (rc == SP_OK) rc = dev_alloc(cg->coef_f, count * kBatchMaxW * sizeof(float2), cs);
    if (rc != SP_OK) return fail(rc);
    cudaError_t e = cudaMemcpy(cg->dvunits->ptr, cg->hvunits.data(), cg->hvunits.size() * sizeof(VUnit),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cg->dvec32->ptr, cg->hvec32.data(), count * sizeof(CGVec), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cg->dvec64->ptr, cg->hvec64.data(), count * sizeof(CGVec), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(cg->cgcol->ptr, 0, cg->cgcol->bytes);
    if (e == cudaSuccess) e = cudaMemset(cg->outer->ptr, 0, cg->outer->bytes);
    if (e == cudaSuccess) e = cudaMemset(cg->vecs->ptr, 0, cg->vecs->bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cg->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        sp_internal_note_cuda_error(e, "cg create", __FILE__, __LINE__);
        return fail(SP_ERR_CUDA);
    }
    int sms = 1;
    device_sm_count(&sms);
    cg->grid_vec = sms * 4;
    *out = cg;
    return SP_OK;
}

static int cg_inner_iteration(sp_cg *cg, int f64, double inner_tol2, cudaStream_t s) {
    Batch &B = f64 ? cg->b64in : cg->b32;
    SP_TRY(batch_launch(B, SP_SPMV_DOT_XX | SP_SPMV_DOT_XY, 1.0, 0.0, s, SP_CG_PLAIN_DOTS != 0));
    k_cg_scalars<<<cg->count, 32 * kBatchMaxW, 0, s>>>((const BMat *)B.dmats->ptr, (const double *)B.partials->ptr,
                                                       cg->count, inner_tol2, (CGCol *)cg->cgcol->ptr,
                                                       (double *)cg->coef->ptr, (float2 *)cg->coef_f->ptr);
    int nu = (int)cg->hvunits.size();
    int g = std::min(nu, cg->grid_vec);
    if (f64)
        k_cg_update<double><<<g, 256, 0, s>>>((const VUnit *)cg->dvunits->ptr, nu, (const CGVec *)cg->dvec64->ptr,
                                              (const double *)cg->coef->ptr, (const float2 *)cg->coef_f->ptr);
    else
        k_cg_update<float><<<g, 256, 0, s>>>((const VUnit *)cg->dvunits->ptr, nu, (const CGVec *)cg->dvec32->ptr,
                                             (const double *)cg->coef->ptr, (const float2 *)cg->coef_f->ptr);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

int sp_cg_solve(sp_cg *cg, const double *const *b, double *const *x, const sp_cg_opts *opts, sp_cg_stats *stats,
                double *rel_res, void *stream) {
    if (!cg || !b || !x) return SP_ERR_ARG;
    const sp_cg_opts defaults = SP_CG_OPTS_INIT;
    sp_cg_opts o = opts ? *opts : defaults;
    if (o.graph_iters < 1 || o.max_outer < 1 || o.max_inner < 1) return SP_ERR_ARG;
    cudaStream_t s = cg->stream;
    SP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    const int f64 = o.inner_f64 ? 1 : 0;
    const double inner_tol2 = o.inner_tol * o.inner_tol;
    const int nu = (int)cg->hvunits.size();
    const int gv = std::min(std::max(nu, 1), cg->grid_vec);
    // load b, zero x
    for (int m = 0; m < cg->count; ++m) {
        int64_t n = cg->nrows[m] * cg->widths[m];
        if (!b[m] || !x[m]) return SP_ERR_ARG;
        SP_CUDA(cudaMemcpyAsync(cg->hvec64[m].b, b[m], n * 8, cudaMemcpyDeviceToDevice, s));
        SP_CUDA(cudaMemsetAsync(cg->hvec64[m].x, 0, n * 8, s));
    }
    // (re)capture the inner graph when its iteration count or tolerance changes
    if (!cg->graph[f64] || cg->graph_iters[f64] != o.graph_iters || cg->graph_tol2[f64] != inner_tol2) {
        if (cg->graph[f64]) cudaGraphExecDestroy(cg->graph[f64]);
        cg->graph[f64] = nullptr;
        cudaGraph_t gr;
        SP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = SP_OK;
        for (int it = 0; it < o.graph_iters && rc == SP_OK; ++it) rc = cg_inner_iteration(cg, f64, inner_tol2, s);
        cudaError_t e = cudaStreamEndCapture(s, &gr);
        if (rc != SP_OK) return rc;
        SP_CUDA(e);
        e = cudaGraphInstantiate(&cg->graph[f64], gr, 0);
        cudaGraphDestroy(gr);
        SP_CUDA(e);
        cg->graph_iters[f64] = o.graph_iters;
        cg->graph_tol2[f64] = inner_tol2;
    }
    const CGVec *dvec = (const CGVec *)(f64 ? cg->dvec64->ptr : cg->dvec32->ptr);
    std::vector<OuterCol> hoc(cg->count * kBatchMaxW);
    std::vector<CGCol> hcg(cg->count * kBatchMaxW);
    int outer = 0, inner = 0, launches = 0, converged = 0;
    double worst = 0.0;
    for (;;) {
        // r64 = b - A x (float64), ||r64||^2 per column
        SP_TRY(batch_launch(cg->b64, SP_SPMV_SCALE | SP_SPMV_AXPBY | SP_SPMV_DOT_YY, -1.0, 1.0, s));
        k_outer_scalars<<<cg->count, 32 * kBatchMaxW, 0, s>>>((const BMat *)cg->b64.dmats->ptr,
                                                              (const double *)cg->b64.partials->ptr, cg->count, o.tol,
                                                              outer == 0, (OuterCol *)cg->outer->ptr,
                                                              (CGCol *)cg->cgcol->ptr);
        SP_CUDA(cudaGetLastError());
        SP_CUDA(cudaMemcpyAsync(hoc.data(), cg->outer->ptr, hoc.size() * sizeof(OuterCol), cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
        int active = 0;
        worst = 0.0;
        for (int m = 0; m < cg->count; ++m)
            for (int k = 0; k < cg->widths[m]; ++k) {
                active += hoc[m * kBatchMaxW + k].active;
                worst = std::max(worst, hoc[m * kBatchMaxW + k].rel);
            }
        if (!active) {
            converged = 1;
            break;
        }
        if (outer >= o.max_outer) break;
        ++outer;
        if (f64)
            k_start_inner<double><<<gv, 256, 0, s>>>((const VUnit *)cg->dvunits->ptr, nu, dvec,
                                                     (const OuterCol *)cg->outer->ptr);
        else
            k_start_inner<float><<<gv, 256, 0, s>>>((const VUnit *)cg->dvunits->ptr, nu, dvec,
                                                    (const OuterCol *)cg->outer->ptr);
        SP_CUDA(cudaGetLastError());
        int done_inner = 0;
        while (done_inner < o.max_inner) {
            SP_CUDA(cudaGraphLaunch(cg->graph[f64], s));
            ++launches;
            done_inner += o.graph_iters;
            SP_CUDA(cudaMemcpyAsync(hcg.data(), cg->cgcol->ptr, hcg.size() * sizeof(CGCol), cudaMemcpyDeviceToHost, s));
            SP_CUDA(cudaStreamSynchronize(s));
            int act = 0;
            for (int m = 0; m < cg->count; ++m)
                for (int k = 0; k < cg->widths[m]; ++k) act += hcg[m * kBatchMaxW + k].active;
            if (!act) break;
        }
        int maxit = 0;
        for (auto &c : hcg) maxit = std::max(maxit, (int)c.it);
        inner += maxit;
        if (f64)
            k_x_update<double><<<gv, 256, 0, s>>>((const VUnit *)cg->dvunits->ptr, nu, dvec,
                                                  (const OuterCol *)cg->outer->ptr);
        else
            k_x_update<float><<<gv, 256, 0, s>>>((const VUnit *)cg->dvunits->ptr, nu, dvec,
                                                 (const OuterCol *)cg->outer->ptr);
        SP_CUDA(cudaGetLastError());
    }
    for (int m = 0; m < cg->count; ++m) {
        int64_t n = cg->nrows[m] * cg->widths[m];
        SP_CUDA(cudaMemcpyAsync(x[m], cg->hvec64[m].x, n * 8, cudaMemcpyDeviceToDevice, s));
    }
    SP_CUDA(cudaStreamSynchronize(s));
    if (rel_res) {
        int q = 0;
        for (int m = 0; m < cg->count; ++m)
            for (int k = 0; k < cg->widths[m]; ++k) rel_res[q++] = hoc[m * kBatchMaxW + k].rel;
    }
    if (stats) {
        stats->outer = outer;
        stats->inner = inner;
        stats->graph_launches = launches;
        stats->converged = converged;
        stats->max_rel_residual = worst;
    }
    return SP_OK;
}

int sp_cg_destroy(sp_cg *cg, void *stream) {
    if (!cg) return SP_ERR_ARG;
    cudaStreamSynchronize((cudaStream_t)stream);
    if (cg->stream) cudaStreamSynchronize(cg->stream);
    for (int f = 0; f < 2; ++f)
        if (cg->graph[f]) cudaGraphExecDestroy(cg->graph[f]);
    for (sp_mat *m : cg->A32) sp_mat_destroy(m, stream);
    if (cg->stream) cudaStreamDestroy(cg->stream);
    delete cg;
    return SP_OK;
}

}  // extern "C"
