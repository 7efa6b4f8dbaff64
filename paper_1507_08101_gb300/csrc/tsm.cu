// Tall and skinny block-vector kernels (the dense-matrix section of the paper:
// V is n x m, W is n x k with m, k << n, X is m x k):
//     tsmttsm:  X <- alpha V^T W + beta X   (inner products of block vectors;
//               with a Kahan-compensated variant for large n)
//     tsmm:     W <- alpha V X + beta W      (also in place, W = V, k = m)
// Row-major blocks on the device, m, k <= 32.  Both stream V and W once.
//
// The paper notes that these products should be memory bound for large n.
// On this GPU that holds in float32; in float64 the FP64 pipe (2 fused
// multiply-adds per SM and cycle) binds once m * k reaches a few dozen, so the
// kernels aim at keeping that pipe busy rather than at fewer bytes.
//
// Both kernels stream tiles of rows into shared memory with cp.async: while a
// block works on tile i the copy of tile i + 1 is in flight (tsmttsm through a
// ring of kTsmStages buffers, tsmm through two).  Each block takes a
// contiguous run of tiles.
//
// tsmttsm: each thread owns an RA x RB block of the outputs; LA x LB threads
// cover the (padded) m x k result and the 256 / (LA LB) groups of such threads
// take different rows of the tile.  Per row a thread reads RA values of V and
// RB values of W (vector loads from shared memory) and does RA RB multiply-adds
// (or Kahan steps).  The groups are summed in a fixed order inside the block,
// the blocks in a fixed order by a second kernel, so results do not depend on
// timing; the Kahan variant carries (sum, compensation) pairs through both
// reductions.
//
// tsmm: each thread keeps an MP x RB slice of X in registers and produces RB
// outputs of one row at a time from the row of V in shared memory; a row of W
// is written only after its tile of V is in shared memory, so the in-place
// form reads every row before it overwrites it.
#include <algorithm>

#include "common.cuh"

namespace sp {

constexpr int kTsmThreads = 256;
constexpr int kTsmMax = 32;
constexpr int kTsmStages = 2;           // tiles per block in shared memory (ring)
constexpr int kTsmTileBytes = 24576;    // bytes of V (and W) per staged tile
constexpr int kTsmMaxBlocksPerSm = 4;
constexpr size_t kTsmSmemMax = 48 * 1024;  // dynamic shared memory without an opt-in attribute
// 1: tiles of dense blocks move by one bulk copy each (cp.async.bulk + mbarrier)
#ifndef SP_TSM_BULK
#define SP_TSM_BULK 1
#endif

// ------------------------------------------------------------------ cp.async staging
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copy rows [row0, row0 + rows) x columns [0, cols) of a row-major block with
// leading dimension ld into shared memory with row stride dstride.  vec: every
// row is a whole number of 16-byte pieces, 16-byte aligned on both sides.
template <class T>
__device__ __forceinline__ void stage_rows(T *dst, int dstride, const T *__restrict__ src, int64_t ld,
                                           int64_t row0, int rows, int cols, bool vec) {
    const int e0 = threadIdx.x;
    if (vec) {
        constexpr int E = 16 / sizeof(T);
        const int cpr = cols / E;  // 16-byte pieces per row
        int r = e0 / cpr, c = e0 - r * cpr;
        const int dr = kTsmThreads / cpr, dc = kTsmThreads - dr * cpr;
        while (r < rows) {
            cp_async<16>(dst + r * dstride + c * E, src + (row0 + r) * ld + c * E);
            r += dr;
            c += dc;
            if (c >= cpr) {
                c -= cpr;
                ++r;
            }
        }
    } else {
        int r = e0 / cols, c = e0 - r * cols;
        const int dr = kTsmThreads / cols, dc = kTsmThreads - dr * cols;
        while (r < rows) {
            cp_async<(int)sizeof(T)>(dst + r * dstride + c, src + (row0 + r) * ld + c);
            r += dr;
            c += dc;
            if (c >= cols) {
                c -= cols;
                ++r;
            }
        }
    }
}

// Copy `pieces` 16-byte pieces from src to dst (rows that are one contiguous
// run on both sides: ld == cols == the shared-memory row stride).
template <class T>
__device__ __forceinline__ void stage_contig(T *dst, const T *__restrict__ src, int pieces) {
    constexpr int E = 16 / sizeof(T);
    for (int e = threadIdx.x; e < pieces; e += kTsmThreads) cp_async<16>(dst + e * E, src + e * E);
}

// ------------------------------------------------------------------ bulk-copy staging
// One thread copies a whole tile of rows that are contiguous in global memory
// with one cp.async.bulk (the copy engine moves it; no per-thread copy
// instructions), completing on the stage's mbarrier with the tile's byte
// count.  Waits are bounded: a wait that runs out records the failure in the
// call's status word (the final kernel then writes NaN into X) and the block
// stops working on its tiles.
constexpr int kTsmBulkStages = 4;
constexpr int kTsmBulkTileBytes = 12288;
// The Kahan variant (four operations per term) gains from fewer, larger
// tiles: 3 x 16 KB measured 247 against 259 us (n = 2^22, m = k = 16,
// float32); the plain one does not (110.5 against 109.7 us).
constexpr int kTsmBulkStagesKahan = 3;
constexpr int kTsmBulkTileBytesKahan = 16384;
template <bool KAHAN>
constexpr int tsm_bulk_stages() { return KAHAN ? kTsmBulkStagesKahan : kTsmBulkStages; }
template <bool KAHAN>
constexpr int tsm_bulk_tile_bytes() { return KAHAN ? kTsmBulkTileBytesKahan : kTsmBulkTileBytes; }
constexpr unsigned kTsmWaitTries = 1u << 22;  // try_wait rounds (each suspends for a while) before giving up

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_to_smem(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// true when the phase with this parity completed within the bound
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
    for (unsigned i = 0; i < kTsmWaitTries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// N consecutive elements from 16-byte-aligned (N * sizeof(T) >= 16) or
// N * sizeof(T)-aligned shared memory.
template <class T, int N>
__device__ __forceinline__ void ld_vec(const T *p, T *out) {
    constexpr int B = N * (int)sizeof(T);
    if constexpr (B >= 16) {
        constexpr int E = 16 / sizeof(T);
#pragma unroll
        for (int q = 0; q < N / E; ++q) {
            const float4 v = *reinterpret_cast<const float4 *>(p + q * E);
            const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int i = 0; i < E; ++i) out[q * E + i] = pv[i];
        }
    } else if constexpr (B == 8) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = pv[i];
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = p[i];
    }
}

// (sum, compensation) pair: the represented value is s + c.  merge adds
// another pair with the exact error of s1 + s2 (Knuth's TwoSum) kept in c.
struct Comp {
    double s, c;
};
__device__ __forceinline__ Comp comp_merge(Comp a, Comp b) {
    const double t = a.s + b.s;
    const double bv = t - a.s;
    const double e = (a.s - (t - bv)) + (b.s - bv);
    return Comp{t, (a.c + b.c) + e};
}

// Rows per staged tile for `row_bytes` bytes of shared memory per row.
inline int tile_rows(int row_bytes, int tile_bytes = kTsmTileBytes) {
    int tr = tile_bytes / row_bytes;
    tr = std::max(32, std::min(1024, tr / 32 * 32));
    return tr;
}

// ------------------------------------------------------------------ tsmttsm
// acc[i RB + j] += va[i] wb[j] (Kahan: cmp carries the low-order part lost by
// the last addition of each sum)
template <class T, bool KAHAN, int RA, int RB>
__device__ __forceinline__ void outer_acc(T (&acc)[RA * RB], T (&cmp)[RA * RB], const T (&va)[RA],
                                          const T (&wb)[RB]) {
#pragma unroll
    for (int i = 0; i < RA; ++i)
#pragma unroll
        for (int j = 0; j < RB; ++j) {
            const int x = i * RB + j;
            if constexpr (KAHAN) {
                const T yv = va[i] * wb[j] - cmp[x];
                const T tv = acc[x] + yv;
                cmp[x] = (tv - acc[x]) - yv;
                acc[x] = tv;
            } else {
                acc[x] = fma(va[i], wb[j], acc[x]);
            }
        }
}

// part[(a * k + b) * nb + block] = (s, c) of the block's sum for output (a, b)
template <class T, bool KAHAN, int RA, int RB, int LA, int LB, bool BULK>
__global__ void __launch_bounds__(kTsmThreads, RA * RB > 16 ? 1 : (KAHAN ? 2 : 4)) k_tsmttsm_tile(const T *__restrict__ V, int64_t ldv,
                                                              const T *__restrict__ W, int64_t ldw, int64_t n, int m,
                                                              int k, int tr, int64_t tiles_per_block, int vec,
                                                              Comp *__restrict__ part, unsigned *status) {
    constexpr int L = LA * LB, G = kTsmThreads / L, MPs = LA * RA, KPs = LB * RB, RR = RA * RB;
    constexpr int S = BULK ? tsm_bulk_stages<KAHAN>() : kTsmStages;
    extern __shared__ __align__(16) unsigned char tsm_smem[];
    T *const st = reinterpret_cast<T *>(tsm_smem);
    const int t = threadIdx.x, l = t % L, g = t / L, ia = l / LB, ib = l % LB;
    const int stage_elems = tr * (MPs + KPs);
    // BULK: the rows of V and W are contiguous and fill the tile's rows (no
    // padding columns); the stages' mbarriers follow the tiles
    uint64_t *const bars = reinterpret_cast<uint64_t *>(st + S * stage_elems);
    if constexpr (!BULK) {
        // padding columns (never written by the copies) hold zeros
        for (int e = t; e < kTsmStages * stage_elems; e += kTsmThreads) {
            const int o = e % stage_elems;
            const bool pad = o < tr * MPs ? (o % MPs) >= m : ((o - tr * MPs) % KPs) >= k;
            if (pad) st[e] = T(0);
        }
    } else {
        if (t == 0) {
            for (int i = 0; i < S; ++i) mbar_init(&bars[i], 1);
            mbar_fence_init();
        }
    }
    __shared__ int failed;  // a copy wait ran out (bulk staging)
    if (t == 0) failed = 0;
    __syncthreads();
    T acc[RR], cmp[RR];
#pragma unroll
    for (int x = 0; x < RR; ++x) acc[x] = cmp[x] = T(0);
    const int64_t ntiles = (n + tr - 1) / tr;
    const int64_t tile0 = (int64_t)blockIdx.x * tiles_per_block;
    const int64_t tile1 = ntiles < tile0 + tiles_per_block ? ntiles : tile0 + tiles_per_block;
    // the compute of one staged tile (rows g, g + G, ...: two per step)
    auto work = [&](int si, int64_t tile) {
        const T *sv = st + si * stage_elems, *sw = sv + tr * MPs;
        const int rows = (int)(n - tile * tr < tr ? n - tile * tr : tr);
        const T *pv = sv + g * MPs + ia * RA, *pw = sw + g * KPs + ib * RB;
        int r = g;
        for (; r + G < rows; r += 2 * G, pv += 2 * G * MPs, pw += 2 * G * KPs) {
            T va0[RA], wb0[RB], va1[RA], wb1[RB];
            ld_vec<T, RA>(pv, va0);
            ld_vec<T, RB>(pw, wb0);
            ld_vec<T, RA>(pv + G * MPs, va1);
            ld_vec<T, RB>(pw + G * KPs, wb1);
            outer_acc<T, KAHAN, RA, RB>(acc, cmp, va0, wb0);
            outer_acc<T, KAHAN, RA, RB>(acc, cmp, va1, wb1);
        }
        if (r < rows) {
            T va[RA], wb[RB];
            ld_vec<T, RA>(pv, va);
            ld_vec<T, RB>(pw, wb);
            outer_acc<T, KAHAN, RA, RB>(acc, cmp, va, wb);
        }
    };
    if constexpr (BULK) {
        // thread 0 keeps up to S tiles in flight; tile i lands in stage i mod S,
        // whose mbarrier completes its (i / S)-th phase
        auto issue = [&](int64_t tile, int si) {
            T *sv = st + si * stage_elems, *sw = sv + tr * MPs;
            const int64_t r0 = tile * tr;
            const int rows = (int)(n - r0 < tr ? n - r0 : tr);
            const unsigned bv = (unsigned)(rows * m * (int)sizeof(T)), bw = (unsigned)(rows * k * (int)sizeof(T));
            mbar_expect_tx(&bars[si], bv + bw);
            bulk_to_smem(sv, V + r0 * ldv, bv, &bars[si]);
            bulk_to_smem(sw, W + r0 * ldw, bw, &bars[si]);
        };
        if (t == 0)
            for (int i = 0; i < S && tile0 + i < tile1; ++i) issue(tile0 + i, i);
        int64_t tile = tile0;
        for (; tile < tile1; ++tile) {
            const int it = (int)(tile - tile0), si = it % S;
            if (!mbar_wait_bounded(&bars[si], (unsigned)(it / S) & 1u)) atomicOr(&failed, 1);
            __syncthreads();
            if (failed) break;
            work(si, tile);
            __syncthreads();  // every thread is done with stage si
            if (t == 0 && tile + S < tile1) {
                fence_proxy_async_smem();
                issue(tile + S, si);
            }
        }
        if (failed) {
            // leave no copy running into this block's shared memory: wait
            // (bounded) for every tile issued after the one that failed
            if (t == 0) {
                for (int64_t u = tile; u < tile1 && u < tile + S; ++u) {
                    const int iu = (int)(u - tile0);
                    mbar_wait_bounded(&bars[iu % S], (unsigned)(iu / S) & 1u);
                }
            }
            __syncthreads();
        }
    }
    // rows of V (W) that are contiguous in memory and fill the tile's rows exactly
    const bool dense_v = (vec & 1) && ldv == m && MPs == m, dense_w = (vec & 2) && ldw == k && KPs == k;
    auto stage = [&](int64_t tile, int s) {
        T *sv = st + s * stage_elems, *sw = sv + tr * MPs;
        const int64_t r0 = tile * tr;
        const int rows = (int)(n - r0 < tr ? n - r0 : tr);
        if (dense_v)
            stage_contig(sv, V + r0 * ldv, rows * (MPs * (int)sizeof(T) / 16));
        else
            stage_rows(sv, MPs, V, ldv, r0, rows, m, vec & 1);
        if (dense_w)
            stage_contig(sw, W + r0 * ldw, rows * (KPs * (int)sizeof(T) / 16));
        else
            stage_rows(sw, KPs, W, ldw, r0, rows, k, (vec & 2) != 0);
    };
    if constexpr (!BULK) {
        // one commit group per tile (empty past the end), so that waiting for all
        // but the newest kTsmStages - 1 groups leaves this tile complete
#pragma unroll
        for (int i = 0; i < kTsmStages - 1; ++i) {
            if (tile0 + i < tile1) stage(tile0 + i, i);
            cp_async_commit();
        }
        for (int64_t tile = tile0; tile < tile1; ++tile) {
            const int it = (int)(tile - tile0), si = it % kTsmStages;
            if (tile + kTsmStages - 1 < tile1) stage(tile + kTsmStages - 1, (it + kTsmStages - 1) % kTsmStages);
            cp_async_commit();
            cp_async_wait<kTsmStages - 1>();
            __syncthreads();
            work(si, tile);
            __syncthreads();
        }
    }
    // Reduction, four outputs at a time (few registers live): the row groups
    // inside a warp (lanes l, l + L, ...) by a fixed xor tree, then the
    // block's warps in order, into shared memory (reusing the tiles).
    Comp *red = reinterpret_cast<Comp *>(tsm_smem);
    const int warp = t >> 5, lane = t & 31;
#pragma unroll
    for (int x0 = 0; x0 < RR; x0 += 4) {
        Comp cs[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) cs[q] = Comp{(double)acc[x0 + q], KAHAN ? -(double)cmp[x0 + q] : 0.0};
#pragma unroll
        for (int off = L; off < 32; off <<= 1)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const Comp o{__shfl_xor_sync(0xffffffffu, cs[q].s, off), __shfl_xor_sync(0xffffffffu, cs[q].c, off)};
                if constexpr (KAHAN)
                    cs[q] = comp_merge(cs[q], o);
                else
                    cs[q].s += o.s;
            }
        for (int w = 0; w < kTsmThreads / 32; ++w) {
            if (warp == w && lane < L) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    Comp &d = red[lane * RR + x0 + q];
                    if (w == 0)
                        d = cs[q];
                    else if (KAHAN)
                        d = comp_merge(d, cs[q]);
                    else
                        d.s += cs[q].s;
                }
            }
            __syncthreads();
        }
    }
    const int nb = gridDim.x;
    for (int o = t; o < L * RR; o += kTsmThreads) {
        const int ll = o / RR, x = o - ll * RR;
        const int a = (ll / LB) * RA + x / RB, b = (ll % LB) * RB + x % RB;
        if (a < m && b < k) part[(int64_t)(a * k + b) * nb + blockIdx.x] = red[o];
    }
    // this block's status word (1: a copy wait ran out), written by every block
    if (t == 0) status[blockIdx.x] = failed ? 1u : 0u;
}

// X[a, b] = alpha * (sum over blocks, in order) + beta X[a, b]: one warp per output
template <class T, bool KAHAN>
__global__ void k_tsmttsm_final(const Comp *__restrict__ part, int nb, int m, int k, double alpha, double beta,
                                T *__restrict__ X, int64_t ldx, const unsigned *status) {
    const int e = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (e >= m * k) return;  // whole warps leave together
    const Comp *p = part + (int64_t)e * nb;
    Comp acc{0.0, 0.0};
    // the lane's partials in block order, four loads in flight at a time
    for (int b0 = lane; b0 < nb; b0 += 4 * 32) {
        Comp v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int bl = b0 + q * 32;
            v[q] = bl < nb ? p[bl] : Comp{0.0, 0.0};
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (b0 + q * 32 < nb) {
                if constexpr (KAHAN)
                    acc = comp_merge(acc, v[q]);
                else
                    acc.s += v[q].s;
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const Comp o{__shfl_xor_sync(0xffffffffu, acc.s, off), __shfl_xor_sync(0xffffffffu, acc.c, off)};
        if constexpr (KAHAN)
            acc = comp_merge(acc, o);
        else
            acc.s += o.s;
    }
    // a tile block that gave up waiting for its copies poisons the result
    bool bad = false;
    for (int bl = lane; bl < nb; bl += 32) bad |= status[bl] != 0u;
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        const int a = e / k, b = e - a * k;
        T *xp = X + (int64_t)a * ldx + b;
        const double old = beta != 0.0 ? (double)*xp : 0.0;
        *xp = bad ? (T)NAN : (T)(alpha * (acc.s + acc.c) + beta * old);
    }
}

// ------------------------------------------------------------------ tsmm
// Lanes per row LB = 2^lbs cover the k outputs of a row in slices of RB; the
// 256 / LB rows a block works on at once are the row groups.
template <class T, int MP, int RB>
__global__ void __launch_bounds__(kTsmThreads) k_tsmm_tile(const T *V, int64_t ldv,
                                                           const T *__restrict__ X, int64_t ldx, T *W, int64_t ldw,
                                                           int64_t n, int m, int k, int lbs, int tr,
                                                           int64_t tiles_per_block, int vec, T alpha, T beta) {
    constexpr int VW = 16 / (int)sizeof(T);  // elements per 16-byte shared-memory load
    constexpr int MPs = MP + VW;             // padded row stride of the V tile (spreads rows over banks)
    extern __shared__ __align__(16) unsigned char tsm_smem[];
    T *const st = reinterpret_cast<T *>(tsm_smem);
    const int t = threadIdx.x, q = t & ((1 << lbs) - 1), g = t >> lbs, G = kTsmThreads >> lbs;
    const int b0 = q * RB;
    T xr[MP][RB];
#pragma unroll
    for (int a = 0; a < MP; ++a)
#pragma unroll
        for (int j = 0; j < RB; ++j) xr[a][j] = (a < m && b0 + j < k) ? X[(int64_t)a * ldx + b0 + j] : T(0);
    const int stage_elems = tr * MPs;
    for (int e = t; e < 2 * stage_elems; e += kTsmThreads)
        if ((e % MPs) >= m) st[e] = T(0);  // padding columns: zeros (0 x 0 in the products)
    const int64_t ntiles = (n + tr - 1) / tr;
    const int64_t tile0 = (int64_t)blockIdx.x * tiles_per_block;
    const int64_t tile1 = ntiles < tile0 + tiles_per_block ? ntiles : tile0 + tiles_per_block;
    auto stage = [&](int64_t tile, int s) {
        const int64_t r0 = tile * tr;
        const int rows = (int)(n - r0 < tr ? n - r0 : tr);
        stage_rows(st + s * stage_elems, MPs, V, ldv, r0, rows, m, vec != 0);
        cp_async_commit();
    };
    // two tiles: the copy of tile i + 1 overlaps the products of tile i
    if (tile0 < tile1) stage(tile0, 0);
    for (int64_t tile = tile0; tile < tile1; ++tile) {
        const int s = (int)((tile - tile0) & 1);
        if (tile + 1 < tile1) {
            stage(tile + 1, s ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();  // the tile of V is in shared memory before W (which may be V) is written
        const T *sv = st + s * stage_elems;
        const int64_t r0 = tile * tr;
        const int rows = (int)(n - r0 < tr ? n - r0 : tr);
        for (int r = g; r < rows; r += G) {
            T out[RB];
#pragma unroll
            for (int j = 0; j < RB; ++j) out[j] = T(0);
#pragma unroll
            for (int a0 = 0; a0 < MP; a0 += VW) {
                T v[VW];
                ld_vec<T, VW>(sv + r * MPs + a0, v);
#pragma unroll
                for (int i = 0; i < VW; ++i)
#pragma unroll
                    for (int j = 0; j < RB; ++j) out[j] = fma(v[i], xr[a0 + i][j], out[j]);
            }
            T *wp = W + (r0 + r) * ldw + b0;
#pragma unroll
            for (int j = 0; j < RB; ++j)
                if (b0 + j < k) {
                    const T old = beta != T(0) ? wp[j] : T(0);
                    wp[j] = fma(alpha, out[j], beta * old);
                }
        }
        __syncthreads();  // before the next copies overwrite this stage
    }
}

static int sms_count() {
    int sms = 1;
    device_sm_count(&sms);
    return sms;
}

// blocks for a grid of contiguous tile runs: SMs x resident blocks (at most
// kTsmMaxBlocksPerSm), no more than there are tiles
template <class K>
static int tsm_grid(K kernel, size_t smem, int64_t ntiles, int64_t *tiles_per_block) {
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kTsmThreads, smem) != cudaSuccess || occ < 1)
        occ = 1;
    const int64_t want = (int64_t)sms_count() * std::min(occ, kTsmMaxBlocksPerSm);
    const int64_t nb0 = std::max<int64_t>(1, std::min<int64_t>(want, ntiles));
    *tiles_per_block = (ntiles + nb0 - 1) / nb0;
    return (int)std::max<int64_t>(1, (ntiles + *tiles_per_block - 1) / *tiles_per_block);
}

static bool vec16_ok(const void *p, int64_t ld, int cols, size_t es) {
    return ((uintptr_t)p % 16) == 0 && (ld * es) % 16 == 0 && (cols * es) % 16 == 0;
}

template <class T, bool KAHAN, int RA, int RB, int LA, int LB>
static int run_tsmttsm(sp_dense *X, const sp_dense *V, const sp_dense *Wd, double alpha, double beta,
                       cudaStream_t s) {
    constexpr int L = LA * LB, RR = RA * RB, MPs = LA * RA, KPs = LB * RB;
    const int64_t n = V->nrows;
    const int m = V->ncols, k = Wd->ncols;
    const int vec = (vec16_ok(V->ptr, V->ld, m, sizeof(T)) ? 1 : 0) | (vec16_ok(Wd->ptr, Wd->ld, k, sizeof(T)) ? 2 : 0);
    // both blocks dense (rows contiguous, 16-byte multiples, no padding
    // columns): one bulk copy per tile and block vector
    const bool bulk = SP_TSM_BULK && vec == 3 && V->ld == m && MPs == m && Wd->ld == k && KPs == k;
    const int S = bulk ? tsm_bulk_stages<KAHAN>() : kTsmStages;
    const int tr = tile_rows((MPs + KPs) * (int)sizeof(T), bulk ? tsm_bulk_tile_bytes<KAHAN>() : kTsmTileBytes);
    const size_t smem = std::max<size_t>((size_t)S * tr * (MPs + KPs) * sizeof(T) + (bulk ? S * sizeof(uint64_t) : 0),
                                         (size_t)L * RR * sizeof(Comp));
    const int64_t ntiles = std::max<int64_t>(1, (n + tr - 1) / tr);
    if (smem > kTsmSmemMax + 1024) return SP_ERR_UNSUPPORTED;  // not reached: tiles are bounded in bytes
    auto kern = bulk ? k_tsmttsm_tile<T, KAHAN, RA, RB, LA, LB, true> : k_tsmttsm_tile<T, KAHAN, RA, RB, LA, LB, false>;
    if (smem > kTsmSmemMax) SP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t tpb = 1;
    const int nb = tsm_grid(kern, smem, ntiles, &tpb);
    Tmp part(s);  // stream-ordered: no device-wide synchronisation per call
    const size_t pbytes = (size_t)nb * m * k * sizeof(Comp);
    SP_TRY(part.alloc(pbytes + (size_t)nb * sizeof(unsigned)));
    unsigned *status = reinterpret_cast<unsigned *>(part.as<char>() + pbytes);  // one word per tile block
    kern<<<nb, kTsmThreads, smem, s>>>((const T *)V->ptr, V->ld, (const T *)Wd->ptr, Wd->ld, n, m, k, tr, tpb, vec,
                                       part.as<Comp>(), status);
    const int fin_blocks = (m * k * 32 + 255) / 256;
    k_tsmttsm_final<T, KAHAN><<<fin_blocks, 256, 0, s>>>(part.as<const Comp>(), nb, m, k, alpha, beta, (T *)X->ptr,
                                                         X->ld, status);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

template <class T, bool KAHAN>
static int dispatch_tsmttsm(sp_dense *X, const sp_dense *V, const sp_dense *W, double alpha, double beta,
                            cudaStream_t s) {
    const int p = std::max(V->ncols, W->ncols);
    if (p <= 2) return run_tsmttsm<T, KAHAN, 2, 2, 1, 1>(X, V, W, alpha, beta, s);
    if (p <= 4) return run_tsmttsm<T, KAHAN, 4, 4, 1, 1>(X, V, W, alpha, beta, s);
    if (p <= 8) return run_tsmttsm<T, KAHAN, 4, 4, 2, 2>(X, V, W, alpha, beta, s);
    if (p <= 16) return run_tsmttsm<T, KAHAN, 4, 4, 4, 4>(X, V, W, alpha, beta, s);
    return run_tsmttsm<T, KAHAN, 4, 8, 8, 4>(X, V, W, alpha, beta, s);
}

template <class T, int MP>
static int run_tsmm(sp_dense *W, const sp_dense *V, const sp_dense *X, double alpha, double beta, cudaStream_t s) {
    // slices of X in registers: MP x RB values per thread
    constexpr int RB = (sizeof(T) == 8 && MP == 32) ? 2 : 4;
    constexpr int MPs = MP + 16 / (int)sizeof(T);
    const int64_t n = V->nrows;
    const int m = V->ncols, k = W->ncols;
    int lbs = 0;
    while ((1 << lbs) * RB < k) ++lbs;
    const int tr = tile_rows(MPs * (int)sizeof(T));
    const size_t smem = (size_t)2 * tr * MPs * sizeof(T);
    const int64_t ntiles = std::max<int64_t>(1, (n + tr - 1) / tr);
    if (smem > kTsmSmemMax) return SP_ERR_UNSUPPORTED;
    auto kern = k_tsmm_tile<T, MP, RB>;
    int64_t tpb = 1;
    const int nb = tsm_grid(kern, smem, ntiles, &tpb);
    const int vec = vec16_ok(V->ptr, V->ld, m, sizeof(T)) ? 1 : 0;
    kern<<<nb, kTsmThreads, smem, s>>>((const T *)V->ptr, V->ld, (const T *)X->ptr, X->ld, (T *)W->ptr, W->ld, n, m,
                                       k, lbs, tr, tpb, vec, (T)alpha, (T)beta);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

template <class T>
static int dispatch_tsmm(sp_dense *W, const sp_dense *V, const sp_dense *X, double alpha, double beta,
                         cudaStream_t s) {
    const int m = V->ncols;
    if (m <= 4) return run_tsmm<T, 4>(W, V, X, alpha, beta, s);
    if (m <= 8) return run_tsmm<T, 8>(W, V, X, alpha, beta, s);
    if (m <= 16) return run_tsmm<T, 16>(W, V, X, alpha, beta, s);
    return run_tsmm<T, 32>(W, V, X, alpha, beta, s);
}

}  // namespace sp

static bool rowmajor_dev(const sp_dense *d) { return d && d->layout == SP_ROW_MAJOR && d->ptr; }

int sp_tsmttsm(sp_dense *X, const sp_dense *V, const sp_dense *W, double alpha, double beta, int kahan,
               void *stream) {
    if (sp::dense_scattered(X) || sp::dense_scattered(V) || sp::dense_scattered(W))
        return sp::scattered_refused("sp_tsmttsm");
    if (!rowmajor_dev(X) || !rowmajor_dev(V) || !rowmajor_dev(W)) return SP_ERR_ARG;
    if (V->nrows != W->nrows || X->nrows != V->ncols || X->ncols != W->ncols) return SP_ERR_DIM;
    if (V->dtype != W->dtype || X->dtype != V->dtype || (V->dtype != SP_F64 && V->dtype != SP_F32))
        return SP_ERR_DTYPE;
    const int m = V->ncols, k = W->ncols;
    if (m < 1 || k < 1) return SP_ERR_ARG;
    if (m > sp::kTsmMax || k > sp::kTsmMax) return SP_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if (V->dtype == SP_F64)
        return kahan ? sp::dispatch_tsmttsm<double, true>(X, V, W, alpha, beta, s)
                     : sp::dispatch_tsmttsm<double, false>(X, V, W, alpha, beta, s);
    return kahan ? sp::dispatch_tsmttsm<float, true>(X, V, W, alpha, beta, s)
                 : sp::dispatch_tsmttsm<float, false>(X, V, W, alpha, beta, s);
}

int sp_tsmm(sp_dense *W, const sp_dense *V, const sp_dense *X, double alpha, double beta, void *stream) {
    if (sp::dense_scattered(W) || sp::dense_scattered(V) || sp::dense_scattered(X)) return sp::scattered_refused("sp_tsmm");
    if (!rowmajor_dev(X) || !rowmajor_dev(V) || !rowmajor_dev(W)) return SP_ERR_ARG;
    if (V->nrows != W->nrows || X->nrows != V->ncols || X->ncols != W->ncols) return SP_ERR_DIM;
    if (V->dtype != W->dtype || X->dtype != V->dtype || (V->dtype != SP_F64 && V->dtype != SP_F32))
        return SP_ERR_DTYPE;
    const int m = V->ncols, k = W->ncols;
    if (m < 1 || k < 1) return SP_ERR_ARG;
    if (m > sp::kTsmMax || k > sp::kTsmMax) return SP_ERR_UNSUPPORTED;
    const bool inplace = W->ptr == V->ptr;
    if (inplace && (W->ld != V->ld || m != k)) return SP_ERR_ARG;
    // a partial overlap of W with V or X (other than the in-place form) is refused
    const size_t xs = V->dtype == SP_F64 ? 8 : 4;
    auto span = [&](const sp_dense *d) { return (size_t)d->ld * d->nrows * xs; };
    auto overl = [&](const sp_dense *a, const sp_dense *b) {
        const char *pa = (const char *)a->ptr, *pb = (const char *)b->ptr;
        return pa < pb + span(b) && pb < pa + span(a);
    };
    if ((!inplace && overl(W, V)) || overl(W, X)) return SP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (V->dtype == SP_F64) return sp::dispatch_tsmm<double>(W, V, X, alpha, beta, s);
    return sp::dispatch_tsmm<float>(W, V, X, alpha, beta, s);
}
