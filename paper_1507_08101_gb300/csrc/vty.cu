// The augmented product fused with the inner products of a tall and skinny
// block V with the new y (the dense-matrix section's X = V^T W with W = y):
//
//     y = alpha (A - gamma I) x + beta y,   z = delta z + eta y,   C = V^T y
//
// in one pass, for block orthogonalisation after a product (the coefficients
// of y against a basis V are formed while y is written, instead of in a second
// pass over y).  Float64 values and vectors; V is n x m, y is n x w, C is
// m x w, with m <= 8 and w <= 8.
//
// Each lane keeps the m x CPL products V[i, a] y[i, k0 + c] of its rows in
// registers; at the end the lanes of a column group are added by a fixed xor
// tree, the warps of a block in order, and the blocks in order by the last
// block to finish (atomic ticket, no waiting), so C does not depend on timing.
#include <algorithm>
#include <vector>

#include "spmv_kernel.cuh"

namespace sp {

constexpr int kVtyThreads = 256;
constexpr int kVtyWarps = kVtyThreads / 32;
constexpr int kVtyMaxM = 8, kVtyMaxW = 8;

template <int WP, int MP>
__global__ void __launch_bounds__(kVtyThreads, 2)
    k_spmmv_vty(const __grid_constant__ SpmvArgs a, const double *__restrict__ V, int64_t ldv, int m, double *C,
                int64_t ldc) {
    constexpr int CPL = cols_per_lane<double, WP>();
    constexpr int G = WP / CPL;
    constexpr int R = 32 / G;
    constexpr int U = CPL >= 4 ? SP_UNROLL_WIDE : SP_UNROLL_NARROW / CPL;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % G, rw = lane / G;
    const int k0 = gl * CPL;
    const int nvalid = a.w - k0 < CPL ? a.w - k0 : CPL;
    const uint32_t f = a.flags;
    const bool shift = (f & (SP_SPMV_SHIFT | SP_SPMV_VSHIFT)) != 0;
    const bool do_scale = (f & SP_SPMV_SCALE) != 0, do_axpby = (f & SP_SPMV_AXPBY) != 0;
    const bool do_chain = (f & SP_SPMV_CHAIN_AXPBY) != 0;
    const double *__restrict__ val = (const double *)a.val;
    const double *__restrict__ xk = (const double *)a.x + k0;
    double *y = (double *)a.y;
    double *z = (double *)a.z;
    double gam[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) gam[c] = (shift && k0 + c < a.w) ? a.gamma[k0 + c] : 0.0;
    double acc2[MP][CPL];
#pragma unroll
    for (int p = 0; p < MP; ++p)
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc2[p][c] = 0.0;

    const int rows_per_block = R * kVtyWarps;
    for (int64_t base = (int64_t)blockIdx.x * rows_per_block; base < a.nslots;
         base += (int64_t)gridDim.x * rows_per_block) {
        const int64_t s = base + warp * R + rw;
        if (s >= a.nslots) continue;
        const int64_t i = a.perm ? (int64_t)a.perm[s] : (s < a.nrows ? s : -1);
        if (i < 0) continue;
        const uint32_t cidx = (uint32_t)s / (uint32_t)a.C;
        const int64_t off = a.chunkptr[cidx] + (int64_t)((uint32_t)s - cidx * (uint32_t)a.C);
        const int len = a.slotlen[s];
        double acc[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[c] = 0.0;
        int bad = 0;
        row_product<double, double, double, CPL, true, U>(val + off, a.col + off, a.C, len, xk, a.xrs, 1, nvalid,
                                                           acc, bad);
        if (nvalid <= 0) continue;
        double xi[CPL], yo[CPL], t[CPL];
        double *yp = y + i * a.yrs + k0;
        if (shift) load_cols<double, CPL, true>(xk + i * a.xrs, 1, nvalid, xi);
        if (do_axpby) load_out<double, CPL, true>(yp, 1, nvalid, yo);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            double v = acc[c];
            if (shift) v = fma_rn(-gam[c], xi[c], v);
            if (do_scale) v = mul_rn(a.alpha, v);
            if (do_axpby) v = fma_rn(a.beta, yo[c], v);
            t[c] = v;
        }
        store_out<double, CPL, true>(yp, 1, nvalid, t);
        if (do_chain) {
            double zo[CPL];
            double *zp = z + i * a.zrs + k0;
            load_out<double, CPL, true>(zp, 1, nvalid, zo);
#pragma unroll
            for (int c = 0; c < CPL; ++c) zo[c] = fma_rn(a.eta, t[c], mul_rn(a.delta, zo[c]));
            store_out<double, CPL, true>(zp, 1, nvalid, zo);
        }
        // this row's share of C = V^T y
        const double *vr = V + i * ldv;
#pragma unroll
        for (int p = 0; p < MP; ++p) {
            if (p < m) {
                const double vv = __ldg(vr + p);
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc2[p][c] = fma_rn(vv, t[c], acc2[p][c]);
            }
        }
    }

    // lanes of a column group (fixed xor tree), warps in order, blocks in order
    __shared__ double sred[kVtyWarps][MP][WP];
    __shared__ int is_last;
#pragma unroll
    for (int p = 0; p < MP; ++p)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
#pragma unroll
            for (int o = G; o < 32; o <<= 1) acc2[p][c] += __shfl_xor_sync(0xffffffffu, acc2[p][c], o);
            if (lane < G) sred[warp][p][k0 + c] = acc2[p][c];
        }
    __syncthreads();
    const int nv = MP * WP, nb = gridDim.x;
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
        const int p = t / WP, k = t - p * WP;
        double sum = 0.0;
        for (int wi = 0; wi < kVtyWarps; ++wi) sum += sred[wi][p][k];
        a.partials[(int64_t)t * nb + blockIdx.x] = sum;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(a.ticket, 1u) == (unsigned)nb - 1u);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int t = warp; t < nv; t += kVtyWarps) {
        const int p = t / WP, k = t - p * WP;
        double sum = 0.0;
        for (int b = lane; b < nb; b += 32) sum += __ldcg(a.partials + (int64_t)t * nb + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0 && p < m && k < a.w) C[(int64_t)p * ldc + k] = sum;
    }
    if (threadIdx.x == 0) *a.ticket = 0u;
}

template <int WP, int MP>
static int launch_vty(const SpmvArgs &a, const double *V, int64_t ldv, int m, double *C, int64_t ldc, int max_blocks,
                      cudaStream_t s) {
    constexpr int CPL = cols_per_lane<double, WP>();
    constexpr int R = 32 / (WP / CPL);
    int sms = 1;
    SP_TRY(device_sm_count(&sms));
    const int64_t need = (a.nslots + (int64_t)R * kVtyWarps - 1) / ((int64_t)R * kVtyWarps);
    // partials: one per (C entry, block); the matrix scratch holds max_blocks x 96
    const int64_t cap = (int64_t)max_blocks * 3 * kMaxTileW / (MP * WP);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>({(int64_t)sms * 2, need, cap}));
    k_spmmv_vty<WP, MP><<<(unsigned)grid, kVtyThreads, 0, s>>>(a, V, ldv, m, C, ldc);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

template <int WP>
static int launch_vty_m(const SpmvArgs &a, const double *V, int64_t ldv, int m, double *C, int64_t ldc,
                        int max_blocks, cudaStream_t s) {
    if (m <= 1) return launch_vty<WP, 1>(a, V, ldv, m, C, ldc, max_blocks, s);
    if (m <= 2) return launch_vty<WP, 2>(a, V, ldv, m, C, ldc, max_blocks, s);
    if (m <= 4) return launch_vty<WP, 4>(a, V, ldv, m, C, ldc, max_blocks, s);
    return launch_vty<WP, 8>(a, V, ldv, m, C, ldc, max_blocks, s);
}

int launch_spmv_vty(const SpmvArgs &a, const double *V, int64_t ldv, int m, double *C, int64_t ldc, int max_blocks,
                    cudaStream_t s) {
    if (a.w <= 1) return launch_vty_m<1>(a, V, ldv, m, C, ldc, max_blocks, s);
    if (a.w <= 2) return launch_vty_m<2>(a, V, ldv, m, C, ldc, max_blocks, s);
    if (a.w <= 4) return launch_vty_m<4>(a, V, ldv, m, C, ldc, max_blocks, s);
    return launch_vty_m<8>(a, V, ldv, m, C, ldc, max_blocks, s);
}

}  // namespace sp
