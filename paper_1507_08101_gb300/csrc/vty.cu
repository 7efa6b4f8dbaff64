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
// These are the main product kernel's variants with MV > 0 (the same work
// split, row loops and epilogue as sp_spmv): each lane keeps the m x CPL
// products V[i, a] y[i, k0 + c] of its rows in registers, and the kernel ends
// with a reduction in a fixed order (reduce_vty), so C does not depend on
// timing.
#include "spmv_launch.cuh"

namespace sp {

template <int WP, bool LS, int MV>
static int launch_vty_variant(const SpmvArgs &a, int max_blocks, cudaStream_t s) {
    return launch_spmv_variant<double, double, WP, true, 0, false, LS, 2, MV>(a, max_blocks, s);
}

template <int WP, bool LS>
static int launch_vty_m(const SpmvArgs &a, int max_blocks, cudaStream_t s) {
    if (a.vty_m <= 1) return launch_vty_variant<WP, LS, 1>(a, max_blocks, s);
    if (a.vty_m <= 2) return launch_vty_variant<WP, LS, 2>(a, max_blocks, s);
    if (a.vty_m <= 4) return launch_vty_variant<WP, LS, 4>(a, max_blocks, s);
    return launch_vty_variant<WP, LS, 8>(a, max_blocks, s);
}

// The lockstep rule of sp_spmv's float64 kernels: always for block vectors,
// for single vectors when the row lengths inside 32-slot blocks spread widely
// (the chain adds float64 work per row, so the lower threshold applies then).
int launch_spmv_vty(const SpmvArgs &a, int max_blocks, cudaStream_t s) {
    if (a.w <= 1) {
        const double thr = (a.flags & SP_SPMV_CHAIN_AXPBY) ? SP_LS_SPREAD_DOTS : SP_LS_SPREAD;
        const bool ls = SP_LOCKSTEP == 2 || (SP_LOCKSTEP == 1 && a.wbounds_src && a.wbounds_src->lane_spread > thr);
        return ls ? launch_vty_m<1, true>(a, max_blocks, s) : launch_vty_m<1, false>(a, max_blocks, s);
    }
    if (a.w <= 2) return launch_vty_m<2, SP_LOCKSTEP != 0>(a, max_blocks, s);
    if (a.w <= 4) return launch_vty_m<4, SP_LOCKSTEP != 0>(a, max_blocks, s);
    return launch_vty_m<8, SP_LOCKSTEP != 0>(a, max_blocks, s);
}

}  // namespace sp
