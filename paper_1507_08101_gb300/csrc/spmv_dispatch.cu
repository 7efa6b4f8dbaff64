// Run-time choice of the SpMMV kernel's padded block width for each
// (value, vector) precision pair; the variants themselves are compiled in
// the spmv_<pair>_<widths>.cu units.
#include "spmv_kernel.cuh"

namespace sp {

template <class VT, class XT, int WP>
int launch_spmv_width(const SpmvArgs &a, bool vec, int max_blocks, cudaStream_t s);

template <class VT, class XT>
int launch_spmv_typed(const SpmvArgs &a, bool vec, int max_blocks, cudaStream_t s) {
    const int w = a.w;
    if (w <= 1) return launch_spmv_width<VT, XT, 1>(a, vec, max_blocks, s);
    if (w <= 2) return launch_spmv_width<VT, XT, 2>(a, vec, max_blocks, s);
    if (w <= 4) return launch_spmv_width<VT, XT, 4>(a, vec, max_blocks, s);
    if (w <= 8) return launch_spmv_width<VT, XT, 8>(a, vec, max_blocks, s);
    if (w <= 16) return launch_spmv_width<VT, XT, 16>(a, vec, max_blocks, s);
    if (w <= 32) return launch_spmv_width<VT, XT, 32>(a, vec, max_blocks, s);
    return SP_ERR_ARG;
}

template int launch_spmv_typed<double, double>(const SpmvArgs &, bool, int, cudaStream_t);
template int launch_spmv_typed<float, double>(const SpmvArgs &, bool, int, cudaStream_t);
template int launch_spmv_typed<float, float>(const SpmvArgs &, bool, int, cudaStream_t);
template int launch_spmv_typed<__nv_bfloat16, double>(const SpmvArgs &, bool, int, cudaStream_t);
template int launch_spmv_typed<__nv_bfloat16, float>(const SpmvArgs &, bool, int, cudaStream_t);

}  // namespace sp
