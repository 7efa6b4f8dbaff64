// SpMMV variants with float64 values and vectors whose row sums run in
// float-float arithmetic on the FP32 pipes (values pre-split into float pairs).
#include "spmv_launch.cuh"

namespace sp {
int launch_spmv_ff(const SpmvArgs &a, bool vec, int max_blocks, cudaStream_t s) {
    return launch_spmv_width<double, double, true>(a, vec, max_blocks, s);
}
}  // namespace sp
