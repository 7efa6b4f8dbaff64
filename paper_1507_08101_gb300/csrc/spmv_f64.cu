// SpMMV variants with float64 values (float64 vectors, float64 accumulation).
#include "spmv_launch.cuh"

namespace sp {
template int launch_spmv_typed<double, double>(const SpmvArgs &, bool, int, cudaStream_t);
}  // namespace sp
