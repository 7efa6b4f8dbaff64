// SpMMV variants with float32 values (float32 accumulation; float64 or float32 vectors).
#include "spmv_launch.cuh"

namespace sp {
template int launch_spmv_typed<float, double>(const SpmvArgs &, bool, int, cudaStream_t);
template int launch_spmv_typed<float, float>(const SpmvArgs &, bool, int, cudaStream_t);
}  // namespace sp
