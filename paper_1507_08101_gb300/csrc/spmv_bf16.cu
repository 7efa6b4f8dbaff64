// SpMMV variants with bfloat16 values (float32 accumulation; float64 or float32 vectors).
#include "spmv_launch.cuh"

namespace sp {
template int launch_spmv_typed<__nv_bfloat16, double>(const SpmvArgs &, bool, int, cudaStream_t);
template int launch_spmv_typed<__nv_bfloat16, float>(const SpmvArgs &, bool, int, cudaStream_t);
}  // namespace sp
