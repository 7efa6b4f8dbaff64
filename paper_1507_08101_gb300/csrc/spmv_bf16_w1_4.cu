// SpMMV kernel variants with bfloat16 values and float32 vectors (float32 accumulation),
// padded block widths 1, 2, 4.
#include "spmv_launch.cuh"

namespace sp {
SP_INSTANTIATE_WIDTH(__nv_bfloat16, float, 1)
SP_INSTANTIATE_WIDTH(__nv_bfloat16, float, 2)
SP_INSTANTIATE_WIDTH(__nv_bfloat16, float, 4)
}  // namespace sp
