// SpMMV kernel variants with float32 values and float32 vectors (float32 accumulation),
// padded block widths 1, 2, 4.
#include "spmv_launch.cuh"

namespace sp {
SP_INSTANTIATE_WIDTH(float, float, 1)
SP_INSTANTIATE_WIDTH(float, float, 2)
SP_INSTANTIATE_WIDTH(float, float, 4)
}  // namespace sp
