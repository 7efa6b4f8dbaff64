// SpMMV kernel variants with float32 values and float32 vectors (float32 accumulation),
// padded block widths 8, 16, 32.
#include "spmv_launch.cuh"

namespace sp {
SP_INSTANTIATE_WIDTH(float, float, 8)
SP_INSTANTIATE_WIDTH(float, float, 16)
SP_INSTANTIATE_WIDTH(float, float, 32)
}  // namespace sp
