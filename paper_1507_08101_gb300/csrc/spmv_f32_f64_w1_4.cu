// SpMMV kernel variants with float32 values and float64 vectors (float32 accumulation),
// padded block widths 1, 2, 4.
#include "spmv_launch.cuh"

namespace sp {
SP_INSTANTIATE_WIDTH(float, double, 1)
SP_INSTANTIATE_WIDTH(float, double, 2)
SP_INSTANTIATE_WIDTH(float, double, 4)
}  // namespace sp
