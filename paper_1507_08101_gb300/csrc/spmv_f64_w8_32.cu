// SpMMV kernel variants with float64 values and float64 vectors (float64 accumulation),
// padded block widths 8, 16, 32.
#include "spmv_launch.cuh"

namespace sp {
SP_INSTANTIATE_WIDTH(double, double, 8)
SP_INSTANTIATE_WIDTH(double, double, 16)
SP_INSTANTIATE_WIDTH(double, double, 32)
}  // namespace sp
