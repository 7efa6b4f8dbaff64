// SpMMV kernel variants with float64 values and float64 vectors (float64 accumulation),
// padded block widths 1, 2, 4.
#include "spmv_launch.cuh"

namespace sp {
SP_INSTANTIATE_WIDTH(double, double, 1)
SP_INSTANTIATE_WIDTH(double, double, 2)
SP_INSTANTIATE_WIDTH(double, double, 4)
}  // namespace sp
