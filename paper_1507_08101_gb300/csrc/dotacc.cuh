// Accumulators of dot products over the products a*b of a vector precision.
//
// float64: plain fused multiply-adds.  float32: the exact product of two
// floats (TwoProd: p = fl(a b), e = fma(a, b, -p)) added into a float-float
// sum hi + lo with Knuth's TwoSum and Dekker's Fast2Sum, so a float32 kernel
// spends no float64 instruction per element (GB300 issues only about two
// float64 fused multiply-adds per SM per cycle).  The relative error per step
// is about 2^-47, far below what float32 vectors carry.  Every operation is
// rounded on its own; the error terms depend on it.
#pragma once

namespace sp {

// Plain accumulation in the vector precision (the float32 inner CG, whose
// iterates need far less than float64 accuracy in their inner products; the
// sums across lanes and units are still added in float64).
template <class XT>
struct DotAccPlain {
    XT v = XT(0);
    __device__ __forceinline__ void add(XT a, XT b) { v = fma(a, b, v); }
    __device__ __forceinline__ double value() const { return (double)v; }
};

template <class XT>
struct DotAcc;

template <>
struct DotAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double a, double b) { v = __fma_rn(a, b, v); }
    __device__ __forceinline__ double value() const { return v; }
};

template <>
struct DotAcc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        const float t = __fadd_rn(hi, p);
        const float bv = __fsub_rn(t, hi);
        const float av = __fsub_rn(t, bv);
        float err = __fadd_rn(__fsub_rn(hi, av), __fsub_rn(p, bv));
        err = __fadd_rn(err, __fadd_rn(lo, e));
        hi = __fadd_rn(t, err);
        lo = __fsub_rn(err, __fsub_rn(hi, t));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace sp
