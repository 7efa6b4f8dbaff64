// Float-float ("double-float") arithmetic for the float64 row sums.
//
// GB300 issues about two float64 fused multiply-adds per SM per cycle, so a
// float64 SpMV with one multiply-add per 12 bytes of matrix stream is bound by
// the float64 pipe long before HBM.  The row sums are therefore carried as an
// unevaluated sum of two floats, s = s_hi + s_lo, on the FP32 pipes:
//
//  * a float64 value a is split into a_hi + a_lo: a_hi keeps the sign, the
//    exponent and the top 23 fraction bits (truncation, exact), a_lo the
//    remaining 29 bits rounded to a float -- integer instructions only, error
//    at most 2^-48 |a|;
//  * a_hi x_hi is formed exactly as p + e (e = fma(a_hi, x_hi, -p)), the cross
//    terms a_hi x_lo + a_lo x_hi are added into e, a_lo x_lo (2^-48) is dropped;
//  * (p, e) is added to (s_hi, s_lo) with Knuth's TwoSum and renormalised with
//    Fast2Sum (Dekker 1971; the "sloppy" double-float addition).
//
// Each step has a relative error of about 2^-47, so a row of n terms is within
// about n 2^-47 of the exact sum relative to sum |a_j x_j| (the float64 kernel
// tolerance is 1e-12).  Zero splits exactly; a matrix with a value whose
// exponent lies outside [-40, 40] gets no split (the float64 kernel runs); a
// row that meets such an x entry (or Inf/NaN) is recomputed in float64, so
// every input is handled.
#pragma once

#include <stdint.h>

namespace sp {

constexpr int kFFMinExp = -40;  // unbiased exponent range allowed for a split
constexpr int kFFMaxExp = 40;  // products stay below 2^82, row sums below 2^113

// Split a double; returns false when d is out of range (then hi = lo = 0).
// Integer and FP32 instructions only: the low 29 bits are turned into a float
// with the exact "magic number" conversion (an integer n < 2^23 or'ed into the
// fraction of 2^23, minus 2^23) in two pieces of 23 and 6 bits, so no
// conversion instruction is issued.
__device__ __forceinline__ bool ff_split(double d, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    if ((b & 0x7fffffffffffffffull) == 0) {
        hi = lo = 0.0f;
        return true;
    }
    if (e < kFFMinExp || e > kFFMaxExp) {
        hi = lo = 0.0f;
        return false;
    }
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const unsigned lowword = (unsigned)b;         // fraction bits 31..0
    const unsigned highword = (unsigned)(b >> 32);
    // top 23 fraction bits: 20 from the high word, 3 from the low word
    hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | ((highword & 0xfffffu) << 3) | (lowword >> 29));
    const unsigned low29 = lowword & 0x1fffffffu;
    const float magic = 8388608.0f;  // 2^23
    const float f23 = __fsub_rn(__uint_as_float(0x4B000000u | (low29 & 0x7fffffu)), magic);
    const float f6 = __fsub_rn(__uint_as_float(0x4B000000u | (low29 >> 23)), magic);
    // (f6 2^23 + f23) 2^(e - 52): one rounding to 24 bits, then an exact scale
    const float l = __fmul_rn(__fmaf_rn(f6, magic, f23), __uint_as_float((unsigned)(e - 52 + 127) << 23));
    lo = __uint_as_float(__float_as_uint(l) | sign);
    return true;
}

struct FFAcc {
    float hi, lo;
    bool bad;  // an x entry of this row could not be split: the row is redone in float64
};

__device__ __forceinline__ void ff_zero(FFAcc &a) {
    a.hi = 0.0f;
    a.lo = 0.0f;
    a.bad = false;
}

// s += (ah + al) x for a split matrix value (always in range: a matrix with
// any value out of range is not given a split and runs the float64 kernel).
// Only FP32 and integer instructions; an x out of range just marks the row.
__device__ __forceinline__ void ff_madd(FFAcc &s, float ah, float al, double x) {
    float xh, xl;
    const bool ok = ff_split(x, xh, xl);
    s.bad |= !ok;
    // every operation rounded on its own: the error terms rely on it
    const float p = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -p);
    e = __fmaf_rn(ah, xl, e);
    e = __fmaf_rn(al, xh, e);
    const float t = __fadd_rn(s.hi, p);  // TwoSum(s.hi, p)
    const float bv = __fsub_rn(t, s.hi);
    const float av = __fsub_rn(t, bv);
    float err = __fadd_rn(__fsub_rn(s.hi, av), __fsub_rn(p, bv));
    err = __fadd_rn(err, __fadd_rn(s.lo, e));
    s.hi = __fadd_rn(t, err);  // Fast2Sum
    s.lo = __fsub_rn(err, __fsub_rn(s.hi, t));
}

__device__ __forceinline__ double ff_value(const FFAcc &s) { return (double)s.hi + (double)s.lo; }

// Combine two partial float-float sums (threads-per-row reduction): a += b.
__device__ __forceinline__ void ff_add(FFAcc &a, float bh, float bl, bool bbad) {
    const float t = __fadd_rn(a.hi, bh);
    const float bv = __fsub_rn(t, a.hi);
    const float av = __fsub_rn(t, bv);
    float err = __fadd_rn(__fsub_rn(a.hi, av), __fsub_rn(bh, bv));
    err = __fadd_rn(err, __fadd_rn(a.lo, bl));
    a.hi = __fadd_rn(t, err);
    a.lo = __fsub_rn(err, __fsub_rn(a.hi, t));
    a.bad = a.bad || bbad;
}

// Accumulator of a dot product over products a*b of the vector precision.
// float64: plain fused multiply-adds.  float32: the exact product (TwoProd)
// added into a float-float sum, so no float64 instruction is spent per element.
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
