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
// tolerance is 1e-12).  Elements whose exponent lies outside [-40, 40]
// (including 0 handled exactly, and Inf/NaN) are not split: those terms go to
// an ordinary float64 accumulator, so every input is handled.
#pragma once

#include <stdint.h>

namespace sp {

constexpr int kFFMinExp = -40;  // unbiased exponent range allowed for a split
constexpr int kFFMaxExp = 40;  // products stay below 2^82, row sums below 2^113

// Split a double; returns false when d is out of range (then hi = lo = 0).
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
    const unsigned long long mant = b & 0x000fffffffffffffull;
    hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(mant >> 29));
    // low 29 bits times 2^(e - 52): an exact power-of-two scale (e - 52 >= -92)
    const float l = __uint2float_rn((unsigned)(mant & 0x1fffffffull)) * __uint_as_float((unsigned)(e - 52 + 127) << 23);
    lo = sign ? -l : l;
    return true;
}

struct FFAcc {
    float hi, lo;
    double nat;  // terms whose x could not be split
};

__device__ __forceinline__ void ff_zero(FFAcc &a) {
    a.hi = 0.0f;
    a.lo = 0.0f;
    a.nat = 0.0;
}

// s += (ah + al) x for a split matrix value (always in range: a matrix with
// any value out of range is not given a split and runs the float64 kernel)
__device__ __forceinline__ void ff_madd(FFAcc &s, float ah, float al, double x) {
    float xh, xl;
    if (ff_split(x, xh, xl)) {
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
    } else {
        s.nat = __fma_rn((double)ah + (double)al, x, s.nat);
    }
}

__device__ __forceinline__ double ff_value(const FFAcc &s) { return ((double)s.hi + (double)s.lo) + s.nat; }

// Combine two partial float-float sums (threads-per-row reduction): a += b.
__device__ __forceinline__ void ff_add(FFAcc &a, float bh, float bl, double bn) {
    const float t = __fadd_rn(a.hi, bh);
    const float bv = __fsub_rn(t, a.hi);
    const float av = __fsub_rn(t, bv);
    float err = __fadd_rn(__fsub_rn(a.hi, av), __fsub_rn(bh, bv));
    err = __fadd_rn(err, __fadd_rn(a.lo, bl));
    a.hi = __fadd_rn(t, err);
    a.lo = __fsub_rn(err, __fsub_rn(a.hi, t));
    a.nat = a.nat + bn;
}

}  // namespace sp
