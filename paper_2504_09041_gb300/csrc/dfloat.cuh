// dfloat.cuh -- double-float ("double-word") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers, so it carries a 48-bit significand
// (unit roundoff about 2^-48, against 2^-53 for FP64).  GB300 issues FP32 operations at 64 times
// its FP64 rate, so an FP64-accurate vector-Jacobian product written in this type runs several
// times faster than the same product in FP64.
//
// The operations are the double-word algorithms analysed by Joldes, Muller and Popescu ("Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic", ACM TOMS 44(2),
// 2017), built on Knuth's TwoSum and the FMA form of the exact product, with the final
// renormalization (Dekker's Fast2Sum) left out:
//   add:  TwoSum of the leading parts, the low parts added to its error term (8 flops).  The
//         pair (s, e + x.lo + y.lo) is the "sloppy" double-word sum before its renormalization:
//         the same value, with the same error, a few u^2 (u = 2^-24) of |x| + |y|;
//   mul:  the leading product with its exact error plus the three cross terms (5 flops).  The
//         lo * lo term is kept because an unnormalized input's low part need not be below
//         ulp(hi) / 2; the error is a few u^2 of |x| |y|;
//   div:  one FP32 quotient of the renormalized operands refined by one correction step.
// Pairs are therefore not normalized (|lo| may exceed ulp(hi) / 2 after a sum that cancels); no
// operation here needs them to be, and the value hi + lo is what every bound above refers to.
// Every FP32 step uses the _rn intrinsics so the compiler cannot contract or reorder the error
// terms.  Range: FP32's (values above 2^-100 in magnitude keep the full 48 bits).
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct __align__(8) dfloat {
    float hi, lo;

    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dfloat(float x) : hi(x), lo(0.0f) {}
    __host__ __device__ constexpr dfloat(int x) : hi((float)x), lo((float)((double)x - (double)(float)x)) {}
    // nearest double-float of an FP64 value (exact for FP64 values with at most 48 significant bits)
    __host__ __device__ constexpr dfloat(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth's TwoSum, 6 flops).
__device__ __forceinline__ dfloat df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfloat(s, e);
}

// s + e = a + b exactly when the exponent of a is at least that of b (Dekker's Fast2Sum).
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// The same value with hi the FP32 number nearest to it (TwoSum of the two parts).
__device__ __forceinline__ dfloat df_normalize(dfloat x) { return df_two_sum(x.hi, x.lo); }

// The sum of two unevaluated pairs (hi, lo), not renormalized.
__device__ __forceinline__ dfloat df_sum_pairs(float xh, float xl, float yh, float yl)
{
    const dfloat s = df_two_sum(xh, yh);
    return dfloat(s.hi, __fadd_rn(s.lo, __fadd_rn(xl, yl)));
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) { return df_sum_pairs(x.hi, x.lo, y.hi, y.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }

// A product: p the FP32 product of the leading parts and e its exact error plus the cross terms.
// It is already a (not renormalized) double-float; the type only records where it came from.
struct dfprod {
    float p, e;
    __device__ __forceinline__ operator dfloat() const { return dfloat(p, e); }
};

__device__ __forceinline__ dfprod operator*(dfloat x, dfloat y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);       // exact error of the leading product
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    e = __fmaf_rn(x.lo, y.lo, e);
    return dfprod{p, e};
}

__device__ __forceinline__ dfprod operator-(dfprod x) { return dfprod{-x.p, -x.e}; }

__device__ __forceinline__ dfloat operator+(dfprod x, dfloat y) { return df_sum_pairs(x.p, x.e, y.hi, y.lo); }
__device__ __forceinline__ dfloat operator+(dfloat x, dfprod y) { return df_sum_pairs(x.hi, x.lo, y.p, y.e); }
__device__ __forceinline__ dfloat operator+(dfprod x, dfprod y) { return df_sum_pairs(x.p, x.e, y.p, y.e); }
__device__ __forceinline__ dfloat operator-(dfprod x, dfloat y) { return df_sum_pairs(x.p, x.e, -y.hi, -y.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfprod y) { return df_sum_pairs(x.hi, x.lo, -y.p, -y.e); }
__device__ __forceinline__ dfloat operator-(dfprod x, dfprod y) { return df_sum_pairs(x.p, x.e, -y.p, -y.e); }
__device__ __forceinline__ dfprod operator*(dfprod x, dfloat y) { return dfloat(x) * y; }
__device__ __forceinline__ dfprod operator*(dfloat x, dfprod y) { return x * dfloat(y); }
__device__ __forceinline__ dfprod operator*(dfprod x, dfprod y) { return dfloat(x) * dfloat(y); }

// Double-float times an FP32 number (3 flops).
__device__ __forceinline__ dfloat df_mul_f(dfloat x, float y)
{
    const float p = __fmul_rn(x.hi, y);
    const float e = __fmaf_rn(x.lo, y, __fmaf_rn(x.hi, y, -p));
    return dfloat(p, e);
}

__device__ __forceinline__ dfloat operator/(dfloat x, dfloat y)
{
    x = df_normalize(x);
    y = df_normalize(y);
    const float q = __fdiv_rn(x.hi, y.hi);
    const dfloat r = x - df_mul_f(y, q);       // remainder, small: one correction term
    return df_fast_two_sum(q, __fdiv_rn(__fadd_rn(r.hi, r.lo), y.hi));
}

__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }
__device__ __forceinline__ dfloat& operator-=(dfloat& x, dfloat y) { return x = x - y; }
__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfprod y) { return x = x + y; }
__device__ __forceinline__ dfloat& operator-=(dfloat& x, dfprod y) { return x = x - y; }
__device__ __forceinline__ dfloat& operator*=(dfloat& x, dfloat y) { return x = x * y; }

}  // namespace lbm
