// dfloat.cuh -- double-float ("double-word") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, so it
// carries a 48-bit significand (unit roundoff about 2^-48, against 2^-53 for FP64).  GB300 issues
// FP32 operations at 64 times its FP64 rate, so an FP64-accurate vector-Jacobian product written
// in this type runs several times faster than the same product in FP64.
//
// The operations follow the double-word algorithms analysed by Joldes, Muller and Popescu
// ("Tight and rigorous error bounds for basic building blocks of double-word arithmetic",
// ACM TOMS 44(2), 2017), built on Knuth's TwoSum, Dekker's Fast2Sum and the FMA form of the
// exact product:
//   add:  the "sloppy" double-word sum (11 flops); its error is a few u^2 (u = 2^-24) of
//         |x| + |y|, like the rounding of an FP64 sum of the same terms, but not relative to a
//         sum that cancels;
//   mul:  the FMA product with the lo*lo term dropped (7 flops with its renormalization, which a
//         following sum absorbs), relative error below 5 u^2;
//   div:  one FP32 quotient refined by one correction step (relative error below 10 u^2).
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

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y)
{
    const dfloat s = df_two_sum(x.hi, y.hi);
    const float w = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return df_fast_two_sum(s.hi, w);
}

__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }

// A product before its renormalization: p + e with p the FP32 product of the leading parts and e
// its exact error plus the cross terms (|e| <= 2^-22 |p|).  Sums consume it directly, which saves
// the Fast2Sum of a product that is then added (a*b + c in 15 flops instead of 18); anything else
// converts it to a double-float.
struct dfprod {
    float p, e;
    __device__ __forceinline__ operator dfloat() const { return df_fast_two_sum(p, e); }
};

__device__ __forceinline__ dfprod operator*(dfloat x, dfloat y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);       // exact error of the leading product
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return dfprod{p, e};
}

__device__ __forceinline__ dfprod operator-(dfprod x) { return dfprod{-x.p, -x.e}; }

// The sloppy sum of two unevaluated pairs (hi, lo), normalized once.
__device__ __forceinline__ dfloat df_sum_pairs(float xh, float xl, float yh, float yl)
{
    const dfloat s = df_two_sum(xh, yh);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(xl, yl)));
}

__device__ __forceinline__ dfloat operator+(dfprod x, dfloat y) { return df_sum_pairs(x.p, x.e, y.hi, y.lo); }
__device__ __forceinline__ dfloat operator+(dfloat x, dfprod y) { return df_sum_pairs(x.hi, x.lo, y.p, y.e); }
__device__ __forceinline__ dfloat operator+(dfprod x, dfprod y) { return df_sum_pairs(x.p, x.e, y.p, y.e); }
__device__ __forceinline__ dfloat operator-(dfprod x, dfloat y) { return df_sum_pairs(x.p, x.e, -y.hi, -y.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfprod y) { return df_sum_pairs(x.hi, x.lo, -y.p, -y.e); }
__device__ __forceinline__ dfloat operator-(dfprod x, dfprod y) { return df_sum_pairs(x.p, x.e, -y.p, -y.e); }
__device__ __forceinline__ dfprod operator*(dfprod x, dfloat y) { return dfloat(x) * y; }
__device__ __forceinline__ dfprod operator*(dfloat x, dfprod y) { return x * dfloat(y); }
__device__ __forceinline__ dfprod operator*(dfprod x, dfprod y) { return dfloat(x) * dfloat(y); }

// Double-float times an FP32 number (6 flops).
__device__ __forceinline__ dfloat df_mul_f(dfloat x, float y)
{
    const float p = __fmul_rn(x.hi, y);
    const float e = __fmaf_rn(x.lo, y, __fmaf_rn(x.hi, y, -p));
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ dfloat operator/(dfloat x, dfloat y)
{
    const float q = __fdiv_rn(x.hi, y.hi);
    const dfloat r = x - df_mul_f(y, q);       // remainder, small: one correction term
    return df_fast_two_sum(q, __fdiv_rn(r.hi, y.hi));
}

__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }
__device__ __forceinline__ dfloat& operator-=(dfloat& x, dfloat y) { return x = x - y; }
__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfprod y) { return x = x + y; }
__device__ __forceinline__ dfloat& operator-=(dfloat& x, dfprod y) { return x = x - y; }
__device__ __forceinline__ dfloat& operator*=(dfloat& x, dfloat y) { return x = x * y; }

}  // namespace lbm
