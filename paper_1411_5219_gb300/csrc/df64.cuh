// Double-float ("df64") arithmetic: a real number as the unevaluated sum
// hi + lo of two FP32 values, |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 executes FP32 at 58x its FP64 rate (measured: 73 vs 1.25 TFLOP/s),
// so FP64-accurate operators written in pairs of FP32 numbers run faster than
// native FP64 ones.  The building blocks are the error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a+b) and the exact error e,
//       a + b = s + e, in six additions;
//   FastTwoSum (Dekker 1971): the same in three additions when |a| >= |b|;
//   TwoProduct with FMA (e.g. Ogita, Rump and Oishi, SIAM J. Sci. Comput.
//       26 (2005)): p = fl(ab), e = fma(a, b, -p), ab = p + e exactly.
// Addition and multiplication below follow the classical double-length
// algorithms built from them (Dekker 1971).  All operations use the _rn
// intrinsics so the compiler cannot contract or reorder them.
#pragma once

#include <cuda_runtime.h>

namespace qcd {

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    // from double: hi = RN(d), lo = RN(d - hi); |d - (hi + lo)| <= 2^-48 |d|
    __host__ __device__ df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit df(float f) : hi(f), lo(0.0f) {}
    __host__ __device__ df(int i) : hi((float)i), lo(0.0f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi; }
};

__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df(s, e);
}

__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df operator+(df x, df y)
{
    const df s = two_sum(x.hi, y.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }

__device__ __forceinline__ df operator*(df x, df y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

// x*y + z with one rounding of the product error into the sum.
__device__ __forceinline__ df fma(df x, df y, df z)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    const df s = two_sum(p, z.hi);
    const float t = __fadd_rn(s.lo, __fadd_rn(e, z.lo));
    return fast_two_sum(s.hi, t);
}

// keep the float/double overloads visible next to the df one
using ::fma;

__device__ __forceinline__ df &operator+=(df &x, df y)
{
    x = x + y;
    return x;
}

}  // namespace qcd
