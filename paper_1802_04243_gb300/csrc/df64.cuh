// df64.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo
// of two floats with |lo| <= ulp(hi)/2, about 48 significant bits, computed
// entirely on the FP32 pipe.
//
// GB300 issues FP64 at 1/64 of its FP32 rate, and the FP64 sweep is bound by
// that pipe.  The DF64 precision mode of the sweep runs the same kernel
// bodies on this type instead of double.
//
// The building blocks are the error-free transformations of floating-point
// addition and multiplication: TwoSum (Knuth, The Art of Computer
// Programming vol. 2, 4.2.2), FastTwoSum (Dekker, "A floating-point technique
// for extending the available precision", Numer. Math. 18, 1971) and the
// product error through a fused multiply-add.  Sum, product, reciprocal and
// square root follow the double-word algorithms of Dekker (1971) and of Hida,
// Li and Bailey ("Algorithms for quad-double precision floating point
// arithmetic", ARITH-15, 2001): a result's relative error is a small multiple
// of 2^-48 except for the sum of nearly opposite values, whose absolute error
// stays below about 2^-47 times the larger operand.
//
// Every float operation below uses the _rn intrinsics, which the compiler
// never contracts into fused multiply-adds: the transformations rely on each
// operation being rounded on its own.
//
// The type and its functions live in their own namespace and are found by
// argument-dependent lookup, so they never hide the double versions of fma or
// sqrt from code in other namespaces.
#pragma once

#include <cuda_runtime.h>

namespace dfl {

struct __align__(8) df64 {
    float hi, lo;

    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    // From a double known at compile time (the literals of the kernel
    // bodies); runtime doubles go through split_host / split_dev.
    __host__ __device__ constexpr df64(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ constexpr df64(int x) : df64((double)x) {}
};

// Split of a runtime double (host side: set-up of tables and coefficients).
__host__ inline df64 split_host(double x)
{
    const float h = (float)x;
    return df64(h, (float)(x - (double)h));
}

namespace dd {

// s + e = a + b exactly (Knuth's TwoSum, no condition on a and b).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker's FastTwoSum).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

}  // namespace dd

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    float s, e;
    dd::two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    float h, l;
    dd::fast_two_sum(s, e, h, l);
    return df64(h, l);
}

__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);                 // exact error of the leading product
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float h, l;
    dd::fast_two_sum(p, e, h, l);
    return df64(h, l);
}

__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }

__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }

// a * b for a float b.
__device__ __forceinline__ df64 mul_f(df64 a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    float h, l;
    dd::fast_two_sum(p, e, h, l);
    return df64(h, l);
}

// 1/a: the correctly rounded float reciprocal r of a.hi (relative error at
// most 2^-24) refined by one Newton-Raphson step r + r (1 - a r), with the
// residual 1 - a r formed in double-float; the step squares the error.
__device__ __forceinline__ df64 recip(df64 a)
{
    const float r = __frcp_rn(a.hi);
    const df64 e = df64(1.0f, 0.0f) - mul_f(a, r);
    float h, l;
    dd::fast_two_sum(r, __fmul_rn(e.hi, r), h, l);
    return df64(h, l);
}

__device__ __forceinline__ df64 operator/(df64 a, df64 b) { return a * recip(b); }

// sqrt(a), a >= 0: the float root s of a.hi refined by one Newton step
// s <- s + (a - s^2) / (2 s) in double-float (Dekker 1971).
__device__ __forceinline__ df64 sqrt(df64 a)
{
    if (a.hi <= 0.0f) return df64(0.0f, 0.0f);
    const float s = __fsqrt_rn(a.hi);
    const float p = __fmul_rn(s, s);
    const float pe = __fmaf_rn(s, s, -p);                // s^2 = p + pe exactly
    const df64 r = a - df64(p, pe);
    const float corr = __fdiv_rn(r.hi, __fmul_rn(2.0f, s));
    float h, l;
    dd::fast_two_sum(s, corr, h, l);
    return df64(h, l);
}

// Ordering of normalised values: the leading parts decide unless equal.
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(df64 a, df64 b) { return b > a; }

// Conversions of runtime values (FP64 pipe: set-up and export only).
__device__ __forceinline__ double join(df64 a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df64 split_dev(double x)
{
    const float h = __double2float_rn(x);
    return df64(h, __double2float_rn(x - (double)h));
}

}  // namespace dfl
