// Double-float arithmetic: a real number carried as the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi) / 2, about 46 significand bits
// computed on the FP32 pipes.  Used for the FP64-class operator applications
// of mixed-precision residual replacement, where this GPU's FP32 rate is ~58x
// its FP64 rate.
//
// Building blocks (error-free transformations, exact in round-to-nearest):
//   TwoSum   s + e = a + b exactly, no condition on |a|, |b|
//            (Knuth, The Art of Computer Programming vol. 2, Sec. 4.2.2);
//   Fast2Sum s + e = a + b exactly when |a| >= |b| (Dekker 1971);
//   TwoProd  p + e = a * b exactly, e from one fused multiply-add.
// Every float operation goes through a _rn intrinsic so the compiler can
// neither contract a product into a later add nor reorder the sums.
#pragma once

#include <cuda_runtime.h>

struct dd {
    float hi, lo;
    dd() = default;
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    // round a double to the nearest double-float
    __device__ explicit dd(double x) {
        hi = __double2float_rn(x);
        lo = __double2float_rn(x - (double)hi);
    }
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dd dd_fast2sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return dd(s, e);
}

__device__ __forceinline__ dd dd_2sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dd(s, e);
}

// a + b: exact sum of the high parts, low parts added to its error term, one
// renormalisation (relative error a few 2^-47 of |a| + |b|).
__device__ __forceinline__ dd operator+(dd a, dd b) {
    const dd s = dd_2sum(a.hi, b.hi);
    return dd_fast2sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }

// a * b: TwoProd of the high parts plus the two cross terms (the lo * lo
// term is below the format's resolution).
__device__ __forceinline__ dd operator*(dd a, dd b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dd_fast2sum(p, e);
}

// a * b + c with one renormalisation: TwoProd of the high parts, TwoSum of
// that product with c.hi, every lower-order term gathered into one float.
__device__ __forceinline__ dd fma(dd a, dd b, dd c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    const dd s = dd_2sum(p, c.hi);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    e = __fadd_rn(e, __fadd_rn(s.lo, c.lo));
    return dd_fast2sum(s.hi, e);
}
