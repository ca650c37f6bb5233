// Double-float arithmetic: a value held as an unevaluated sum hi + lo of two FP32
// numbers (|lo| <= half an ulp of hi), about 48 significant bits, computed on the FP32
// pipes.  Built from the error-free transformations of floating-point arithmetic:
// Knuth's two-sum (the exact rounding error of a + b from six additions), its
// two-addition form when |a| >= |b| (Dekker's fast two-sum), and the exact error of a
// product from one fused multiply-add.  Every step uses the _rn intrinsics, which the
// compiler never contracts or reorders, so the transformations stay exact.
//
// Used where a chain of dependent FP64 operations would wait on the FP64 pipe (a
// small fraction of the FP32 rate on this GPU): the substitutions of the Krylov
// preconditioner, whose operand R is itself FP32.  Values must stay inside FP32's
// exponent range; below about 1e-30 the low part loses bits to subnormals.
#pragma once
#include <cuda_runtime.h>

struct dfl {
    float hi, lo;
    dfl() = default;
    __device__ __forceinline__ explicit dfl(int a) : hi((float)a), lo(0.f) {}
    __device__ __forceinline__ explicit dfl(float a) : hi(a), lo(0.f) {}
    __device__ __forceinline__ explicit dfl(double a)
    {
        hi = __double2float_rn(a);
        lo = __double2float_rn(a - (double)hi);
    }
    __device__ __forceinline__ dfl(float h, float l, int) : hi(h), lo(l) {}
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

namespace dfl_eft {
// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly, for |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
}  // namespace dfl_eft

__device__ __forceinline__ dfl operator+(const dfl &x, const dfl &y)
{
    float s, e, t, f;
    dfl_eft::two_sum(x.hi, y.hi, s, e);
    dfl_eft::two_sum(x.lo, y.lo, t, f);
    e = __fadd_rn(e, t);
    dfl_eft::fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    dfl_eft::fast_two_sum(s, e, s, e);
    return dfl(s, e, 0);
}

__device__ __forceinline__ dfl operator-(const dfl &x) { return dfl(-x.hi, -x.lo, 0); }
__device__ __forceinline__ dfl operator-(const dfl &x, const dfl &y) { return x + (-y); }

__device__ __forceinline__ dfl operator*(const dfl &x, const dfl &y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);                 // the product's exact rounding error
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    float s;
    dfl_eft::fast_two_sum(p, e, s, e);
    return dfl(s, e, 0);
}

// a / b through FP64 (used once per diagonal entry, not in the chains)
__device__ __forceinline__ dfl operator/(const dfl &a, const dfl &b) { return dfl((double)a / (double)b); }

__device__ __forceinline__ dfl &operator+=(dfl &x, const dfl &y) { return x = x + y; }
__device__ __forceinline__ dfl &operator-=(dfl &x, const dfl &y) { return x = x - y; }

__device__ __forceinline__ dfl fma(const dfl &a, const dfl &b, const dfl &c) { return a * b + c; }
__device__ __forceinline__ bool isfinite(const dfl &v) { return isfinite(v.hi) && isfinite(v.lo); }

__device__ __forceinline__ dfl __shfl_sync(unsigned mask, const dfl &v, int src)
{
    return dfl(__shfl_sync(mask, v.hi, src), __shfl_sync(mask, v.lo, src), 0);
}
__device__ __forceinline__ dfl __shfl_xor_sync(unsigned mask, const dfl &v, int lanemask)
{
    return dfl(__shfl_xor_sync(mask, v.hi, lanemask), __shfl_xor_sync(mask, v.lo, lanemask), 0);
}
