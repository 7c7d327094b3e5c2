// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers (about 44 significant bits).  Products use the exact FMA residual
// (TwoProduct), sums Knuth's TwoSum; dot products in the kernels follow the
// compensated Dot2 scheme of Ogita, Rump and Oishi (2005).  Used by the
// mixed-precision path for the work it keeps off the FP64 pipe (FP64 issues at
// about 1/64 of the FP32 rate on this part).
#pragma once
#include <cuda_runtime.h>

namespace afq {

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl df_quick(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    const dfl s = df_two_sum(a.hi, b.hi), t = df_two_sum(a.lo, b.lo);
    const dfl u = df_quick(s.hi, s.lo + t.hi);
    return df_quick(u.hi, u.lo + t.lo);
}
// a + b with one two-sum of the high parts and the low parts added in FP32 (the
// "sloppy" double-double addition of Hida, Li and Bailey's QD library): about 2^-44
// of max(|a|, |b|), half the operations of df_add.
__device__ __forceinline__ dfl df_add_fast(dfl a, dfl b) {
    const dfl s = df_two_sum(a.hi, b.hi);
    return df_quick(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_quick(p, e);
}
__device__ __forceinline__ dfl df_from(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }

// acc += a * b in Dot2 form: acc_hi carries the sum, acc_lo the accumulated errors.
__device__ __forceinline__ void dot2_fma(float& acc_hi, float& acc_lo, dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float q = fmaf(a.hi, b.hi, -p);
    q = fmaf(a.hi, b.lo, q);
    q = fmaf(a.lo, b.hi, q);
    const float t = acc_hi + p, z = t - acc_hi;
    acc_lo += q + ((acc_hi - (t - z)) + (p - z));
    acc_hi = t;
}

}  // namespace afq
