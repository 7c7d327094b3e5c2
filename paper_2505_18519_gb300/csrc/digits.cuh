// Error-free splitting of double-float values into 8-bit integer digits, for
// matrix products on the tensor cores as sums of exact FP16 digit products
// (Ozaki, Ogita, Oishi and Rump, error-free transformation of a matrix product
// into sums of products of low-precision matrices, Numer. Algorithms 59, 2012).
//
// A value scaled so that its row's largest entry lies in [128, 256) is
//     y = d_0 + d_1 2^-8 + d_2 2^-16 + d_3 2^-24 + d_4 2^-32 + r,   |r| <= 2^-33,
// |d_0| <= 256, |d_j| <= 129 (j >= 1): integers, so exact in FP16.  A product of
// two such operands over K <= 128 terms accumulates each digit order q = i + j in
// one FP32 accumulator whose partial sums stay integers below 2^24, so the tensor
// cores add them exactly; the epilogue weighs the accumulators by 2^-8q.
#pragma once
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "df.cuh"

namespace afq {

constexpr int DG_DIG = 5;   // digits per value

// 2^e as a float, for |e| <= 126.
__device__ __forceinline__ float dg_p2f(int e) {
    e = max(-126, min(126, e));
    return __int_as_float((e + 127) << 23);
}

// Exponent e with m 2^e in [128, 256) (0 for m = 0 or not finite).
__device__ __forceinline__ int dg_exp(float m) {
    if (!(m > 0.f) || !isfinite(m)) return 0;
    return max(-100, min(100, 7 - ilogbf(m)));
}

// Byte offset of element (row r, K index k < 64) in a K-major 128-byte swizzled
// region (rows of 128 bytes, groups of 8 rows 1024 bytes apart).
__device__ __forceinline__ uint32_t dg_swz(int r, int k) {
    return (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u + (uint32_t)((((k >> 3) ^ (r & 7)) << 4) | ((k & 7) << 1));
}

// The five digits of y = yh + yl (|y| < 257, scaled), as FP16 bit patterns.
// Every subtraction below is exact; the one rounded addition (b) errs by
// less than 2^-41.
__device__ __forceinline__ void dg_digits(float yh, float yl, uint16_t (&d)[DG_DIG]) {
    const float d0 = rintf(yh);
    float a = yh - d0;                                    // |a| <= 1/2
    const float d1 = rintf(a * 0x1p8f);
    a -= d1 * 0x1p-8f;                                    // |a| <= 2^-9
    const float d2 = rintf((a + yl) * 0x1p16f);
    a -= d2 * 0x1p-16f;
    const dfl r = df_two_sum(a, yl);                      // |r| <= about 2^-17
    const float d3 = rintf(r.hi * 0x1p24f);
    const float b = (r.hi - d3 * 0x1p-24f) + r.lo;
    const float d4 = rintf(b * 0x1p32f);
    d[0] = __half_as_ushort(__float2half_rn(d0));
    d[1] = __half_as_ushort(__float2half_rn(d1));
    d[2] = __half_as_ushort(__float2half_rn(d2));
    d[3] = __half_as_ushort(__float2half_rn(d3));
    d[4] = __half_as_ushort(__float2half_rn(d4));
}

// Eight FP16 bit patterns as one 16-byte unit.
__device__ __forceinline__ uint4 dg_pack8(const uint16_t (&h)[8]) {
    uint4 v;
    v.x = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
    v.y = (uint32_t)h[2] | ((uint32_t)h[3] << 16);
    v.z = (uint32_t)h[4] | ((uint32_t)h[5] << 16);
    v.w = (uint32_t)h[6] | ((uint32_t)h[7] << 16);
    return v;
}

// sum_q A_q 2^-8q of six exact integer accumulators, as a double-float value.
__device__ __forceinline__ dfl dg_combine6(float a0, float a1, float a2, float a3, float a4, float a5) {
    const float t1 = a1 * 0x1p-8f, t2 = a2 * 0x1p-16f;
    const float t3 = fmaf(a5, 0x1p-40f, fmaf(a4, 0x1p-32f, a3 * 0x1p-24f));
    const dfl x = df_two_sum(t2, t3);
    dfl y = df_two_sum(t1, x.hi);
    y.lo += x.lo;
    dfl z = df_two_sum(a0, y.hi);
    z.lo += y.lo;
    return df_quick(z.hi, z.lo);
}

// The same for five accumulators (orders 0 .. 4).
__device__ __forceinline__ dfl dg_combine5(float a0, float a1, float a2, float a3, float a4) {
    return dg_combine6(a0, a1, a2, a3, a4, 0.f);
}

}  // namespace afq
