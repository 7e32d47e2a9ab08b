// float <-> double conversions through the IEEE-754 bit fields, on the
// integer pipe.
//
// GB300 runs FP64 arithmetic, and the F2F conversions between float and
// double, on a unit with 1/64 of the FP32 rate; in the FP64-bound downward and
// force passes a conversion costs as much as a double-precision add.  These
// helpers move the conversions to integer instructions.  They handle zeros,
// normal numbers, infinities and NaNs; subnormal inputs flush to a signed zero
// (the passes never produce magnitudes below 1e-38 in float or 1e-308 in
// double).
#pragma once

#include <cuda_runtime.h>

#include "fmm_dfloat.cuh"

namespace fmm {

// exact: a normal float is a double with the same sign, the exponent
// re-biased from 127 to 1023 and the 23 mantissa bits on top of 52
__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned m = u & 0x7FFFFFu;
    const unsigned e64 = e == 0xFFu ? 0x7FFu : e + (1023u - 127u);
    const unsigned hi = e == 0 ? sign : sign | (e64 << 20) | (m >> 3);
    const unsigned lo = e == 0 ? 0u : m << 29;
    return __hiloint2double(int(hi), int(lo));
}

// exact sum of a (hi, lo) float pair in double: both converted exactly, one
// double add
__device__ __forceinline__ double pair_to_double(float hi, float lo)
{
    return f2d_bits(hi) + f2d_bits(lo);
}

// truncating (toward zero): the 23 leading mantissa bits of the double;
// magnitudes outside float's normal range flush to zero or saturate to
// infinity; NaN stays NaN
__device__ __forceinline__ float d2f_trunc(double d)
{
    const unsigned hi = unsigned(__double2hiint(d)), lo = unsigned(__double2loint(d));
    const unsigned sign = hi & 0x80000000u;
    const int e64 = int((hi >> 20) & 0x7FFu);
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const int e = e64 - (1023 - 127);
    unsigned u;
    if (e64 == 0x7FF)
        u = sign | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u);
    else if (e <= 0)
        u = sign;
    else if (e >= 0xFF)
        u = sign | 0x7F800000u;
    else
        u = sign | (unsigned(e) << 23) | m;
    return __uint_as_float(u);
}

// rounded to nearest (ties to even): the 23 leading mantissa bits plus one
// when the 29 dropped bits exceed half an ulp (or equal it and the kept bits
// are odd); a carry out of the mantissa lands in the exponent, which is
// exactly the rounded value, and overflows to infinity
__device__ __forceinline__ float d2f_rn(double d)
{
    const unsigned hi = unsigned(__double2hiint(d)), lo = unsigned(__double2loint(d));
    const unsigned sign = hi & 0x80000000u;
    const int e64 = int((hi >> 20) & 0x7FFu);
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;
    const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    const int e = e64 - (1023 - 127);
    unsigned u;
    if (e64 == 0x7FF)
        u = sign | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u);
    else if (e <= 0)
        u = sign;
    else if (e >= 0xFF)
        u = sign | 0x7F800000u;
    else
        u = sign | ((unsigned(e) << 23) + m + up);
    return __uint_as_float(u);
}

// double -> double-float: the rounded float and the rounded remainder (one
// double subtraction, exact; the two conversions on the integer pipe)
__device__ __forceinline__ dfloat df_from_double(double v)
{
    const float hi = d2f_rn(v);
    return dfloat(hi, d2f_rn(v - f2d_bits(hi)));
}

// double-float -> double: both parts converted exactly, one double add
__device__ __forceinline__ double df_to_double(dfloat v) { return f2d_bits(v.hi) + f2d_bits(v.lo); }

}  // namespace fmm
