// Double-float arithmetic on the FP32 pipe.
//
// A dfloat is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  Sums and products are built from error-free
// transformations: Knuth's TwoSum (s + e == a + b exactly), Dekker's
// Fast2Sum (the same when |a| >= |b|) and the product error fma(a, b, -a*b);
// the add and multiply below are the "sloppy" double-word algorithms of
// Dekker (1971) and Hida, Li & Bailey (2001).  The conserving precision of the
// same-level pass runs in this arithmetic: GB300 issues FP32 operations at 64
// times its FP64 rate, so a dozen FP32 operations per double-float operation
// still beat one FP64 operation several times over.
#pragma once

#include <cuda_runtime.h>

namespace fmm {

struct dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dfloat(float h) : hi(h), lo(0.f) {}
    __host__ __device__ constexpr dfloat(int i) : hi(float(i)), lo(0.f) {}
    // round-to-nearest split of a double: hi + lo carries 48 of its 53 bits
    __host__ __device__ explicit dfloat(double v) : hi(float(v)), lo(float(v - double(float(v)))) {}
    __host__ __device__ double to_double() const { return double(hi) + double(lo); }
};

// s = fl(a + b), e = a + b - s exactly (any magnitudes)
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// the same when |a| >= |b| (or a == 0)
__device__ __forceinline__ dfloat df_fast(float a, float b)
{
    const float s = a + b;
    return dfloat(s, b - (s - a));
}

// exact product of two floats
__device__ __forceinline__ dfloat df_two_prod(float a, float b)
{
    const float p = a * b;
    return dfloat(p, fmaf(a, b, -p));
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b)
{
    float s, e;
    df_two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    return df_fast(s, e);
}

__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast(p, e);
}

// by a float (small integer constants, exact powers of two, ...)
__device__ __forceinline__ dfloat operator*(float a, dfloat b)
{
    const float p = a * b.hi;
    float e = fmaf(a, b.hi, -p);
    e = fmaf(a, b.lo, e);
    return df_fast(p, e);
}
__device__ __forceinline__ dfloat operator*(dfloat a, float b) { return b * a; }

// a / b: one float quotient, the exact remainder a - q b in double-float,
// and a second quotient of the remainder (long division, Hida-Li-Bailey)
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b)
{
    const float q1 = a.hi / b.hi;
    const dfloat r = a - q1 * b;
    const float q2 = r.hi / b.hi;
    return df_fast(q1, q2);
}

// a * b + c in one pass: the product's error terms join the sum's low part
// before a single renormalisation (one Fast2Sum fewer than a product then a
// sum)
__device__ __forceinline__ dfloat fmadd(dfloat a, dfloat b, dfloat c)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float s, t;
    df_two_sum(p, c.hi, s, t);
    t += e + c.lo;
    return df_fast(s, t);
}

// The same without the closing Fast2Sum: the low part may grow past half an
// ulp of the high part.  Chains of these (a running sum, a dot product) stay
// exact to the double-float level as long as the low part stays small next
// to the high part; renorm() restores the canonical form, and the kernels
// call it at the end of every chain and every 16 stencil entries.
__device__ __forceinline__ dfloat fmadd_u(dfloat a, dfloat b, dfloat c)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float s, t;
    df_two_sum(p, c.hi, s, t);
    return dfloat(s, t + (e + c.lo));
}
__device__ __forceinline__ dfloat add_u(dfloat a, dfloat b)
{
    float s, e;
    df_two_sum(a.hi, b.hi, s, e);
    return dfloat(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ dfloat renorm(dfloat a) { return df_fast(a.hi, a.lo); }

__device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat &operator-=(dfloat &a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat &operator*=(dfloat &a, dfloat b) { return a = a * b; }

// 1/sqrt(v): the float estimate y refined by one Newton step for
// f(y) = 1/y^2 - v, y' = y + y (1 - v y^2) / 2; the residual 1 - v y^2 is
// formed in double-float (y^2 exactly), which doubles the estimate's bits
__device__ __forceinline__ dfloat df_rsqrt(dfloat v)
{
    const float y = rsqrtf(v.hi);
    const dfloat t = v * df_two_prod(y, y);
    const dfloat res = dfloat(1.f) - t;
    const float c = 0.5f * y * (res.hi + res.lo);
    return df_fast(y, c);
}

}  // namespace fmm
