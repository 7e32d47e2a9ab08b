// Device helpers: symmetric-tensor index maps and the derivative tensors of
// 1/|R| used by the same-level interactions (Sec. 4.3: Taylor coefficients of
// a cell's potential from the multipole moments of its partners).
//
// Symmetric components are stored once each:
//   rank 2 (6):  xx xy xz yy yz zz
//   rank 3 (10): xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
//   rank 4 (15): xxxx xxxy xxxz xxyy xxyz xxzz xyyy xyyz xyzz xzzz
//                yyyy yyyz yyzz yzzz zzzz
#pragma once

#include <cuda_runtime.h>

#include "fmm_dfloat.cuh"

namespace fmm {

// number of index orderings of each symmetric component
__host__ __device__ constexpr int mult2(int q) { return (q == 1 || q == 2 || q == 4) ? 2 : 1; }
__host__ __device__ constexpr int mult3(int q)
{
    return q == 0 || q == 6 || q == 9 ? 1 : (q == 4 ? 6 : 3);
}

// rank-3 component (i, q2) for i in 0..2 and q2 a rank-2 component
__host__ __device__ constexpr int r3_of(int i, int q)
{
    constexpr int t[3][6] = {{0, 1, 2, 3, 4, 5}, {1, 3, 4, 6, 7, 8}, {2, 4, 5, 7, 8, 9}};
    return t[i][q];
}
// rank-4 component (i, q3) for i in 0..2 and q3 a rank-3 component
__host__ __device__ constexpr int r4_of(int i, int q)
{
    constexpr int t[3][10] = {{0, 1, 2, 3, 4, 5, 6, 7, 8, 9},
                              {1, 3, 4, 6, 7, 8, 10, 11, 12, 13},
                              {2, 4, 5, 7, 8, 9, 11, 12, 13, 14}};
    return t[i][q];
}
// rank-2 component (i, j)
__host__ __device__ constexpr int r2_of(int i, int j)
{
    constexpr int t[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    return t[i][j];
}
// rank-3 component (i, j, k)
__host__ __device__ constexpr int r3_ijk(int i, int j, int k) { return r3_of(i, r2_of(j, k)); }
// the index pair / triple of a rank-2 / rank-3 component
__host__ __device__ constexpr int i2_at(int q, int which)
{
    constexpr int t[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    return t[q][which];
}
__host__ __device__ constexpr int i3_at(int q, int which)
{
    constexpr int t[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                              {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
    return t[q][which];
}

// a * b + c in the element type (fused in float and double; fmm_dfloat.cuh
// has the double-float one)
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
// chain forms (double-float skips the renormalisation until renorm())
__device__ __forceinline__ float fmadd_u(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmadd_u(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float add_u(float a, float b) { return a + b; }
__device__ __forceinline__ double add_u(double a, double b) { return a + b; }
__device__ __forceinline__ float renorm(float a) { return a; }
__device__ __forceinline__ double renorm(double a) { return a; }

template <typename T> __device__ __forceinline__ T rsqrt_t(T v);
// float: the hardware's approximate reciprocal square root with subnormal
// inputs flushed to zero (the PTX instruction itself), which spares the
// subnormal-input handling around it; the kernels give it squared
// distances of about a cell width or more, always normal numbers, for
// which flushing changes nothing
__device__ __forceinline__ float rsqrt_ftz(float v)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
template <> __device__ __forceinline__ float rsqrt_t<float>(float v) { return rsqrt_ftz(v); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double v) { return 1.0 / sqrt(v); }
template <> __device__ __forceinline__ dfloat rsqrt_t<dfloat>(dfloat v) { return df_rsqrt(v); }

// Derivative tensors of 1/|R| (Cartesian closed forms):
//   D1_i = d1 R_i,  D2_ij = d2 R_i R_j + d1 delta_ij,
//   D3_ijk = d3 R_i R_j R_k + d2 (R_i delta_jk + R_j delta_ik + R_k delta_ij),
//   D4_ijkl = d4 R_i R_j R_k R_l + d3 (sum of the six R R delta terms)
//             + d2 (delta_ij delta_kl + delta_ik delta_jl + delta_il delta_jk),
// with d0 = 1/r, d1 = -1/r^3, d2 = 3/r^5, d3 = -15/r^7, d4 = 105/r^9.
template <typename T, bool WITH_D4>
struct DTensors {
    T D0, D1[3], D2[6], D3[10], D4[15];

    __device__ __forceinline__ void eval(T x, T y, T z)
    {
        T r2 = x * x + y * y + z * z;
        T ri = rsqrt_t<T>(r2);
        T ri2 = ri * ri;
        T d0 = ri;
        T d1 = -d0 * ri2;
        T d2 = T(-3) * d1 * ri2;
        T d3 = T(-5) * d2 * ri2;
        D0 = d0;
        D1[0] = d1 * x; D1[1] = d1 * y; D1[2] = d1 * z;
        T xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
        D2[0] = d2 * xx + d1; D2[1] = d2 * xy; D2[2] = d2 * xz;
        D2[3] = d2 * yy + d1; D2[4] = d2 * yz; D2[5] = d2 * zz + d1;
        T d3x = d3 * x, d3y = d3 * y, d3z = d3 * z;
        D3[0] = d3x * xx + T(3) * d2 * x;
        D3[1] = d3x * xy + d2 * y;
        D3[2] = d3x * xz + d2 * z;
        D3[3] = d3x * yy + d2 * x;
        D3[4] = d3x * yz;
        D3[5] = d3x * zz + d2 * x;
        D3[6] = d3y * yy + T(3) * d2 * y;
        D3[7] = d3y * yz + d2 * z;
        D3[8] = d3y * zz + d2 * y;
        D3[9] = d3z * zz + T(3) * d2 * z;
        if (WITH_D4) {
            T d4 = T(-7) * d3 * ri2;
            T d4xx = d4 * xx, d4yy = d4 * yy, d4xy = d4 * xy, d4xz = d4 * xz, d4yz = d4 * yz;
            D4[0] = d4xx * xx + T(6) * d3 * xx + T(3) * d2;
            D4[1] = d4xx * xy + T(3) * d3 * xy;
            D4[2] = d4xx * xz + T(3) * d3 * xz;
            D4[3] = d4xx * yy + d3 * (xx + yy) + d2;
            D4[4] = d4xx * yz + d3 * yz;
            D4[5] = d4xx * zz + d3 * (xx + zz) + d2;
            D4[6] = d4xy * yy + T(3) * d3 * xy;
            D4[7] = d4xy * yz + d3 * xz;
            D4[8] = d4xy * zz + d3 * xy;
            D4[9] = d4xz * zz + T(3) * d3 * xz;
            D4[10] = d4yy * yy + T(6) * d3 * yy + T(3) * d2;
            D4[11] = d4yy * yz + T(3) * d3 * yz;
            D4[12] = d4yy * zz + d3 * (yy + zz) + d2;
            D4[13] = d4yz * zz + T(3) * d3 * yz;
            D4[14] = d4 * zz * zz + T(6) * d3 * zz + T(3) * d2;
        }
    }
};

// The same tensors in traceless bases.  Every D^(n), n >= 2, is traceless in
// each index pair, so only some components are independent:
//   rank 2 (5): xx yy xy xz yz                     (zz = -xx - yy)
//   rank 3 (7): xxx xxy xxz xyy xyz yyy yyz        (xzz = -xxx - xyy,
//                                                   yzz = -xxy - yyy,
//                                                   zzz = -xxz - yyz)
// and contracting a traceless tensor T with a symmetric moment only sees the
// moment's traceless part, which is stored in the matching basis:
//   B2 = [A2xx - A2zz, A2yy - A2zz, A2xy, A2xz, A2yz],
//   B3 = [A3xxx - A3xzz, A3xxy - A3yzz, A3xxz - A3zzz, A3xyy - A3xzz, A3xyz,
//         A3yyy - A3yzz, A3yyz - A3zzz],
// so that sum_q A2_q T_q = B2 . T(5) and sum_q A3_q T_q = B3 . T(7).
// D4 enters only through the slices U_i = D4[i, basis-7 triples]; the twelve
// components those need are the nine independent ones below plus
// xxzz = -xxxx - xxyy, xyzz = -xxxy - xyyy, yyzz = -xxyy - yyyy.
template <typename T>
struct DTraceless {
    T D0, D1[3];
    T D2[5];                 // xx yy xy xz yz
    T D3[9];                 // xxx xxy xxz xyy xyz yyy yyz | xzz yzz
    T U[3][7];               // D4 slices for the B3 basis

    template <bool WITH_D4>
    __device__ __forceinline__ void eval(T x, T y, T z)
    {
        const T r2 = fmadd(x, x, fmadd(y, y, z * z));
        const T ri = rsqrt_t<T>(r2);
        const T ri2 = ri * ri;
        const T d1 = -ri * ri2;
        const T d2 = d1 * (T(-3) * ri2);
        const T d3 = d2 * (T(-5) * ri2);
        D0 = ri;
        D1[0] = d1 * x; D1[1] = d1 * y; D1[2] = d1 * z;
        const T xx = x * x, yy = y * y, xy = x * y, xz = x * z, yz = y * z;
        D2[0] = fmadd(d2, xx, d1);
        D2[1] = fmadd(d2, yy, d1);
        D2[2] = d2 * xy;
        D2[3] = d2 * xz;
        D2[4] = d2 * yz;
        const T d3x = d3 * x, d3y = d3 * y;
        const T t2 = T(3) * d2;
        D3[0] = fmadd(d3x, xx, t2 * x);      // xxx
        D3[1] = fmadd(d3x, xy, d2 * y);      // xxy
        D3[2] = fmadd(d3x, xz, d2 * z);      // xxz
        D3[3] = fmadd(d3x, yy, d2 * x);      // xyy
        D3[4] = d3x * yz;                    // xyz
        D3[5] = fmadd(d3y, yy, t2 * y);      // yyy
        D3[6] = fmadd(d3y, yz, d2 * z);      // yyz
        D3[7] = -(D3[0] + D3[3]);            // xzz
        D3[8] = -(D3[1] + D3[5]);            // yzz
        if (WITH_D4) {
            const T d4 = d3 * (T(-7) * ri2);
            const T t3 = T(3) * d3, t6 = T(6) * d3;
            const T d4xx = d4 * xx, d4yy = d4 * yy, d4xy = d4 * xy;
            const T xxxx = fmadd(d4xx, xx, fmadd(t6, xx, t2));
            const T xxxy = fmadd(d4xx, xy, t3 * xy);
            const T xxxz = fmadd(d4xx, xz, t3 * xz);
            const T xxyy = fmadd(d4xx, yy, fmadd(d3, xx + yy, d2));
            const T xxyz = fmadd(d4xx, yz, d3 * yz);
            const T xyyy = fmadd(d4xy, yy, t3 * xy);
            const T xyyz = fmadd(d4xy, yz, d3 * xz);
            const T yyyy = fmadd(d4yy, yy, fmadd(t6, yy, t2));
            const T yyyz = fmadd(d4yy, yz, t3 * yz);
            const T xxzz = -(xxxx + xxyy), xyzz = -(xxxy + xyyy), yyzz = -(xxyy + yyyy);
            // slices in the B3 basis (xxx xxy xxz xyy xyz yyy yyz)
            U[0][0] = xxxx; U[0][1] = xxxy; U[0][2] = xxxz; U[0][3] = xxyy;
            U[0][4] = xxyz; U[0][5] = xyyy; U[0][6] = xyyz;
            U[1][0] = xxxy; U[1][1] = xxyy; U[1][2] = xxyz; U[1][3] = xyyy;
            U[1][4] = xyyz; U[1][5] = yyyy; U[1][6] = yyyz;
            U[2][0] = xxxz; U[2][1] = xxyz; U[2][2] = xxzz; U[2][3] = xyyz;
            U[2][4] = xyzz; U[2][5] = yyyz; U[2][6] = yyzz;
        }
    }

    // D3[i, B2 pair] for L1_i = sum_k B2_k D3slice(i, k)
    __device__ __forceinline__ T d3slice(int i, int k) const
    {
        // i = x: xxx xyy xxy xxz xyz ; y: xxy yyy xyy xyz yyz ; z: xxz yyz xyz xzz yzz
        constexpr int idx[3][5] = {{0, 3, 1, 2, 4}, {1, 5, 3, 4, 6}, {2, 6, 4, 7, 8}};
        return D3[idx[i][k]];
    }
};

// paired FP32 subtraction (sub.rn.f32x2: each half rounds as the scalar
// subtraction does)
__device__ __forceinline__ float2 fsub2_rn(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// float: the same values, bit for bit, with the independent products that
// share a form issued in pairs on the paired FP32 pipe (mul/fma.rn.f32x2,
// each half rounding as the scalar instruction does).  The natural pairs are
// the (x, y) and (xz, yz) products of one radial factor; the radial factors
// themselves are scalar and duplicated into pairs where needed.
template <>
struct DTraceless<float> {
    float D0, D1[3];
    float D2[5];             // xx yy xy xz yz
    float D3[9];             // xxx xxy xxz xyy xyz yyy yyz | xzz yzz
    float U[3][7];           // D4 slices for the B3 basis

    template <bool WITH_D4>
    __device__ __forceinline__ void eval(float x, float y, float z)
    {
        const float r2 = fmaf(x, x, fmaf(y, y, z * z));
        const float ri = rsqrt_ftz(r2);
        const float ri2 = ri * ri;
        const float d1 = -ri * ri2;
        const float d2 = d1 * (-3.f * ri2);
        const float d3 = d2 * (-5.f * ri2);
        const float t2 = 3.f * d2;
        const float2 d1p = make_float2(d1, d1), d2p = make_float2(d2, d2);
        const float2 rxy = make_float2(x, y);
        const float2 sq = __fmul2_rn(rxy, rxy);                       // xx, yy
        const float2 xzyz = __fmul2_rn(rxy, make_float2(z, z));       // xz, yz
        const float xy = x * y;
        D0 = ri;
        const float2 d1xy = __fmul2_rn(d1p, rxy);
        D1[0] = d1xy.x; D1[1] = d1xy.y; D1[2] = d1 * z;
        const float2 d2a = __ffma2_rn(d2p, sq, d1p);                   // D2 xx, yy
        const float2 d2b = __fmul2_rn(d2p, xzyz);                      // D2 xz, yz
        D2[0] = d2a.x; D2[1] = d2a.y; D2[2] = d2 * xy; D2[3] = d2b.x; D2[4] = d2b.y;
        const float2 d3xy = __fmul2_rn(make_float2(d3, d3), rxy);     // d3 x, d3 y
        const float2 t2xy = __fmul2_rn(make_float2(t2, t2), rxy);     // t2 x, t2 y
        const float2 d2xy = __fmul2_rn(d2p, rxy);                      // d2 x, d2 y
        const float d2z = d2 * z;
        const float2 d3a = __ffma2_rn(d3xy, sq, t2xy);                 // xxx, yyy
        const float2 d3b = __ffma2_rn(d3xy, xzyz, make_float2(d2z, d2z));   // xxz, yyz
        D3[0] = d3a.x;
        D3[1] = fmaf(d3xy.x, xy, d2xy.y);                              // xxy
        D3[2] = d3b.x;
        D3[3] = fmaf(d3xy.x, sq.y, d2xy.x);                            // xyy
        D3[4] = d3xy.x * xzyz.y;                                       // xyz
        D3[5] = d3a.y;
        D3[6] = d3b.y;
        D3[7] = -(D3[0] + D3[3]);                                      // xzz
        D3[8] = -(D3[1] + D3[5]);                                      // yzz
        if (WITH_D4) {
            const float d4 = d3 * (-7.f * ri2);
            const float t3 = 3.f * d3, t6 = 6.f * d3;
            const float2 d4sq = __fmul2_rn(make_float2(d4, d4), sq);   // d4 xx, d4 yy
            const float d4xy = d4 * xy;
            const float2 q4 = __ffma2_rn(d4sq, sq, __ffma2_rn(make_float2(t6, t6), sq,
                                                              make_float2(t2, t2)));   // xxxx, yyyy
            const float2 z4 = __ffma2_rn(d4sq, xzyz, __fmul2_rn(make_float2(t3, t3), xzyz));
                                                                       // xxxz, yyyz
            const float t3xy = t3 * xy;
            const float xxxx = q4.x, yyyy = q4.y, xxxz = z4.x, yyyz = z4.y;
            const float xxxy = fmaf(d4sq.x, xy, t3xy);
            const float xxyy = fmaf(d4sq.x, sq.y, fmaf(d3, sq.x + sq.y, d2));
            const float2 d3z = __fmul2_rn(make_float2(d3, d3), xzyz);    // d3 xz, d3 yz
            const float xxyz = fmaf(d4sq.x, xzyz.y, d3z.y);
            const float xyyy = fmaf(d4xy, sq.y, t3xy);
            const float xyyz = fmaf(d4xy, xzyz.y, d3z.x);
            const float xxzz = -(xxxx + xxyy), xyzz = -(xxxy + xyyy), yyzz = -(xxyy + yyyy);
            U[0][0] = xxxx; U[0][1] = xxxy; U[0][2] = xxxz; U[0][3] = xxyy;
            U[0][4] = xxyz; U[0][5] = xyyy; U[0][6] = xyyz;
            U[1][0] = xxxy; U[1][1] = xxyy; U[1][2] = xxyz; U[1][3] = xyyy;
            U[1][4] = xyyz; U[1][5] = yyyy; U[1][6] = yyyz;
            U[2][0] = xxxz; U[2][1] = xxyz; U[2][2] = xxzz; U[2][3] = xyyz;
            U[2][4] = xyzz; U[2][5] = yyyz; U[2][6] = yyzz;
        }
    }

    __device__ __forceinline__ float d3slice(int i, int k) const
    {
        constexpr int idx[3][5] = {{0, 3, 1, 2, 4}, {1, 5, 3, 4, 6}, {2, 6, 4, 7, 8}};
        return D3[idx[i][k]];
    }
};

// cell (x,y,z) of a node -> parity-split position
__host__ __device__ __forceinline__ int parity_index(int x, int y, int z)
{
    return ((x & 1) + 2 * (y & 1) + 4 * (z & 1)) * 64 + (x >> 1) + 4 * (y >> 1) + 16 * (z >> 1);
}

// TwoSum (Knuth): s + e == a + b exactly, s = fl(a + b)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

}  // namespace fmm
