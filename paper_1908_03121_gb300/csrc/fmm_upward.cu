// Upward pass (Sec. 4.3, first step): cell masses from the leaf densities,
// then, level by level from the deepest, each refined cell's mass, centre of
// mass and central moments from its eight child cells, in FP64.
//
// GB300's FP64 pipe runs at a small fraction of its FP32 rate, so the kernels
// keep FP64 operation counts low: cell widths come from a per-level table
// (no divisions), and when the eight children are leaf cells -- the bulk of
// the work, at the finest refined level -- their offsets from the parent
// cell centre are exactly (+-h/2, +-h/2, +-h/2), so the raw moments about
// that centre are signed sums of the eight masses (a 3-D Hadamard transform),
// shifted to the centre of mass afterwards.
#include <type_traits>

#include "fmm_convert.cuh"
#include "fmm_internal.h"
#include "fmm_tensor.cuh"

namespace fmm {

namespace {

// the packed same-level mass of a leaf cell, as the pack kernel stores it
template <typename T>
__device__ __forceinline__ T packed_mass(double m)
{
    if constexpr (std::is_same<T, float>::value) {
        return d2f_rn(m);
    } else if constexpr (std::is_same<T, dfloat>::value) {
        return df_from_double(m);
    } else {
        return m;
    }
}

// P2M: leaf cells hold m = rho h^3 at their centre (point-mass reading of a
// locally homogeneous density).  Two cells per thread, cells x-fastest, as
// 16-byte loads and stores: the density may sit in pinned host memory, and
// wider requests keep more of it in flight over the host link.  A density
// that is not positive (zero, negative, NaN) sets FMM_STATUS_BAD_DENSITY in
// the status word: the centres of mass divide by masses.  With a packed-mass
// array (T not void), the kernel also stores the masses in the same-level
// pass's parity-split order and element type, which the pack kernel would
// otherwise do for the leaves in a launch of its own.
template <typename T>
__global__ void __launch_bounds__(NCELL / 2) p2m_kernel(const NodeInfo *__restrict__ info,
                                                        const int32_t *__restrict__ leaves,
                                                        const double *__restrict__ levels,
                                                        const double *__restrict__ rho,
                                                        double *__restrict__ M,
                                                        int32_t *__restrict__ status,
                                                        T *__restrict__ mass)
{
    const int node = leaves[blockIdx.x];
    const NodeInfo ni = info[node];
    const double h3 = levels[ni.level * LEVEL_FIELDS + LV_H3];
    const int c = 2 * threadIdx.x;
    const double2 r = *reinterpret_cast<const double2 *>(rho + size_t(ni.leaf_row) * NCELL + c);
    if (!(r.x > 0.0) || !(r.y > 0.0)) atomicOr(status, FMM_STATUS_BAD_DENSITY);
    const double m0 = r.x * h3, m1 = r.y * h3;
    *reinterpret_cast<double2 *>(M + (size_t(node) * NCOMP) * NCELL + c) = make_double2(m0, m1);
    if constexpr (!std::is_void<T>::value) {
        // cells c and c + 1 differ in x parity only
        const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
        const int pi = parity_index(x, y, z);
        mass[size_t(node) * NCELL + pi] = packed_mass<T>(m0);
        mass[size_t(node) * NCELL + pi + 64] = packed_mass<T>(m1);
    }
}

// Central moments about X = ref + d from raw moments S2, S3 about ref:
//   M2_ij = S2_ij - M0 d_i d_j,
//   M3_ijk = S3_ijk - (S2_ij d_k + S2_ik d_j + S2_jk d_i) + 2 M0 d_i d_j d_k.
// T = double (fused multiply-adds) or dfloat.
template <typename T>
__device__ __forceinline__ void central_from_raw(T m0, const T d[3], const T S2[6], const T S3[10],
                                                 T M2[6], T M3[10])
{
    // the products m0 d_i d_j serve both orders
    const T md[3] = {m0 * d[0], m0 * d[1], m0 * d[2]};
    T mdd[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) mdd[q] = md[i2_at(q, 0)] * d[i2_at(q, 1)];
#pragma unroll
    for (int q = 0; q < 6; ++q) M2[q] = S2[q] - mdd[q];
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        const int a = i3_at(q, 0), b = i3_at(q, 1), c = i3_at(q, 2);
        T v = S3[q] + (mdd[r2_of(a, b)] + mdd[r2_of(a, b)]) * d[c];
        v = v - S2[r2_of(a, b)] * d[c];
        v = v - S2[r2_of(a, c)] * d[b];
        M3[q] = v - S2[r2_of(b, c)] * d[a];
    }
}

// M2M: parent cell (x,y,z) of a refined node takes the 2x2x2 child cells of
// child node (x>>2, y>>2, z>>2) at child-local (2(x&3)+dx, ...):
//   M0 = sum m_c,  X = sum m_c X_c / M0,  s_c = X_c - X,
//   M2_ij  = sum (M2c_ij + m_c s_i s_j),
//   M3_ijk = sum (M3c_ijk + M2c_ij s_k + M2c_ik s_j + M2c_jk s_i + m_c s_i s_j s_k).
// 64 threads per CTA, 8 CTAs per node: coarse levels have few nodes, and
// spreading each node over 8 SMs keeps their FP64 work off a single SM
constexpr int kSliceThreads = 64;

__global__ void __launch_bounds__(kSliceThreads) m2m_kernel(const NodeInfo *__restrict__ info,
                                                            const int32_t *__restrict__ children,
                                                            const int32_t *__restrict__ nodes,
                                                            const double *__restrict__ levels,
                                                            double *__restrict__ M,
                                                            double *__restrict__ com, double lo_x,
                                                            double lo_y, double lo_z)
{
    const int node = nodes[blockIdx.x >> 3];
    const NodeInfo ni = info[node];
    const int c = (blockIdx.x & 7) * kSliceThreads + threadIdx.x;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const int k = (x >> 2) + 2 * (y >> 2) + 4 * (z >> 2);
    const int ch = children[node * 8 + k];
    const bool child_leaf = info[ch].leaf_row >= 0;
    const double hp = levels[ni.level * LEVEL_FIELDS + LV_H];
    const double q = 0.25 * hp;                 // half a child cell width
    const double ref[3] = {lo_x + (8.0 * ni.ix + x + 0.5) * hp, lo_y + (8.0 * ni.iy + y + 0.5) * hp,
                           lo_z + (8.0 * ni.iz + z + 0.5) * hp};
    const size_t cbase = size_t(ch) * NCOMP * NCELL;
    const int c0 = 2 * (x & 3) + 16 * (y & 3) + 128 * (z & 3);   // child cell of j = 0
    double m0, d[3], M2[6], M3[10];
    if (child_leaf) {
        // child j sits at ref + q (e_x, e_y, e_z), e = +-1 from the bits of j
        double m[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            m[j] = M[cbase + c0 + (j & 1) + 8 * ((j >> 1) & 1) + 64 * (j >> 2)];
        // Hadamard transform over the three sign bits
        double a[8];
#pragma unroll
        for (int j = 0; j < 8; j += 2) { a[j] = m[j] + m[j + 1]; a[j + 1] = m[j + 1] - m[j]; }
        double b[8];
#pragma unroll
        for (int j = 0; j < 8; j += 4)
#pragma unroll
            for (int i = 0; i < 2; ++i) { b[j + i] = a[j + i] + a[j + i + 2]; b[j + i + 2] = a[j + i + 2] - a[j + i]; }
        double e[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) { e[i] = b[i] + b[i + 4]; e[i + 4] = b[i + 4] - b[i]; }
        // e[bits] = sum_j m_j prod_{axis in bits} e_axis(j): 0 -> M0, 1 -> Ex,
        // 2 -> Ey, 3 -> Exy, 4 -> Ez, 5 -> Exz, 6 -> Eyz, 7 -> Exyz
        m0 = e[0];
        const double im0 = 1.0 / m0;
        d[0] = q * e[1] * im0;
        d[1] = q * e[2] * im0;
        d[2] = q * e[4] * im0;
        const double q2 = q * q, q3 = q2 * q;
        const double S2[6] = {q2 * m0, q2 * e[3], q2 * e[5], q2 * m0, q2 * e[6], q2 * m0};
        const double S3[10] = {q3 * e[1], q3 * e[2], q3 * e[4], q3 * e[1], q3 * e[7],
                               q3 * e[1], q3 * e[2], q3 * e[4], q3 * e[2], q3 * e[4]};
        central_from_raw(m0, d, S2, S3, M2, M3);
    } else {
        double mj[8], X[8][3];
        m0 = 0.0;
        double mr[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int cc = c0 + (j & 1) + 8 * ((j >> 1) & 1) + 64 * (j >> 2);
            mj[j] = M[cbase + cc];
#pragma unroll
            for (int t = 0; t < 3; ++t) X[j][t] = com[(size_t(ch) * 3 + t) * NCELL + cc] - ref[t];
            m0 += mj[j];
#pragma unroll
            for (int t = 0; t < 3; ++t) mr[t] += mj[j] * X[j][t];
        }
        const double im0 = 1.0 / m0;
#pragma unroll
        for (int t = 0; t < 3; ++t) d[t] = mr[t] * im0;
        constexpr int I2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
        constexpr int I3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                                   {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
#pragma unroll
        for (int t = 0; t < 6; ++t) M2[t] = 0.0;
#pragma unroll
        for (int t = 0; t < 10; ++t) M3[t] = 0.0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int cc = c0 + (j & 1) + 8 * ((j >> 1) & 1) + 64 * (j >> 2);
            const double s[3] = {X[j][0] - d[0], X[j][1] - d[1], X[j][2] - d[2]};
            double c2[6];
#pragma unroll
            for (int t = 0; t < 6; ++t) c2[t] = M[cbase + (4 + t) * NCELL + cc];
#pragma unroll
            for (int t = 0; t < 6; ++t) M2[t] += c2[t] + mj[j] * s[I2[t][0]] * s[I2[t][1]];
#pragma unroll
            for (int t = 0; t < 10; ++t) {
                const int a = I3[t][0], b = I3[t][1], e = I3[t][2];
                M3[t] += M[cbase + (10 + t) * NCELL + cc] + c2[r2_of(a, b)] * s[e] +
                         c2[r2_of(a, e)] * s[b] + c2[r2_of(b, e)] * s[a] + mj[j] * s[a] * s[b] * s[e];
            }
        }
    }
    double *out = M + size_t(node) * NCOMP * NCELL + c;
    out[0] = m0;
    out[1 * NCELL] = 0.0;
    out[2 * NCELL] = 0.0;
    out[3 * NCELL] = 0.0;
#pragma unroll
    for (int t = 0; t < 6; ++t) out[(4 + t) * NCELL] = M2[t];
#pragma unroll
    for (int t = 0; t < 10; ++t) out[(10 + t) * NCELL] = M3[t];
#pragma unroll
    for (int t = 0; t < 3; ++t) com[(size_t(node) * 3 + t) * NCELL + c] = ref[t] + d[t];
}

// The mixed and double-float precisions run the upward pass in double-float
// arithmetic (about 48 bits, on the FP32 pipe).  A refined node also leaves
// its results as double-float pairs in the `up` workspace, up[row][20][512] =
// (M0, centre-of-mass offset from the cell centre, M2, M3), which its parent
// reads without conversion; a child cell's offset from the parent cell's
// centre is then exactly (+-q, +-q, +-q) plus its own centre-of-mass offset
// (q = half a child width).  The FP64 operations left per parent cell are the
// splits of leaf-child masses (one subtraction each) and the conversions of
// the 17 moments and 3 coordinates written to M and com (one add each).
// Two launch shapes: one thread per parent cell (the recurrences above, with
// the Hadamard transform for leaf children) for levels with many nodes, and
// eight threads per parent cell for levels with few, where one thread's long
// dependent sequence of double-float operations would set the time.
__device__ __forceinline__ void write_up(const NodeInfo &ni, int node, int c, int x, int y, int z,
                                         double hp, const dfloat &m0, const dfloat d[3],
                                         const dfloat M2[6], const dfloat M3[10], double *M,
                                         double *com, dfloat *up, double lo_x, double lo_y,
                                         double lo_z)
{
    double *out = M + size_t(node) * NCOMP * NCELL + c;
    out[0] = df_to_double(m0);
    out[1 * NCELL] = 0.0;
    out[2 * NCELL] = 0.0;
    out[3 * NCELL] = 0.0;
#pragma unroll
    for (int t = 0; t < 6; ++t) out[(4 + t) * NCELL] = df_to_double(M2[t]);
#pragma unroll
    for (int t = 0; t < 10; ++t) out[(10 + t) * NCELL] = df_to_double(M3[t]);
    double *cm = com + size_t(node) * 3 * NCELL + c;
    cm[0] = fma(f2d_bits(float(8 * ni.ix + x) + 0.5f), hp, lo_x) + df_to_double(d[0]);
    cm[NCELL] = fma(f2d_bits(float(8 * ni.iy + y) + 0.5f), hp, lo_y) + df_to_double(d[1]);
    cm[2 * NCELL] = fma(f2d_bits(float(8 * ni.iz + z) + 0.5f), hp, lo_z) + df_to_double(d[2]);
    dfloat *ou = up + size_t(ni.mp_row) * 20 * NCELL + c;
    ou[0] = m0;
#pragma unroll
    for (int t = 0; t < 3; ++t) ou[(1 + t) * NCELL] = d[t];
#pragma unroll
    for (int t = 0; t < 6; ++t) ou[(4 + t) * NCELL] = M2[t];
#pragma unroll
    for (int t = 0; t < 10; ++t) ou[(10 + t) * NCELL] = M3[t];
}

// one thread per parent cell, 8 CTAs of 64 threads per node.  LEAF_KIDS:
// every child of the launch's nodes is a leaf (the deepest refined level,
// the bulk of the upward pass's cells), so only the leaf-children branch is
// compiled: far fewer registers than the general kernel, which lets the
// launch share its SMs with the persistent monopole kernel that runs beside
// the upward pass in fmm_step.
template <bool LEAF_KIDS>
__global__ void __launch_bounds__(kSliceThreads) m2m_df_kernel(const NodeInfo *__restrict__ info,
                                                               const int32_t *__restrict__ children,
                                                               const int32_t *__restrict__ nodes,
                                                               const double *__restrict__ levels,
                                                               double *__restrict__ M,
                                                               double *__restrict__ com,
                                                               dfloat *__restrict__ up, double lo_x,
                                                               double lo_y, double lo_z)
{
    const int node = nodes[blockIdx.x >> 3];
    const NodeInfo ni = info[node];
    const int c = (blockIdx.x & 7) * kSliceThreads + threadIdx.x;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const int k = (x >> 2) + 2 * (y >> 2) + 4 * (z >> 2);
    const int ch = children[node * 8 + k];
    const NodeInfo ci = info[ch];
    const double hp = levels[ni.level * LEVEL_FIELDS + LV_H];
    const dfloat q = df_from_double(0.25 * hp);           // half a child cell width
    const int c0 = 2 * (x & 3) + 16 * (y & 3) + 128 * (z & 3);   // child cell of j = 0
    dfloat m0, d[3], M2[6], M3[10];
    if (LEAF_KIDS || ci.leaf_row >= 0) {
        // child j sits at ref + q (e_x, e_y, e_z), e = +-1 from the bits of j
        const size_t cbase = size_t(ch) * NCOMP * NCELL;
        dfloat m[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            m[j] = df_from_double(M[cbase + c0 + (j & 1) + 8 * ((j >> 1) & 1) + 64 * (j >> 2)]);
        dfloat a[8];
#pragma unroll
        for (int j = 0; j < 8; j += 2) { a[j] = m[j] + m[j + 1]; a[j + 1] = m[j + 1] - m[j]; }
        dfloat b[8];
#pragma unroll
        for (int j = 0; j < 8; j += 4)
#pragma unroll
            for (int i = 0; i < 2; ++i) { b[j + i] = a[j + i] + a[j + i + 2]; b[j + i + 2] = a[j + i + 2] - a[j + i]; }
        dfloat e[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) { e[i] = b[i] + b[i + 4]; e[i + 4] = b[i + 4] - b[i]; }
        m0 = e[0];
        const dfloat qm = q / m0;
        d[0] = qm * e[1];
        d[1] = qm * e[2];
        d[2] = qm * e[4];
        const dfloat q2 = q * q, q3 = q2 * q;
        const dfloat q2m = q2 * m0;
        const dfloat S2[6] = {q2m, q2 * e[3], q2 * e[5], q2m, q2 * e[6], q2m};
        const dfloat q3x = q3 * e[1], q3y = q3 * e[2], q3z = q3 * e[4];
        const dfloat S3[10] = {q3x, q3y, q3z, q3x, q3 * e[7], q3x, q3y, q3z, q3y, q3z};
        central_from_raw(m0, d, S2, S3, M2, M3);
    } else if constexpr (!LEAF_KIDS) {
        const dfloat *cu = up + size_t(ci.mp_row) * 20 * NCELL;
        dfloat mj[8], X[8][3];
        m0 = dfloat(0.f);
        dfloat mr[3] = {dfloat(0.f), dfloat(0.f), dfloat(0.f)};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int cc = c0 + (j & 1) + 8 * ((j >> 1) & 1) + 64 * (j >> 2);
            mj[j] = cu[cc];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const dfloat sq = ((j >> t) & 1) ? q : -q;
                X[j][t] = sq + cu[(1 + t) * NCELL + cc];
            }
            m0 += mj[j];
#pragma unroll
            for (int t = 0; t < 3; ++t) mr[t] += mj[j] * X[j][t];
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) d[t] = mr[t] / m0;
#pragma unroll
        for (int t = 0; t < 6; ++t) M2[t] = dfloat(0.f);
#pragma unroll
        for (int t = 0; t < 10; ++t) M3[t] = dfloat(0.f);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int cc = c0 + (j & 1) + 8 * ((j >> 1) & 1) + 64 * (j >> 2);
            const dfloat s3[3] = {X[j][0] - d[0], X[j][1] - d[1], X[j][2] - d[2]};
            const dfloat ms[3] = {mj[j] * s3[0], mj[j] * s3[1], mj[j] * s3[2]};
            dfloat c2[6];
#pragma unroll
            for (int t = 0; t < 6; ++t) c2[t] = cu[(4 + t) * NCELL + cc];
            dfloat mss[6];
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                mss[t] = ms[i2_at(t, 0)] * s3[i2_at(t, 1)];
                M2[t] += c2[t] + mss[t];
            }
#pragma unroll
            for (int t = 0; t < 10; ++t) {
                const int a = i3_at(t, 0), b = i3_at(t, 1), e = i3_at(t, 2);
                M3[t] += cu[(10 + t) * NCELL + cc] + c2[r2_of(a, b)] * s3[e] + c2[r2_of(a, e)] * s3[b] +
                         c2[r2_of(b, e)] * s3[a] + mss[r2_of(a, b)] * s3[e];
            }
        }
    }
    write_up(ni, node, c, x, y, z, hp, m0, d, M2, M3, M, com, up, lo_x, lo_y, lo_z);
}

// eight threads per parent cell, one per child cell: each forms its child's
// raw moments about the parent cell's centre ref,
//   m,  m X,  M2c + m X X,  M3c + (M2c X, three terms) + m X X X,
// X = child centre of mass - ref (a leaf child's M2c, M3c vanish), the eight
// are summed by a butterfly of shuffles (every lane ends with the same sums:
// double-float addition is commutative), and every lane turns them into
// central moments about X = ref + m X / m and writes its share of the outputs.
constexpr int kCellsPerCta = 8;
// levels with fewer refined nodes than this take eight threads per cell
constexpr int64_t kLanesBelow = 128;

__device__ __forceinline__ dfloat shfl_xor_df(dfloat v, int mask)
{
    return dfloat(__shfl_xor_sync(0xffffffffu, v.hi, mask), __shfl_xor_sync(0xffffffffu, v.lo, mask));
}

__global__ void __launch_bounds__(8 * kCellsPerCta) m2m_df_lanes_kernel(const NodeInfo *__restrict__ info,
                                                                  const int32_t *__restrict__ children,
                                                                  const int32_t *__restrict__ nodes,
                                                                  const double *__restrict__ levels,
                                                                  double *__restrict__ M,
                                                                  double *__restrict__ com,
                                                                  dfloat *__restrict__ up, double lo_x,
                                                                  double lo_y, double lo_z)
{
    constexpr int kCtasPerNode = NCELL / kCellsPerCta;
    const int node = nodes[blockIdx.x / kCtasPerNode];
    const NodeInfo ni = info[node];
    const int c = (blockIdx.x % kCtasPerNode) * kCellsPerCta + (threadIdx.x >> 3);
    const int j = threadIdx.x & 7;                            // child cell of this lane
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const int k = (x >> 2) + 2 * (y >> 2) + 4 * (z >> 2);
    const int ch = children[node * 8 + k];
    const NodeInfo ci = info[ch];
    const double hp = levels[ni.level * LEVEL_FIELDS + LV_H];
    const dfloat q = df_from_double(0.25 * hp);
    const int cc = 2 * (x & 3) + 16 * (y & 3) + 128 * (z & 3) + (j & 1) + 8 * ((j >> 1) & 1) +
                   64 * (j >> 2);
    dfloat X[3], m, c2[6], c3[10];
#pragma unroll
    for (int t = 0; t < 3; ++t) X[t] = ((j >> t) & 1) ? q : -q;
    if (ci.leaf_row >= 0) {
        m = df_from_double(M[size_t(ch) * NCOMP * NCELL + cc]);
#pragma unroll
        for (int t = 0; t < 6; ++t) c2[t] = dfloat(0.f);
#pragma unroll
        for (int t = 0; t < 10; ++t) c3[t] = dfloat(0.f);
    } else {
        const dfloat *cu = up + size_t(ci.mp_row) * 20 * NCELL + cc;
        m = cu[0];
#pragma unroll
        for (int t = 0; t < 3; ++t) X[t] += cu[(1 + t) * NCELL];
#pragma unroll
        for (int t = 0; t < 6; ++t) c2[t] = cu[(4 + t) * NCELL];
#pragma unroll
        for (int t = 0; t < 10; ++t) c3[t] = cu[(10 + t) * NCELL];
    }
    // raw moments of this child about ref: v = (m, m X, S2, S3)
    dfloat v[20];
    v[0] = m;
#pragma unroll
    for (int t = 0; t < 3; ++t) v[1 + t] = m * X[t];
#pragma unroll
    for (int t = 0; t < 6; ++t) v[4 + t] = c2[t] + v[1 + i2_at(t, 0)] * X[i2_at(t, 1)];
#pragma unroll
    for (int t = 0; t < 10; ++t) {
        const int a = i3_at(t, 0), b = i3_at(t, 1), e = i3_at(t, 2);
        v[10 + t] = c3[t] + c2[r2_of(a, b)] * X[e] + c2[r2_of(a, e)] * X[b] + c2[r2_of(b, e)] * X[a] +
                    (v[1 + a] * X[b]) * X[e];
    }
#pragma unroll
    for (int off = 1; off < 8; off <<= 1)
#pragma unroll
        for (int t = 0; t < 20; ++t) v[t] += shfl_xor_df(v[t], off);
    const dfloat m0 = v[0];
    dfloat d[3], M2[6], M3[10];
#pragma unroll
    for (int t = 0; t < 3; ++t) d[t] = v[1 + t] / m0;
    central_from_raw(m0, d, v + 4, v + 10, M2, M3);
    // lane j writes components j, j + 8, j + 16 of (M0, offset, M2, M3), and
    // lanes 0-3 the FP64 dipole zeros, lanes 4-6 the centre of mass
    const dfloat outv[20] = {m0,    d[0],  d[1],  d[2],  M2[0], M2[1], M2[2], M2[3], M2[4], M2[5],
                             M3[0], M3[1], M3[2], M3[3], M3[4], M3[5], M3[6], M3[7], M3[8], M3[9]};
    double *out = M + size_t(node) * NCOMP * NCELL + c;
    dfloat *ou = up + size_t(ni.mp_row) * 20 * NCELL + c;
#pragma unroll
    for (int comp = 0; comp < 20; ++comp) {
        if ((comp & 7) != j) continue;
        ou[comp * NCELL] = outv[comp];
        if (comp == 0 || comp >= 4) out[comp * NCELL] = df_to_double(outv[comp]);
    }
    if (j >= 1 && j <= 3) out[j * NCELL] = 0.0;
    double *cm = com + size_t(node) * 3 * NCELL + c;
    if (j == 4) cm[0] = (lo_x + (8.0 * ni.ix + x + 0.5) * hp) + df_to_double(d[0]);
    if (j == 5) cm[NCELL] = (lo_y + (8.0 * ni.iy + y + 0.5) * hp) + df_to_double(d[1]);
    if (j == 6) cm[2 * NCELL] = (lo_z + (8.0 * ni.iz + z + 0.5) * hp) + df_to_double(d[2]);
}

}  // namespace

cudaError_t launch_p2m(const fmm_tree_s *t, const double *rho, double *M, cudaStream_t s,
                       bool pack_leaves)
{
    const ListRange &r = t->plan.leaves;
    if (r.count == 0) return cudaSuccess;
    // 16-byte accesses: rho and M must be 16-byte aligned (checked by the
    // public calls)
    const unsigned grid = unsigned(r.count);
    const int32_t *leaves = t->dev.lists + r.off;
    int32_t *status = t->dev.counters + kStatusSlot;
    if (!pack_leaves)
        p2m_kernel<void><<<grid, NCELL / 2, 0, s>>>(t->dev.info, leaves, t->dev.levels, rho, M,
                                                   status, nullptr);
    else if (t->cfg.precision == FMM_MIXED)
        p2m_kernel<float><<<grid, NCELL / 2, 0, s>>>(t->dev.info, leaves, t->dev.levels, rho, M,
                                                    status, static_cast<float *>(t->dev.mass));
    else if (t->cfg.precision == FMM_DFLOAT)
        p2m_kernel<dfloat><<<grid, NCELL / 2, 0, s>>>(t->dev.info, leaves, t->dev.levels, rho, M,
                                                     status, static_cast<dfloat *>(t->dev.mass));
    else
        p2m_kernel<double><<<grid, NCELL / 2, 0, s>>>(t->dev.info, leaves, t->dev.levels, rho, M,
                                                     status, static_cast<double *>(t->dev.mass));
    return cudaGetLastError();
}

cudaError_t launch_m2m_level(const fmm_tree_s *t, int level, double *M, double *com,
                             cudaStream_t s)
{
    const ListRange &r = t->plan.refined_at[size_t(level)];
    if (r.count == 0) return cudaSuccess;
    if (t->cfg.precision != FMM_FP64 && r.count >= kLanesBelow) {
        // nodes with only leaf children through the lean kernel, the others
        // through the general one
        const ListRange &rl = t->plan.leafkids_at[size_t(level)];
        const ListRange &rm = t->plan.mixedkids_at[size_t(level)];
        if (rl.count)
            m2m_df_kernel<true><<<unsigned(rl.count * 8), kSliceThreads, 0, s>>>(
                t->dev.info, t->dev.children, t->dev.lists + rl.off, t->dev.levels, M, com,
                reinterpret_cast<dfloat *>(t->dev.up), t->cfg.box_lo[0], t->cfg.box_lo[1],
                t->cfg.box_lo[2]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess || rm.count == 0) return e;
        m2m_df_kernel<false><<<unsigned(rm.count * 8), kSliceThreads, 0, s>>>(
            t->dev.info, t->dev.children, t->dev.lists + rm.off, t->dev.levels, M, com,
            reinterpret_cast<dfloat *>(t->dev.up), t->cfg.box_lo[0], t->cfg.box_lo[1],
            t->cfg.box_lo[2]);
        return cudaGetLastError();
    }
    if (t->cfg.precision != FMM_FP64) {
        m2m_df_lanes_kernel<<<unsigned(r.count * (NCELL / kCellsPerCta)), 8 * kCellsPerCta, 0, s>>>(
            t->dev.info, t->dev.children, t->dev.lists + r.off, t->dev.levels, M, com,
            reinterpret_cast<dfloat *>(t->dev.up), t->cfg.box_lo[0], t->cfg.box_lo[1],
            t->cfg.box_lo[2]);
        return cudaGetLastError();
    }
    m2m_kernel<<<unsigned(r.count * 8), kSliceThreads, 0, s>>>(t->dev.info, t->dev.children,
                                                               t->dev.lists + r.off,
                                                 t->dev.levels, M, com, t->cfg.box_lo[0],
                                                 t->cfg.box_lo[1], t->cfg.box_lo[2]);
    return cudaGetLastError();
}

}  // namespace fmm
