// Downward pass (Sec. 4.3, third step) and leaf forces.
//
// l2l_kernel, one launch per level from the root down: each cell converts its
// own same-level result from level units to physical units, adds its parent's
// final expansion re-centred at its own centre of mass,
//   L^(n) += sum_{k=0}^{3-n} (1/k!) L_parent^(n+k) . d^k,  d = X - X_parent,
// and inherits the parent's accumulated angular-momentum correction.  The
// FP64 precision accumulates in FP64 and the double-float one with one FP64
// operation per component; in the mixed precision the shift increments (the
// k >= 1 terms, small next to the parent's own coefficient) are formed in
// float and the final expansion in double-float from the parent's
// double-float copy, so GB300's slow FP64 pipe does one add per component
// (forming L64).  The correction is carried in FP64 in every precision.
// forces_kernel: phi = L0, g = -(L1 + dL1), f = m g, and fixed-order FP64
// block sums of f and x cross f (plus the |f|, |x cross f| normalisers) per
// leaf node; reduce_chunk_kernel and reduce_final_kernel fold those per tree.
#include "fmm_convert.cuh"
#include "fmm_internal.h"
#include "fmm_tensor.cuh"

namespace fmm {

namespace {

// shift increments of a parent expansion P by d (orders up to NMAX), i.e.
// everything in L'^(n) - P^(n); in the precision of T
template <typename T, int NMAX>
__device__ __forceinline__ void shift_increments(const T P[20], const T d[3], T out[20])
{
    const T dd[6] = {d[0] * d[0], d[0] * d[1], d[0] * d[2], d[1] * d[1], d[1] * d[2], d[2] * d[2]};
    // order 0: P1.d + 1/2 P2:dd + 1/6 P3:ddd
    T v0 = P[1] * d[0];
#pragma unroll
    for (int i = 1; i < 3; ++i) v0 = fmadd(P[1 + i], d[i], v0);
#pragma unroll
    for (int q = 0; q < 6; ++q) v0 = fmadd(T(0.5 * mult2(q)) * P[4 + q], dd[q], v0);
#pragma unroll
    for (int q = 0; q < 10; ++q)
        v0 = fmadd(T(mult3(q) / 6.0) * P[10 + q], dd[r2_of(i3_at(q, 0), i3_at(q, 1))] * d[i3_at(q, 2)],
                   v0);
    out[0] = v0;
    // order 1: P2_ij d_j + 1/2 P3_ijk d_j d_k
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T v = P[4 + r2_of(i, 0)] * d[0];
#pragma unroll
        for (int j = 1; j < 3; ++j) v = fmadd(P[4 + r2_of(i, j)], d[j], v);
#pragma unroll
        for (int q = 0; q < 6; ++q) v = fmadd(T(0.5 * mult2(q)) * P[10 + r3_of(i, q)], dd[q], v);
        out[1 + i] = v;
    }
    if (NMAX >= 2) {
        // order 2: P3_ijk d_k ; order 3: nothing
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            T v = P[10 + r3_ijk(i2_at(q, 0), i2_at(q, 1), 0)] * d[0];
#pragma unroll
            for (int k = 1; k < 3; ++k) v = fmadd(P[10 + r3_ijk(i2_at(q, 0), i2_at(q, 1), k)], d[k], v);
            out[4 + q] = v;
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) out[10 + q] = T(0);
    }
}

// FP64 path: the whole re-centring in double.
template <int NMAX>
__device__ __forceinline__ void l2l_cell_fp64(const NodeInfo &ni, int node, int c,
                                              const double *__restrict__ lv,
                                              const void *__restrict__ Lv, const double *dL1,
                                              const double *__restrict__ com,
                                              double *__restrict__ L64, double *dacc, double lo_x,
                                              double lo_y, double lo_z, double (&out)[20],
                                              double (&corr)[3])
{
    constexpr int NK = NMAX == 1 ? 4 : 20;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const double *L = lv + ni.level * LEVEL_FIELDS;
    const double sc[4] = {L[LV_S0], L[LV_S1], L[LV_S2], L[LV_S3]};
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const size_t idx = (size_t(node) * NCOMP + k) * NCELL + c;
        const double own = static_cast<const double *>(Lv)[idx];
        out[k] = own * sc[k == 0 ? 0 : k < 4 ? 1 : k < 10 ? 2 : 3];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) corr[a] = dL1[(size_t(node) * 3 + a) * NCELL + c] * sc[1];
    if (ni.parent >= 0) {
        const int pc = (4 * (ni.ix & 1) + (x >> 1)) + 8 * (4 * (ni.iy & 1) + (y >> 1)) +
                       64 * (4 * (ni.iz & 1) + (z >> 1));
        double X[3];
        if (NMAX == 1) {                      // leaf cell: centre of mass = centre
            const double h = L[LV_H];
            X[0] = lo_x + (8.0 * ni.ix + x + 0.5) * h;
            X[1] = lo_y + (8.0 * ni.iy + y + 0.5) * h;
            X[2] = lo_z + (8.0 * ni.iz + z + 0.5) * h;
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) X[a] = com[(size_t(node) * 3 + a) * NCELL + c];
        }
        double d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = X[a] - com[(size_t(ni.parent) * 3 + a) * NCELL + pc];
        double P[20];
#pragma unroll
        for (int k = 0; k < 20; ++k) P[k] = L64[(size_t(ni.parent) * NCOMP + k) * NCELL + pc];
        double inc[20];
        shift_increments<double, NMAX>(P, d, inc);
#pragma unroll
        for (int k = 0; k < NK; ++k) out[k] += P[k] + inc[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) corr[a] += dacc[(size_t(ni.parent) * 3 + a) * NCELL + pc];
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) L64[(size_t(node) * NCOMP + k) * NCELL + c] = out[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) dacc[(size_t(node) * 3 + a) * NCELL + c] = corr[a];
}

// Mixed path.  The parent level left a float copy of each refined cell's
// final expansion and of its centre-of-mass offset from the cell centre in
// `down`, so the shift d = (child centre - parent centre) + child offset -
// parent offset (the first term is exactly +-h/2 per axis) and the
// increments are formed in float; they are folded into the cell's own
// (hi, lo) level-unit pair by TwoSum, and the one FP64 operation per
// component is the final accumulation L64 = (hi + lo) G h^-(n+1) + L64_parent.
template <int NMAX>
__device__ __forceinline__ void l2l_cell_mixed(const NodeInfo &ni, int node, int c,
                                               const NodeInfo *__restrict__ info,
                                               const double *__restrict__ lv,
                                               const dfloat *__restrict__ lvdf,
                                               const float *__restrict__ Lhi,
                                               const float *__restrict__ Llo, const double *dL1,
                                               const double *__restrict__ com,
                                               double *__restrict__ L64, double *dacc,
                                               dfloat *__restrict__ down, double lo_x,
                                               double lo_y, double lo_z, double (&out)[20],
                                               double (&corr)[3])
{
    constexpr int NK = NMAX == 1 ? 4 : 20;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const double *L = lv + ni.level * LEVEL_FIELDS;
    const dfloat *Ld = lvdf + ni.level * LEVEL_DF_FIELDS;
    const double sc1 = L[LV_S1];
    float hi[20], lo[20];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const size_t idx = (size_t(node) * NCOMP + k) * NCELL + c;
        hi[k] = Lhi[idx];
        lo[k] = Llo[idx];
    }
    float offc[3] = {0.f, 0.f, 0.f};          // own centre-of-mass offset
    if (NMAX == 3) {
        const double h = L[LV_H];
        offc[0] = d2f_trunc(com[(size_t(node) * 3 + 0) * NCELL + c] - (lo_x + (8.0 * ni.ix + x + 0.5) * h));
        offc[1] = d2f_trunc(com[(size_t(node) * 3 + 1) * NCELL + c] - (lo_y + (8.0 * ni.iy + y + 0.5) * h));
        offc[2] = d2f_trunc(com[(size_t(node) * 3 + 2) * NCELL + c] - (lo_z + (8.0 * ni.iz + z + 0.5) * h));
    }
    // the cell's final expansion in double-float: own (level units) x scale
    // + the parent's final expansion, which the parent level left in `down`
    // as (hi, lo) pairs; one FP64 add per component then forms L64
    dfloat res[20];
    if (ni.parent >= 0) {
        const int pc = (4 * (ni.ix & 1) + (x >> 1)) + 8 * (4 * (ni.iy & 1) + (y >> 1)) +
                       64 * (4 * (ni.iz & 1) + (z >> 1));
        const int prow = info[ni.parent].mp_row;
        const dfloat *pd = down + size_t(prow) * 23 * NCELL + pc;
        float Pf[20];
        dfloat Pb[20];
#pragma unroll
        for (int k = 0; k < 20; ++k) {
            const dfloat v = pd[k * NCELL];
            Pf[k] = v.hi;
            if (k < NK) Pb[k] = v;
        }
        const float hc = d2f_trunc(L[LV_H]);
        const float d[3] = {(float(x & 1) - 0.5f) * hc + offc[0] - pd[20 * NCELL].hi,
                            (float(y & 1) - 0.5f) * hc + offc[1] - pd[21 * NCELL].hi,
                            (float(z & 1) - 0.5f) * hc + offc[2] - pd[22 * NCELL].hi};
        float inc[20];
        shift_increments<float, NMAX>(Pf, d, inc);
        const float rs[4] = {d2f_trunc(L[LV_R0]), d2f_trunc(L[LV_R1]), d2f_trunc(L[LV_R2]),
                             d2f_trunc(L[LV_R3])};
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            float s, e;
            two_sum(hi[k], inc[k] * rs[k == 0 ? 0 : k < 4 ? 1 : k < 10 ? 2 : 3], s, e);
            hi[k] = s;
            lo[k] += e;
        }
#pragma unroll
        for (int k = 0; k < NK; ++k)
            res[k] = fmadd(dfloat(hi[k], lo[k]), Ld[5 + (k == 0 ? 0 : k < 4 ? 1 : k < 10 ? 2 : 3)],
                           Pb[k]);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            corr[a] = fma(dL1[(size_t(node) * 3 + a) * NCELL + c], sc1,
                          dacc[(size_t(ni.parent) * 3 + a) * NCELL + pc]);
    } else {
#pragma unroll
        for (int k = 0; k < NK; ++k)
            res[k] = dfloat(hi[k], lo[k]) * Ld[5 + (k == 0 ? 0 : k < 4 ? 1 : k < 10 ? 2 : 3)];
#pragma unroll
        for (int a = 0; a < 3; ++a) corr[a] = dL1[(size_t(node) * 3 + a) * NCELL + c] * sc1;
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        out[k] = df_to_double(res[k]);
        L64[(size_t(node) * NCOMP + k) * NCELL + c] = out[k];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) dacc[(size_t(node) * 3 + a) * NCELL + c] = corr[a];
    if (NMAX == 3) {
        dfloat *od = down + size_t(ni.mp_row) * 23 * NCELL + c;
#pragma unroll
        for (int k = 0; k < 20; ++k) od[k * NCELL] = res[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) od[(20 + a) * NCELL] = dfloat(offc[a]);
    }
}

// Double-float precision: the shift increments are formed in double-float
// (about 48 bits, FP32 pipe) from double-float copies of the parent's final
// expansion and centre-of-mass offset (`down`, written by the parent level),
// folded into the cell's own (hi, lo) level-unit pair, and the one FP64
// operation per component is again the final accumulation
// L64 = (own + increments) G h^-(n+1) + L64_parent.
template <int NMAX>
__device__ __forceinline__ void l2l_cell_df(const NodeInfo &ni, int node, int c,
                                            const NodeInfo *__restrict__ info,
                                            const double *__restrict__ lv,
                                            const dfloat *__restrict__ lvdf,
                                            const float *__restrict__ Lhi,
                                            const float *__restrict__ Llo, const double *dL1,
                                            const double *__restrict__ com,
                                            double *__restrict__ L64, double *dacc,
                                            dfloat *__restrict__ down, double lo_x, double lo_y,
                                            double lo_z, double (&out)[20], double (&corr)[3])
{
    constexpr int NK = NMAX == 1 ? 4 : 20;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const double *L = lv + ni.level * LEVEL_FIELDS;
    const dfloat *Ld = lvdf + ni.level * LEVEL_DF_FIELDS;
    const double sc[4] = {L[LV_S0], L[LV_S1], L[LV_S2], L[LV_S3]};
    dfloat own[20];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const size_t idx = (size_t(node) * NCOMP + k) * NCELL + c;
        own[k] = dfloat(Lhi[idx], Llo[idx]);
    }
    dfloat offc[3] = {dfloat(0.f), dfloat(0.f), dfloat(0.f)};   // own centre-of-mass offset
    if (NMAX == 3) {
        const double h = L[LV_H];
        offc[0] = df_from_double(com[(size_t(node) * 3 + 0) * NCELL + c] -
                                 fma(f2d_bits(float(8 * ni.ix + x) + 0.5f), h, lo_x));
        offc[1] = df_from_double(com[(size_t(node) * 3 + 1) * NCELL + c] -
                                 fma(f2d_bits(float(8 * ni.iy + y) + 0.5f), h, lo_y));
        offc[2] = df_from_double(com[(size_t(node) * 3 + 2) * NCELL + c] -
                                 fma(f2d_bits(float(8 * ni.iz + z) + 0.5f), h, lo_z));
    }
    if (ni.parent >= 0) {
        const int pc = (4 * (ni.ix & 1) + (x >> 1)) + 8 * (4 * (ni.iy & 1) + (y >> 1)) +
                       64 * (4 * (ni.iz & 1) + (z >> 1));
        const int prow = info[ni.parent].mp_row;
        const dfloat *pd = down + size_t(prow) * 23 * NCELL + pc;
        dfloat Pd[20];
#pragma unroll
        for (int k = 0; k < 20; ++k) Pd[k] = pd[k * NCELL];
        const dfloat hc = Ld[0];
        const dfloat d[3] = {(x & 1 ? 0.5f : -0.5f) * hc + offc[0] - pd[20 * NCELL],
                             (y & 1 ? 0.5f : -0.5f) * hc + offc[1] - pd[21 * NCELL],
                             (z & 1 ? 0.5f : -0.5f) * hc + offc[2] - pd[22 * NCELL]};
        dfloat inc[20];
        shift_increments<dfloat, NMAX>(Pd, d, inc);
#pragma unroll
        for (int k = 0; k < NK; ++k) own[k] += inc[k] * Ld[1 + (k == 0 ? 0 : k < 4 ? 1 : k < 10 ? 2 : 3)];
#pragma unroll
        for (int k = 0; k < NK; ++k)
            out[k] = fma(df_to_double(own[k]), sc[k == 0 ? 0 : k < 4 ? 1 : k < 10 ? 2 : 3],
                         L64[(size_t(ni.parent) * NCOMP + k) * NCELL + pc]);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            corr[a] = fma(dL1[(size_t(node) * 3 + a) * NCELL + c], sc[1],
                          dacc[(size_t(ni.parent) * 3 + a) * NCELL + pc]);
    } else {
#pragma unroll
        for (int k = 0; k < NK; ++k)
            out[k] = df_to_double(own[k]) * sc[k == 0 ? 0 : k < 4 ? 1 : k < 10 ? 2 : 3];
#pragma unroll
        for (int a = 0; a < 3; ++a) corr[a] = dL1[(size_t(node) * 3 + a) * NCELL + c] * sc[1];
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) L64[(size_t(node) * NCOMP + k) * NCELL + c] = out[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) dacc[(size_t(node) * 3 + a) * NCELL + c] = corr[a];
    if (NMAX == 3) {
        dfloat *od = down + size_t(ni.mp_row) * 23 * NCELL + c;
#pragma unroll
        for (int k = 0; k < 20; ++k) od[k * NCELL] = df_from_double(out[k]);
#pragma unroll
        for (int a = 0; a < 3; ++a) od[(20 + a) * NCELL] = offc[a];
    }
}

// one cell's shift in the tree's precision (MODE: FMM_FP64, FMM_MIXED or
// FMM_DFLOAT); besides being stored, the results come back in out, corr
template <int MODE, int NMAX>
__device__ __forceinline__ void l2l_cell(const NodeInfo *__restrict__ info, const NodeInfo &ni,
                                         int node, int c, const double *__restrict__ levels,
                                         const dfloat *__restrict__ levels_df,
                                         const void *__restrict__ Lv, const float *__restrict__ Lc,
                                         const double *dL1, const double *__restrict__ com,
                                         double *__restrict__ L64, double *dacc, float *down,
                                         double lo_x, double lo_y, double lo_z, double (&out)[20],
                                         double (&corr)[3])
{
    if constexpr (MODE == FMM_MIXED)
        l2l_cell_mixed<NMAX>(ni, node, c, info, levels, levels_df, static_cast<const float *>(Lv),
                             Lc, dL1, com, L64, dacc, reinterpret_cast<dfloat *>(down), lo_x, lo_y,
                             lo_z, out, corr);
    else if constexpr (MODE == FMM_DFLOAT)
        l2l_cell_df<NMAX>(ni, node, c, info, levels, levels_df, static_cast<const float *>(Lv), Lc,
                          dL1, com, L64, dacc, reinterpret_cast<dfloat *>(down), lo_x, lo_y, lo_z,
                          out, corr);
    else
        l2l_cell_fp64<NMAX>(ni, node, c, levels, Lv, dL1, com, L64, dacc, lo_x, lo_y, lo_z, out,
                            corr);
}

// 64 threads per CTA, 8 CTAs per node, so that the few nodes of a coarse
// level still spread their FP64 work over many SMs
constexpr int kSliceThreads = 64;

// MODE: FMM_FP64, FMM_MIXED or FMM_DFLOAT (FP64 shift of a float-pair input)
template <int MODE>
__global__ void __launch_bounds__(kSliceThreads) l2l_kernel(const NodeInfo *__restrict__ info,
                                                            const int32_t *__restrict__ nodes,
                                                            const double *__restrict__ levels,
                                                            const dfloat *__restrict__ levels_df,
                                                            const void *__restrict__ Lv,
                                                            const float *__restrict__ Lc,
                                                            const double *dL1,  // may alias dacc
                                                            const double *__restrict__ com,
                                                            double *__restrict__ L64, double *dacc,
                                                            float *__restrict__ down, double lo_x,
                                                            double lo_y, double lo_z)
{
    const int node = nodes[blockIdx.x >> 3];
    const NodeInfo ni = info[node];
    const int c = (blockIdx.x & 7) * kSliceThreads + threadIdx.x;
    double out[20], corr[3];
    if (ni.leaf_row >= 0)
        l2l_cell<MODE, 1>(info, ni, node, c, levels, levels_df, Lv, Lc, dL1, com, L64, dacc, down,
                          lo_x, lo_y, lo_z, out, corr);
    else
        l2l_cell<MODE, 3>(info, ni, node, c, levels, levels_df, Lv, Lc, dL1, com, L64, dacc, down,
                          lo_x, lo_y, lo_z, out, corr);
}

// 64 threads per leaf node, one (x, y) column of 8 cells each.
// The torque sum uses that x and y are fixed along a column, X2 = Z0 + z h:
//   sum m (X x g) = (X1 F2 - S1, S0 - X0 F2, X0 F1 - X1 F0),
//   F = sum m g,  S_a = sum m X2 g_a = Z0 F_a + h sum z m g_a  (a = 0, 1),
// which takes 6 FP64 operations per cell instead of 12 (GB300's FP64 unit
// bounds this pass).  The normalisers need float precision only and are
// formed and summed in float, with the double -> float conversions on the
// integer pipe.
constexpr int kForceThreads = 64;

// block sum of NV values of type V, fixed order; result in thread 0
template <int THREADS, typename V, int NV>
__device__ __forceinline__ void block_sum(V v[NV], V (*sh)[NV])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < NV; ++k) {
            V s = V(0);
            for (int w = 0; w < THREADS / 32; ++w) s += sh[w][k];
            v[k] = s;
        }
    }
}

// per-thread state of the force pass: the (x, y) column's position and sums
struct ForceColumn {
    double X0, X1, Z0, h, h3;
    float X0f, X1f, Z0f, hf;
    double F[3] = {0.0, 0.0, 0.0}, T[2] = {0.0, 0.0};
    float nf = 0.f, nt = 0.f;

    __device__ __forceinline__ ForceColumn(const NodeInfo &ni, const double *levels,
                                           double box_size)
    {
        h = levels[ni.level * LEVEL_FIELDS + LV_H];
        h3 = levels[ni.level * LEVEL_FIELDS + LV_H3];
        const double half = 0.5 * box_size;
        const int x = threadIdx.x & 7, y = threadIdx.x >> 3;
        // position from the box centre (the box corner cancels); x, y fixed per thread
        X0 = (8.0 * ni.ix + x + 0.5) * h - half;
        X1 = (8.0 * ni.iy + y + 0.5) * h - half;
        Z0 = (8.0 * ni.iz + 0.5) * h - half;
        X0f = d2f_trunc(X0);
        X1f = d2f_trunc(X1);
        Z0f = d2f_trunc(Z0);
        hf = d2f_trunc(h);
    }

    // cell z of the column, of mass m: phi = L0, g = -(L1 + dL1), and its
    // terms of the sums
    __device__ __forceinline__ void cell(int row, int c, int z, double m, double L0,
                                         const double L1[3], const double acc[3],
                                         double *__restrict__ phi, double *__restrict__ g)
    {
        phi[size_t(row) * NCELL + c] = L0;
        double gv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gv[a] = -(L1[a] + acc[a]);
            g[(size_t(row) * 3 + a) * NCELL + c] = gv[a];
            F[a] = fma(m, gv[a], F[a]);                 // f = m g
        }
        if (z > 0) {
            const double mz = z == 1 ? m : m * double(z);
            T[0] = fma(mz, gv[0], T[0]);
            T[1] = fma(mz, gv[1], T[1]);
        }
        // normalisers |f| = m |g| and |x cross f| = m |x cross g|, in float
        // (g and x are O(1), so float does not underflow where m is tiny)
        const float mf = d2f_trunc(m);
        const float gf[3] = {d2f_trunc(gv[0]), d2f_trunc(gv[1]), d2f_trunc(gv[2])};
        const float X2f = fmaf(float(z), hf, Z0f);
        // (explicit fused forms: the fused leaf pass must round exactly as
        // the force pass does)
        const float uf[3] = {fmaf(X1f, gf[2], -(X2f * gf[1])), fmaf(X2f, gf[0], -(X0f * gf[2])),
                             fmaf(X0f, gf[1], -(X1f * gf[0]))};
        nf = fmaf(mf, sqrtf(fmaf(gf[0], gf[0], fmaf(gf[1], gf[1], gf[2] * gf[2]))), nf);
        nt = fmaf(mf, sqrtf(fmaf(uf[0], uf[0], fmaf(uf[1], uf[1], uf[2] * uf[2]))), nt);
    }

    // the node's fixed-order block sums into its partials row
    // The node's six FP64 sums over its 64 columns, in a fixed order: eight
    // threads per value add eight columns each, then six threads add the
    // eight partial sums.  That is 63 adds per value, where a shuffle tree
    // has every lane of both warps add at each of its five levels (five
    // times the FP64 operations, on the pipe that bounds this pass).
    __device__ __forceinline__ void finish(int row, double *__restrict__ partials)
    {
        __shared__ double sh[6][kForceThreads];
        __shared__ double sh8[6][8];
        __shared__ float shf[kForceThreads / 32][2];
        const double S0 = fma(h, T[0], Z0 * F[0]), S1 = fma(h, T[1], Z0 * F[1]);
        const double v[6] = {F[0], F[1], F[2], fma(X1, F[2], -S1), fma(-X0, F[2], S0),
                             fma(X0, F[1], -X1 * F[0])};
#pragma unroll
        for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = v[k];
        float vf[2] = {nf, nt};
        block_sum<kForceThreads, float, 2>(vf, shf);     // (its barrier publishes sh)
        if (threadIdx.x < 48) {
            const int k = threadIdx.x % 6, q = threadIdx.x / 6;
            double t = sh[k][8 * q];
#pragma unroll
            for (int i = 1; i < 8; ++i) t += sh[k][8 * q + i];
            sh8[k][q] = t;
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            double t = sh8[threadIdx.x][0];
#pragma unroll
            for (int q = 1; q < 8; ++q) t += sh8[threadIdx.x][q];
            partials[size_t(row) * 8 + threadIdx.x] = t;
        }
        if (threadIdx.x == 0) {
            partials[size_t(row) * 8 + 6] = double(vf[0]);
            partials[size_t(row) * 8 + 7] = double(vf[1]);
        }
    }
};

__global__ void __launch_bounds__(kForceThreads) forces_kernel(
    const NodeInfo *__restrict__ info, const int32_t *__restrict__ leaves,
    const double *__restrict__ levels, const double *__restrict__ L64,
    const double *__restrict__ dacc, const double *__restrict__ rho, double *__restrict__ phi,
    double *__restrict__ g, double *__restrict__ partials, double box_size)
{
    const int node = leaves[blockIdx.x];
    const NodeInfo ni = info[node];
    const int row = ni.leaf_row;
    ForceColumn col(ni, levels, box_size);
#pragma unroll
    for (int z = 0; z < 8; ++z) {
        const int c = threadIdx.x + 64 * z;
        double L1[3], acc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            L1[a] = L64[(size_t(node) * NCOMP + 1 + a) * NCELL + c];
            acc[a] = dacc[(size_t(node) * 3 + a) * NCELL + c];
        }
        col.cell(row, c, z, rho[size_t(row) * NCELL + c] * col.h3, L64[(size_t(node) * NCOMP) * NCELL + c],
                 L1, acc, phi, g);
    }
    col.finish(row, partials);
}

// fmm_step's last pass over the leaves: each leaf cell's shift (as
// l2l_kernel) and its forces (as forces_kernel) in one kernel, the shifted
// expansion going straight from registers into the force terms; the same
// arithmetic, in the same order, as the two kernels.  At most 80 registers
// (12 CTAs per SM, 24 warps, no spills): the pass is bound by the FP64 pipe,
// and the extra warps keep more FP64 operations in flight than the 96
// registers it would otherwise take
template <int MODE>
__global__ void __launch_bounds__(kForceThreads, 12) leaf_finish_kernel(
    const NodeInfo *__restrict__ info, const int32_t *__restrict__ leaves,
    const double *__restrict__ levels, const dfloat *__restrict__ levels_df,
    const void *__restrict__ Lv, const float *__restrict__ Lc, const double *dL1,
    const double *__restrict__ com, double *__restrict__ L64, double *dacc, float *down,
    const double *__restrict__ M, double *__restrict__ phi, double *__restrict__ g,
    double *__restrict__ partials, double lo_x, double lo_y, double lo_z, double box_size)
{
    const int node = leaves[blockIdx.x];
    const NodeInfo ni = info[node];
    const int row = ni.leaf_row;
    ForceColumn col(ni, levels, box_size);
#pragma unroll
    for (int z = 0; z < 8; ++z) {
        const int c = threadIdx.x + 64 * z;
        double out[20], corr[3];
        l2l_cell<MODE, 1>(info, ni, node, c, levels, levels_df, Lv, Lc, dL1, com, L64, dacc, down,
                          lo_x, lo_y, lo_z, out, corr);
        // the cell mass as P2M left it in M (rho h^3, the same product): the
        // step reads the density in P2M only, so it may sit in pinned host
        // memory
        col.cell(row, c, z, M[(size_t(node) * NCOMP) * NCELL + c], out[0], out + 1, corr, phi, g);
    }
    col.finish(row, partials);
}

// ---------------------------------------------------------------- dataflow
// The downward pass as one persistent launch (the device-side counterpart of
// the paper's futurized tree traversal, Sec. 4.1 and Sec. 5.1): CTAs pull
// items from one queue -- every refined node's eight 64-cell slices, root
// level first, then every leaf node, coarse levels first -- and an item
// starts as soon as its parent's eight slices are done (a readiness counter
// per node), rather than when the whole previous level's launch has ended.
// Every item's producer sits earlier in the queue, and a CTA only waits
// after it has dequeued its item, so the items it waits on were dequeued by
// CTAs that are already running: progress does not depend on how many CTAs
// are resident.  Each wait is bounded: past its budget it sets
// FMM_STATUS_TIMEOUT and an abort flag that ends every later wait at once,
// and the kernel returns (the step's outputs are then undefined).  The
// arithmetic per cell is that of l2l_kernel and leaf_finish_kernel, so the
// results are the same bits.
struct DflowParams {
    const NodeInfo *info;
    const int32_t *items;
    int32_t n_items, n_refined_items;
    int32_t *head, *ready, *abort_flag, *status;
    long long budget_ns;
    const double *levels;
    const dfloat *levels_df;
    const void *L;
    const float *Lc;
    const double *dL1;
    const double *com;
    double *L64, *dacc;
    float *down;
    const double *M;
    double *phi, *g, *partials;
    double lo_x, lo_y, lo_z, box_size;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// thread 0: wait until the node's eight slices are done; 0 if the wait gave
// up (its budget ran out here, or another wait's did)
__device__ int wait_node(const DflowParams &P, int node)
{
    if (ld_acquire(P.ready + node) >= 8) return 1;
    const unsigned long long t0 = global_ns();
    // the iteration cap bounds the wait even if the timer did not advance
    for (int it = 0; it < (1 << 26); ++it) {
        __nanosleep(128);
        if (ld_acquire(P.ready + node) >= 8) return 1;
        if (ld_acquire(P.abort_flag)) return 0;
        if ((long long)(global_ns() - t0) > P.budget_ns) break;
    }
    atomicOr(P.status, FMM_STATUS_TIMEOUT);
    atomicExch(P.abort_flag, 1);
    return 0;
}

template <int MODE>
__global__ void __launch_bounds__(kForceThreads, 12) dataflow_kernel(DflowParams P)
{
    __shared__ int s_pos, s_go;
    for (;;) {
        __syncthreads();                 // the previous item's shared state is done with
        if (threadIdx.x == 0) s_pos = atomicAdd(P.head, 1);
        __syncthreads();
        const int pos = s_pos;
        if (pos >= P.n_items) break;
        const bool refined = pos < P.n_refined_items;
        const int it = P.items[pos];
        const int node = refined ? it >> 3 : it;
        const NodeInfo ni = P.info[node];
        if (threadIdx.x == 0) s_go = ni.parent < 0 ? 1 : wait_node(P, ni.parent);
        __syncthreads();
        if (!s_go) continue;
        if (refined) {
            const int c = (it & 7) * kForceThreads + threadIdx.x;
            double out[20], corr[3];
            l2l_cell<MODE, 3>(P.info, ni, node, c, P.levels, P.levels_df, P.L, P.Lc, P.dL1, P.com,
                              P.L64, P.dacc, P.down, P.lo_x, P.lo_y, P.lo_z, out, corr);
            // publish: every thread's stores, then the counter
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(P.ready + node, 1);
        } else {
            const int row = ni.leaf_row;
            ForceColumn col(ni, P.levels, P.box_size);
#pragma unroll
            for (int z = 0; z < 8; ++z) {
                const int c = threadIdx.x + 64 * z;
                double out[20], corr[3];
                l2l_cell<MODE, 1>(P.info, ni, node, c, P.levels, P.levels_df, P.L, P.Lc, P.dL1,
                                  P.com, P.L64, P.dacc, P.down, P.lo_x, P.lo_y, P.lo_z, out, corr);
                col.cell(row, c, z, P.M[(size_t(node) * NCOMP) * NCELL + c], out[0], out + 1, corr,
                         P.phi, P.g);
            }
            col.finish(row, P.partials);
        }
    }
}

// Per-tree sums of the per-leaf-node partials in two fixed-order stages, so
// the FP64 adds spread over many SMs: chunks of kReduceRows leaf rows per CTA,
// then one warp per tree over its chunks.
__global__ void __launch_bounds__(512) reduce_chunk_kernel(const int32_t *__restrict__ off,
                                                           const int32_t *__restrict__ rows,
                                                           const double *__restrict__ partials,
                                                           double *__restrict__ chunk_sums)
{
    __shared__ double sh[16][8];
    const int tree = blockIdx.x, chunk = blockIdx.y;
    const int lo = off[tree] + chunk * kReduceRows;
    const int hi = min(lo + kReduceRows, off[tree + 1]);
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] += partials[size_t(rows[i]) * 8 + k];
    block_sum<512, double, 8>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) chunk_sums[(size_t(tree) * gridDim.y + chunk) * 8 + k] = v[k];
}

__global__ void __launch_bounds__(32) reduce_final_kernel(const double *__restrict__ chunk_sums,
                                                          int chunks, double *__restrict__ totals)
{
    const int tree = blockIdx.x, k = threadIdx.x;
    if (k >= 8) return;
    double v = 0.0;
    for (int c = 0; c < chunks; ++c) v += chunk_sums[(size_t(tree) * chunks + c) * 8 + k];
    totals[size_t(tree) * 8 + k] = v;
}

}  // namespace

cudaError_t launch_l2l_level(const fmm_tree_s *t, int level, const void *L, const float *Lc,
                             const double *dL1, const double *com, double *L64, double *dacc,
                             cudaStream_t s)
{
    return launch_l2l_nodes(t, t->plan.nodes_at[size_t(level)], L, Lc, dL1, com, L64, dacc, s);
}

// any list of nodes whose parents are done (one level, the refined nodes of
// one level, or every leaf once every refined node is done)
cudaError_t launch_l2l_nodes(const fmm_tree_s *t, const ListRange &r, const void *L,
                             const float *Lc, const double *dL1, const double *com, double *L64,
                             double *dacc, cudaStream_t s)
{
    if (r.count == 0) return cudaSuccess;
    const auto &c = t->cfg;
    const unsigned grid = unsigned(r.count * 8);
    const int32_t *nodes = t->dev.lists + r.off;
    const dfloat *ldf = reinterpret_cast<const dfloat *>(t->dev.levels_df);
    if (c.precision == FMM_MIXED)
        l2l_kernel<FMM_MIXED><<<grid, kSliceThreads, 0, s>>>(t->dev.info, nodes, t->dev.levels, ldf, L,
                                                            Lc, dL1, com, L64, dacc, t->dev.down,
                                                            c.box_lo[0], c.box_lo[1], c.box_lo[2]);
    else if (c.precision == FMM_DFLOAT)
        l2l_kernel<FMM_DFLOAT><<<grid, kSliceThreads, 0, s>>>(t->dev.info, nodes, t->dev.levels, ldf, L,
                                                             Lc, dL1, com, L64, dacc, t->dev.down,
                                                             c.box_lo[0], c.box_lo[1], c.box_lo[2]);
    else
        l2l_kernel<FMM_FP64><<<grid, kSliceThreads, 0, s>>>(t->dev.info, nodes, t->dev.levels, ldf, L,
                                                           Lc, dL1, com, L64, dacc, nullptr,
                                                           c.box_lo[0], c.box_lo[1], c.box_lo[2]);
    return cudaGetLastError();
}

cudaError_t launch_leaf_finish(const fmm_tree_s *t, const void *L, const float *Lc,
                               const double *dL1, const double *com, double *L64, double *dacc,
                               const double *M, double *phi, double *g, cudaStream_t s)
{
    const ListRange &r = t->plan.leaves;
    if (r.count == 0) return cudaSuccess;
    const auto &c = t->cfg;
    const dfloat *ldf = reinterpret_cast<const dfloat *>(t->dev.levels_df);
    const int32_t *nodes = t->dev.lists + r.off;
    const unsigned grid = unsigned(r.count);
    if (c.precision == FMM_MIXED)
        leaf_finish_kernel<FMM_MIXED><<<grid, kForceThreads, 0, s>>>(
            t->dev.info, nodes, t->dev.levels, ldf, L, Lc, dL1, com, L64, dacc, t->dev.down, M,
            phi, g, t->dev.partials, c.box_lo[0], c.box_lo[1], c.box_lo[2], c.box_size);
    else if (c.precision == FMM_DFLOAT)
        leaf_finish_kernel<FMM_DFLOAT><<<grid, kForceThreads, 0, s>>>(
            t->dev.info, nodes, t->dev.levels, ldf, L, Lc, dL1, com, L64, dacc, t->dev.down, M,
            phi, g, t->dev.partials, c.box_lo[0], c.box_lo[1], c.box_lo[2], c.box_size);
    else
        leaf_finish_kernel<FMM_FP64><<<grid, kForceThreads, 0, s>>>(
            t->dev.info, nodes, t->dev.levels, ldf, L, Lc, dL1, com, L64, dacc, nullptr, M, phi,
            g, t->dev.partials, c.box_lo[0], c.box_lo[1], c.box_lo[2], c.box_size);
    return cudaGetLastError();
}

cudaError_t launch_downward_dataflow(const fmm_tree_s *t, const void *L, const float *Lc,
                                     const double *dL1, const double *com, double *L64,
                                     double *dacc, const double *M, double *phi, double *g,
                                     cudaStream_t s)
{
    const Plan &Pl = t->plan;
    if (Pl.dflow_items == 0) return cudaSuccess;
    const auto &c = t->cfg;
    DflowParams P{};
    P.info = t->dev.info;
    // the test injection leaves the first refined node's eight items out
    const int drop = (t->tuning.drop_first_producer && Pl.dflow_refined_items >= 8) ? 8 : 0;
    P.items = t->dev.dflow_items + drop;
    P.n_items = int32_t(Pl.dflow_items - drop);
    P.n_refined_items = int32_t(Pl.dflow_refined_items - drop);
    P.head = t->dev.counters + kDflowHeadSlot;
    P.abort_flag = t->dev.counters + kDflowAbortSlot;
    P.status = t->dev.counters + kStatusSlot;
    P.ready = t->dev.dflow_ready;
    P.budget_ns = t->tuning.wait_budget_us > 0 ? 1000ll * t->tuning.wait_budget_us
                                               : kDefaultWaitBudgetNs;
    P.levels = t->dev.levels;
    P.levels_df = reinterpret_cast<const dfloat *>(t->dev.levels_df);
    P.L = L;
    P.Lc = Lc;
    P.dL1 = dL1;
    P.com = com;
    P.L64 = L64;
    P.dacc = dacc;
    P.down = t->dev.down;
    P.M = M;
    P.phi = phi;
    P.g = g;
    P.partials = t->dev.partials;
    P.lo_x = c.box_lo[0];
    P.lo_y = c.box_lo[1];
    P.lo_z = c.box_lo[2];
    P.box_size = c.box_size;
    cudaError_t e = cudaMemsetAsync(t->dev.dflow_ready, 0, size_t(t->n) * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.head, 0, 2 * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    auto launch = [&](auto kern) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kForceThreads, 0) !=
                cudaSuccess || per_sm < 1)
            per_sm = 1;
        const int64_t cap = int64_t(per_sm) * sm_count_of_current_device();
        const unsigned grid = unsigned(P.n_items < cap ? P.n_items : cap);
        kern<<<grid, kForceThreads, 0, s>>>(P);
        return cudaGetLastError();
    };
    if (c.precision == FMM_MIXED) return launch(dataflow_kernel<FMM_MIXED>);
    if (c.precision == FMM_DFLOAT) return launch(dataflow_kernel<FMM_DFLOAT>);
    return launch(dataflow_kernel<FMM_FP64>);
}

cudaError_t launch_forces(const fmm_tree_s *t, const double *L64, const double *dacc,
                          const double *rho, double *phi, double *g, double *totals,
                          cudaStream_t s)
{
    const ListRange &r = t->plan.leaves;
    if (r.count > 0) {
        timing_begin(t, FMM_K_FORCES, s);
        forces_kernel<<<unsigned(r.count), kForceThreads, 0, s>>>(
            t->dev.info, t->dev.lists + r.off, t->dev.levels, L64, dacc, rho, phi, g,
            t->dev.partials, t->cfg.box_size);
        timing_end(t, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_force_sums(t, totals, s);
}

cudaError_t launch_force_sums(const fmm_tree_s *t, double *totals, cudaStream_t s)
{
    timing_begin(t, FMM_K_REDUCE, s);
    const int chunks = t->plan.reduce_chunks;
    reduce_chunk_kernel<<<dim3(unsigned(t->n_trees), unsigned(chunks)), 512, 0, s>>>(
        t->dev.tree_leaf_off, t->dev.tree_leaf_rows, t->dev.partials, t->dev.chunk_sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_final_kernel<<<unsigned(t->n_trees), 32, 0, s>>>(t->dev.chunk_sums, chunks, totals);
    timing_end(t, s);
    return cudaGetLastError();
}

}  // namespace fmm
