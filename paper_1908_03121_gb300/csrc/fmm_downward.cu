// Downward pass (Sec. 4.3, third step) and leaf forces, in FP64.
//
// l2l_kernel, one launch per level from the root down: each cell converts its
// own same-level result from level units (float hi + lo, or double) to
// physical units, adds its parent's final expansion re-centred at its own
// centre of mass,
//   L^(n) += sum_{k=0}^{3-n} (1/k!) L_parent^(n+k) . d^k,  d = X - X_parent,
// and inherits the parent's accumulated angular-momentum correction.
// forces_kernel: phi = L0, g = -(L1 + dL1), f = m g, and fixed-order FP64
// block sums of f, x cross f, |f|, |x cross f| per leaf node; reduce_kernel
// folds those per tree.  All HBM-bound streams.
#include "fmm_internal.h"
#include "fmm_tensor.cuh"

namespace fmm {

namespace {

__device__ __forceinline__ double cell_width(double box_size, int level)
{
    return box_size / (8.0 * double(1u << (level - 1)));
}

template <bool MIXED>
__global__ void __launch_bounds__(512) l2l_kernel(const NodeInfo *__restrict__ info,
                                                  const int32_t *__restrict__ nodes,
                                                  const void *__restrict__ Lv,
                                                  const float *__restrict__ Lc,
                                                  const double *dL1,  // may alias dacc
                                                  const double *__restrict__ com,
                                                  double *__restrict__ L64, double *dacc,
                                                  double G, double lo_x, double lo_y,
                                                  double lo_z, double box_size)
{
    const int node = nodes[blockIdx.x];
    const NodeInfo ni = info[node];
    const bool leaf = ni.leaf_row >= 0;
    const int nk = leaf ? 4 : 20;
    const int c = threadIdx.x;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const double h = cell_width(box_size, ni.level);
    const double ih = 1.0 / h;
    // level units -> physical: G h^-(n+1)
    const double s0 = G * ih, s1 = s0 * ih, s2 = s1 * ih, s3 = s2 * ih;
    double L[20];
#pragma unroll
    for (int k = 0; k < 20; ++k) {
        if (k >= nk) { L[k] = 0.0; continue; }
        const size_t idx = (size_t(node) * NCOMP + k) * NCELL + c;
        double v;
        if (MIXED) v = double(static_cast<const float *>(Lv)[idx]) + double(Lc[idx]);
        else v = static_cast<const double *>(Lv)[idx];
        L[k] = v * (k == 0 ? s0 : k < 4 ? s1 : k < 10 ? s2 : s3);
    }
    double corr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) corr[a] = dL1[(size_t(node) * 3 + a) * NCELL + c] * s1;
    if (ni.parent >= 0) {
        const NodeInfo pi = info[ni.parent];
        const int qx = 4 * (ni.ix & 1) + (x >> 1), qy = 4 * (ni.iy & 1) + (y >> 1),
                  qz = 4 * (ni.iz & 1) + (z >> 1);
        const int pc = qx + 8 * qy + 64 * qz;
        double X[3];
        if (leaf) {
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
        (void)pi;
        // powers of d on symmetric components
        const double dd[6] = {d[0] * d[0], d[0] * d[1], d[0] * d[2], d[1] * d[1], d[1] * d[2],
                              d[2] * d[2]};
        constexpr int I3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                                   {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
        // order 0: P0 + P1.d + 1/2 P2:dd + 1/6 P3:ddd
        double v0 = P[0];
#pragma unroll
        for (int i = 0; i < 3; ++i) v0 += P[1 + i] * d[i];
#pragma unroll
        for (int q = 0; q < 6; ++q) v0 += 0.5 * mult2(q) * P[4 + q] * dd[q];
#pragma unroll
        for (int q = 0; q < 10; ++q)
            v0 += (1.0 / 6.0) * mult3(q) * P[10 + q] * d[I3[q][0]] * d[I3[q][1]] * d[I3[q][2]];
        L[0] += v0;
        // order 1: P1_i + P2_ij d_j + 1/2 P3_ijk d_j d_k
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double v = P[1 + i];
#pragma unroll
            for (int j = 0; j < 3; ++j) v += P[4 + r2_of(i, j)] * d[j];
#pragma unroll
            for (int q = 0; q < 6; ++q) v += 0.5 * mult2(q) * P[10 + r3_of(i, q)] * dd[q];
            L[1 + i] += v;
        }
        if (!leaf) {
            // order 2: P2_ij + P3_ijk d_k ; order 3: P3
            constexpr int I2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                double v = P[4 + q];
#pragma unroll
                for (int k = 0; k < 3; ++k) v += P[10 + r3_ijk(I2[q][0], I2[q][1], k)] * d[k];
                L[4 + q] += v;
            }
#pragma unroll
            for (int q = 0; q < 10; ++q) L[10 + q] += P[10 + q];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) corr[a] += dacc[(size_t(ni.parent) * 3 + a) * NCELL + pc];
    }
#pragma unroll
    for (int k = 0; k < 20; ++k)
        if (k < nk) L64[(size_t(node) * NCOMP + k) * NCELL + c] = L[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) dacc[(size_t(node) * 3 + a) * NCELL + c] = corr[a];
}

// block sum of 8 doubles over 512 threads, fixed order; result in thread 0
__device__ __forceinline__ void block_sum8(double v[8], double (*sh)[8])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 8; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < 8; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[w][k];
            v[k] = s;
        }
    }
}

__global__ void __launch_bounds__(512) forces_kernel(const NodeInfo *__restrict__ info,
                                                     const int32_t *__restrict__ leaves,
                                                     const double *__restrict__ L64,
                                                     const double *__restrict__ dacc,
                                                     const double *__restrict__ rho,
                                                     double *__restrict__ phi,
                                                     double *__restrict__ g,
                                                     double *__restrict__ partials, double lo_x,
                                                     double lo_y, double lo_z, double box_size)
{
    __shared__ double sh[16][8];
    const int node = leaves[blockIdx.x];
    const NodeInfo ni = info[node];
    const int row = ni.leaf_row;
    const int c = threadIdx.x;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const double h = cell_width(box_size, ni.level);
    const double m = rho[size_t(row) * NCELL + c] * h * h * h;
    phi[size_t(row) * NCELL + c] = L64[(size_t(node) * NCOMP) * NCELL + c];
    double f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double gv = -(L64[(size_t(node) * NCOMP + 1 + a) * NCELL + c] +
                            dacc[(size_t(node) * 3 + a) * NCELL + c]);
        g[(size_t(row) * 3 + a) * NCELL + c] = gv;
        f[a] = m * gv;
    }
    const double half = 0.5 * box_size;
    const double X[3] = {lo_x + (8.0 * ni.ix + x + 0.5) * h - (lo_x + half),
                         lo_y + (8.0 * ni.iy + y + 0.5) * h - (lo_y + half),
                         lo_z + (8.0 * ni.iz + z + 0.5) * h - (lo_z + half)};
    const double t[3] = {X[1] * f[2] - X[2] * f[1], X[2] * f[0] - X[0] * f[2],
                         X[0] * f[1] - X[1] * f[0]};
    double v[8] = {f[0], f[1], f[2], t[0], t[1], t[2],
                   sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]),
                   sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2])};
    block_sum8(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) partials[size_t(row) * 8 + k] = v[k];
}

__global__ void __launch_bounds__(512) reduce_kernel(const int32_t *__restrict__ off,
                                                     const int32_t *__restrict__ rows,
                                                     const double *__restrict__ partials,
                                                     double *__restrict__ totals)
{
    __shared__ double sh[16][8];
    const int tree = blockIdx.x;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = off[tree] + threadIdx.x; i < off[tree + 1]; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] += partials[size_t(rows[i]) * 8 + k];
    block_sum8(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) totals[size_t(tree) * 8 + k] = v[k];
}

}  // namespace

cudaError_t launch_l2l_level(const fmm_tree_s *t, int level, const void *L, const float *Lc,
                             const double *dL1, const double *com, double *L64, double *dacc,
                             cudaStream_t s)
{
    const ListRange &r = t->plan.nodes_at[size_t(level)];
    if (r.count == 0) return cudaSuccess;
    const auto &c = t->cfg;
    if (c.precision == FMM_MIXED)
        l2l_kernel<true><<<unsigned(r.count), 512, 0, s>>>(t->dev.info, t->dev.lists + r.off, L, Lc,
                                                           dL1, com, L64, dacc, c.G, c.box_lo[0],
                                                           c.box_lo[1], c.box_lo[2], c.box_size);
    else
        l2l_kernel<false><<<unsigned(r.count), 512, 0, s>>>(t->dev.info, t->dev.lists + r.off, L, Lc,
                                                            dL1, com, L64, dacc, c.G, c.box_lo[0],
                                                            c.box_lo[1], c.box_lo[2], c.box_size);
    return cudaGetLastError();
}

cudaError_t launch_forces(const fmm_tree_s *t, const double *L64, const double *dacc,
                          const double *rho, double *phi, double *g, double *totals,
                          cudaStream_t s)
{
    const ListRange &r = t->plan.leaves;
    const auto &c = t->cfg;
    if (r.count > 0) {
        timing_begin(t, FMM_K_FORCES, s);
        forces_kernel<<<unsigned(r.count), 512, 0, s>>>(t->dev.info, t->dev.lists + r.off, L64, dacc,
                                                        rho, phi, g, t->dev.partials, c.box_lo[0],
                                                        c.box_lo[1], c.box_lo[2], c.box_size);
        timing_end(t, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    timing_begin(t, FMM_K_REDUCE, s);
    reduce_kernel<<<unsigned(t->n_trees), 512, 0, s>>>(t->dev.tree_leaf_off, t->dev.tree_leaf_rows,
                                                       t->dev.partials, totals);
    timing_end(t, s);
    return cudaGetLastError();
}

}  // namespace fmm
