// Upward pass (Sec. 4.3, first step): cell masses from the leaf densities,
// then, level by level from the deepest, each refined cell's mass, centre of
// mass and central moments from its eight child cells.  FP64 throughout.
// HBM-bound: every child value is read once and every parent value written
// once.
#include "fmm_internal.h"
#include "fmm_tensor.cuh"

namespace fmm {

namespace {

__device__ __forceinline__ double cell_width(double box_size, int level)
{
    return box_size / (8.0 * double(1u << (level - 1)));
}

// P2M: leaf cells hold m = rho h^3 at their centre (point-mass reading of a
// locally homogeneous density).  One thread per cell, cells x-fastest.
__global__ void __launch_bounds__(512) p2m_kernel(const NodeInfo *__restrict__ info,
                                                  const int32_t *__restrict__ leaves,
                                                  const double *__restrict__ rho,
                                                  double *__restrict__ M, double box_size)
{
    const int node = leaves[blockIdx.x];
    const NodeInfo ni = info[node];
    const double h = cell_width(box_size, ni.level);
    const double h3 = h * h * h;
    const int c = threadIdx.x;
    M[(size_t(node) * NCOMP) * NCELL + c] = rho[size_t(ni.leaf_row) * NCELL + c] * h3;
}

// M2M: parent cell (x,y,z) of a refined node takes the 2x2x2 child cells of
// child node (x>>2, y>>2, z>>2) at child-local (2(x&3)+dx, ...):
//   M0 = sum m_c,  X = sum m_c X_c / M0,  s_c = X_c - X,
//   M2_ij  = sum (M2c_ij + m_c s_i s_j),
//   M3_ijk = sum (M3c_ijk + M2c_ij s_k + M2c_ik s_j + M2c_jk s_i + m_c s_i s_j s_k).
// Leaf child cells are point masses at their centre (no M2, M3 reads).
__global__ void __launch_bounds__(512) m2m_kernel(const NodeInfo *__restrict__ info,
                                                  const int32_t *__restrict__ children,
                                                  const int32_t *__restrict__ nodes,
                                                  double *__restrict__ M, double *__restrict__ com,
                                                  double lo_x, double lo_y, double lo_z,
                                                  double box_size)
{
    const int node = nodes[blockIdx.x];
    const NodeInfo ni = info[node];
    const int c = threadIdx.x;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const int k = (x >> 2) + 2 * (y >> 2) + 4 * (z >> 2);
    const int ch = children[node * 8 + k];
    const NodeInfo ci = info[ch];
    const bool child_leaf = ci.leaf_row >= 0;
    const double hc = cell_width(box_size, ni.level + 1);
    const double hp = 2.0 * hc;
    // reference point: the parent cell centre (keeps the sums well scaled)
    const double ref[3] = {lo_x + (8.0 * ni.ix + x + 0.5) * hp, lo_y + (8.0 * ni.iy + y + 0.5) * hp,
                           lo_z + (8.0 * ni.iz + z + 0.5) * hp};
    double m[8], X[8][3];
    double m0 = 0.0, mx[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int cx = 2 * (x & 3) + (j & 1), cy = 2 * (y & 3) + ((j >> 1) & 1),
                  cz = 2 * (z & 3) + (j >> 2);
        const int cc = cx + 8 * cy + 64 * cz;
        m[j] = M[(size_t(ch) * NCOMP) * NCELL + cc];
        if (child_leaf) {
            X[j][0] = lo_x + (8.0 * ci.ix + cx + 0.5) * hc;
            X[j][1] = lo_y + (8.0 * ci.iy + cy + 0.5) * hc;
            X[j][2] = lo_z + (8.0 * ci.iz + cz + 0.5) * hc;
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) X[j][a] = com[(size_t(ch) * 3 + a) * NCELL + cc];
        }
        m0 += m[j];
#pragma unroll
        for (int a = 0; a < 3; ++a) mx[a] += m[j] * (X[j][a] - ref[a]);
    }
    double Xp[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Xp[a] = ref[a] + mx[a] / m0;
    double M2[6] = {0, 0, 0, 0, 0, 0};
    double M3[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    constexpr int I2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    constexpr int I3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                               {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int cx = 2 * (x & 3) + (j & 1), cy = 2 * (y & 3) + ((j >> 1) & 1),
                  cz = 2 * (z & 3) + (j >> 2);
        const int cc = cx + 8 * cy + 64 * cz;
        const double s[3] = {X[j][0] - Xp[0], X[j][1] - Xp[1], X[j][2] - Xp[2]};
        double c2[6] = {0, 0, 0, 0, 0, 0};
        if (!child_leaf) {
#pragma unroll
            for (int q = 0; q < 6; ++q) c2[q] = M[(size_t(ch) * NCOMP + 4 + q) * NCELL + cc];
#pragma unroll
            for (int q = 0; q < 10; ++q) M3[q] += M[(size_t(ch) * NCOMP + 10 + q) * NCELL + cc];
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) M2[q] += c2[q] + m[j] * s[I2[q][0]] * s[I2[q][1]];
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            const int a = I3[q][0], b = I3[q][1], d = I3[q][2];
            M3[q] += c2[r2_of(a, b)] * s[d] + c2[r2_of(a, d)] * s[b] + c2[r2_of(b, d)] * s[a] +
                     m[j] * s[a] * s[b] * s[d];
        }
    }
    double *out = M + size_t(node) * NCOMP * NCELL + c;
    out[0] = m0;
    out[1 * NCELL] = 0.0;
    out[2 * NCELL] = 0.0;
    out[3 * NCELL] = 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) out[(4 + q) * NCELL] = M2[q];
#pragma unroll
    for (int q = 0; q < 10; ++q) out[(10 + q) * NCELL] = M3[q];
#pragma unroll
    for (int a = 0; a < 3; ++a) com[(size_t(node) * 3 + a) * NCELL + c] = Xp[a];
}

}  // namespace

cudaError_t launch_p2m(const fmm_tree_s *t, const double *rho, double *M, cudaStream_t s)
{
    const ListRange &r = t->plan.leaves;
    if (r.count == 0) return cudaSuccess;
    p2m_kernel<<<unsigned(r.count), 512, 0, s>>>(t->dev.info, t->dev.lists + r.off, rho, M,
                                                 t->cfg.box_size);
    return cudaGetLastError();
}

cudaError_t launch_m2m_level(const fmm_tree_s *t, int level, double *M, double *com,
                             cudaStream_t s)
{
    const ListRange &r = t->plan.refined_at[size_t(level)];
    if (r.count == 0) return cudaSuccess;
    m2m_kernel<<<unsigned(r.count), 512, 0, s>>>(t->dev.info, t->dev.children, t->dev.lists + r.off,
                                                 M, com, t->cfg.box_lo[0], t->cfg.box_lo[1],
                                                 t->cfg.box_lo[2], t->cfg.box_size);
    return cudaGetLastError();
}

}  // namespace fmm
