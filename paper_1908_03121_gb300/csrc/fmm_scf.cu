// Self-consistent-field (SCF) initial models: the second caller of the
// gravity solve.  The paper builds its V1309 initial model with Octo-Tiger's
// SCF module, which iterates the FMM solve (Sec. 3, Sec. 4.2; the method is
// Hachisu's 1986 self-consistent field for rotating stars and binaries).
//
// fmm_scf_update performs one iteration's density update after a solve of
// the same tree, for polytropes P = K rho^(1 + 1/n) in synchronous rotation
// about the z axis through the centre of mass:
//   H = C_i - Phi + Omega^2 w^2 / 2   (the enthalpy (n + 1) K_i rho^(1/n)
//                                     inside star i, w the axis distance),
//   Omega^2, C_1, C_2 from H = 0 at surface points A, B (star 1) and C
//   (star 2),  rho' = max(rho_floor, rho_max,i (H / H_max,i)^n) where H > 0.
// The per-cell work (centre of mass, H and its per-star maximum, the new
// density) runs in three kernels over the leaf nodes; the host reads back
// per-node partial sums and the potential at the three surface cells, and
// forms the few scalars of the iteration in FP64.
#include <cmath>
#include <string>
#include <vector>

#include "fmm_internal.h"

namespace fmm {
namespace {

constexpr int kScfThreads = 256;       // 2 cells per thread

struct ScfGeo {
    double lo[3];
    double size;
};

__device__ __forceinline__ void cell_centre(const NodeInfo &ni, const double *levels, const ScfGeo &g,
                                            int c, double x[3])
{
    const double h = levels[ni.level * LEVEL_FIELDS + LV_H];
    x[0] = g.lo[0] + (8.0 * ni.ix + (c & 7) + 0.5) * h;
    x[1] = g.lo[1] + (8.0 * ni.iy + ((c >> 3) & 7) + 0.5) * h;
    x[2] = g.lo[2] + (8.0 * ni.iz + (c >> 6) + 0.5) * h;
}

// fixed-order block sum / max of NV values over kScfThreads threads; result
// in thread 0
template <int NV, bool MAX>
__device__ __forceinline__ void block_reduce(double v[NV])
{
    __shared__ double sh[kScfThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_down_sync(0xffffffffu, v[k], off);
            v[k] = MAX ? fmax(v[k], o) : v[k] + o;
        }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < NV; ++k) {
            double s = sh[0][k];
            for (int w = 1; w < kScfThreads / 32; ++w) s = MAX ? fmax(s, sh[w][k]) : s + sh[w][k];
            v[k] = s;
        }
}

// per leaf node: sum m, sum m x, sum m y, sum m z (m = rho h^3) into
// partials[row][0..3]
__global__ void __launch_bounds__(kScfThreads) scf_com_kernel(const NodeInfo *__restrict__ info,
                                                               const int32_t *__restrict__ leaves,
                                                               const double *__restrict__ levels,
                                                               const double *__restrict__ rho,
                                                               double *__restrict__ partials, ScfGeo g)
{
    const NodeInfo ni = info[leaves[blockIdx.x]];
    const double h3 = levels[ni.level * LEVEL_FIELDS + LV_H3];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = threadIdx.x; c < NCELL; c += kScfThreads) {
        double x[3];
        cell_centre(ni, levels, g, c, x);
        const double m = rho[size_t(ni.leaf_row) * NCELL + c] * h3;
        v[0] += m;
#pragma unroll
        for (int a = 0; a < 3; ++a) v[1 + a] = fma(m, x[a], v[1 + a]);
    }
    block_reduce<4, false>(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) partials[size_t(ni.leaf_row) * 8 + k] = v[k];
}

struct ScfStars {
    double omega2, C[2], com[2], x_split;
    double centre[2][3], r2lim[2];
    int live[2];                         // star i exists (rho_max > 0)
};

// the star a cell belongs to (0, 1) or -1, and its enthalpy
__device__ __forceinline__ int star_of(const double x[3], const ScfStars &s)
{
    const int i = x[0] < s.x_split ? 0 : 1;
    if (!s.live[i]) return -1;
    double d2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) d2 = fma(x[a] - s.centre[i][a], x[a] - s.centre[i][a], d2);
    return d2 < s.r2lim[i] ? i : -1;
}

__device__ __forceinline__ double enthalpy(const double x[3], double phi, int star, const ScfStars &s)
{
    const double wx = x[0] - s.com[0], wy = x[1] - s.com[1];
    return s.C[star] - phi + 0.5 * s.omega2 * fma(wx, wx, wy * wy);
}

// per leaf node: the largest H of each star's cells into partials[row][4..5]
__global__ void __launch_bounds__(kScfThreads) scf_hmax_kernel(const NodeInfo *__restrict__ info,
                                                                const int32_t *__restrict__ leaves,
                                                                const double *__restrict__ levels,
                                                                const double *__restrict__ phi,
                                                                double *__restrict__ partials, ScfGeo g,
                                                                ScfStars s)
{
    const NodeInfo ni = info[leaves[blockIdx.x]];
    double v[2] = {-1e300, -1e300};
    for (int c = threadIdx.x; c < NCELL; c += kScfThreads) {
        double x[3];
        cell_centre(ni, levels, g, c, x);
        const int star = star_of(x, s);
        if (star >= 0) {
            const double H = enthalpy(x, phi[size_t(ni.leaf_row) * NCELL + c], star, s);
            v[star] = fmax(v[star], H);
        }
    }
    block_reduce<2, true>(v);
    if (threadIdx.x == 0) {
        partials[size_t(ni.leaf_row) * 8 + 4] = v[0];
        partials[size_t(ni.leaf_row) * 8 + 5] = v[1];
    }
}

// the new density: max(floor, rho_max,i (H / H_max,i)^n) inside star i where
// H > 0, the floor elsewhere (continuous in H: a cell whose H is zero to
// rounding takes the floor on either side of zero)
__global__ void __launch_bounds__(kScfThreads) scf_density_kernel(
    const NodeInfo *__restrict__ info, const int32_t *__restrict__ leaves,
    const double *__restrict__ levels, const double *__restrict__ phi, double *__restrict__ rho_out,
    ScfGeo g, ScfStars s, double n, double rho_max0, double rho_max1, double ih0, double ih1,
    double floor_value)
{
    const NodeInfo ni = info[leaves[blockIdx.x]];
    for (int c = threadIdx.x; c < NCELL; c += kScfThreads) {
        double x[3];
        cell_centre(ni, levels, g, c, x);
        const size_t idx = size_t(ni.leaf_row) * NCELL + c;
        const int star = star_of(x, s);
        double r = floor_value;
        if (star >= 0) {
            const double H = enthalpy(x, phi[idx], star, s);
            if (H > 0.0)
                r = fmax(floor_value, (star ? rho_max1 : rho_max0) * pow(H * (star ? ih1 : ih0), n));
        }
        rho_out[idx] = r;
    }
}

int scf_fail(int code, const std::string &msg)
{
    record_error("fmm_scf_update: " + msg);
    return code;
}

// leaf row, cell and cell centre of the leaf cell containing a point (false
// if none)
bool find_cell(const fmm_tree_s *t, const double p[3], int64_t &row, int &cell, double centre[3])
{
    const double *lo = t->cfg.box_lo;
    for (const NodeInfo &ni : t->info) {
        if (ni.leaf_row < 0) continue;
        const double n = std::ldexp(1.0, ni.level - 1);
        double q[3];
        const int32_t ij[3] = {ni.ix, ni.iy, ni.iz};
        bool in = true;
        for (int a = 0; a < 3; ++a) {
            q[a] = (p[a] - lo[a]) / t->cfg.box_size * n - ij[a];
            in = in && q[a] >= 0.0 && q[a] < 1.0;
        }
        if (!in) continue;
        row = ni.leaf_row;
        int k[3];
        for (int a = 0; a < 3; ++a) k[a] = int(std::floor(q[a] * 8.0));
        cell = k[0] + 8 * k[1] + 64 * k[2];
        const double h = t->cfg.box_size / (8.0 * n);
        for (int a = 0; a < 3; ++a) centre[a] = lo[a] + (8.0 * ij[a] + k[a] + 0.5) * h;
        return true;
    }
    return false;
}

}  // namespace
}  // namespace fmm

extern "C" int fmm_scf_update(fmm_tree_t t, const fmm_scf_params *p, const double *phi,
                              const double *rho, double *rho_out, fmm_scf_result *out,
                              fmm_stream_t stream)
{
    using namespace fmm;
    if (!t || !p || !phi || !rho || !rho_out || !out) return scf_fail(FMM_ERR_INVALID_ARG, "NULL argument");
    if (t->host_only) return scf_fail(FMM_ERR_INVALID_ARG, "tree was planned with FMM_FLAG_HOST_ONLY");
    if (t->n_trees != 1) return scf_fail(FMM_ERR_INVALID_ARG, "the tree must hold a single tree");
    if (!(p->n > 0.0) || !(p->rho_max[0] > 0.0) || !(p->rho_max[1] >= 0.0) ||
        !(p->rho_floor >= 0.0) || !(p->r_lim[0] > 0.0) ||
        !(p->r_lim[1] >= 0.0) || (p->rho_max[1] > 0.0 && !(p->r_lim[1] > 0.0)))
        return scf_fail(FMM_ERR_INVALID_ARG, "n, rho_max[0] and r_lim[0] must be positive, "
                                             "rho_max[1], r_lim[1] and rho_floor not negative");
    const int64_t nl = t->n_leaf;
    // the surface conditions hold at the centres of the cells containing the
    // points, where the potential is known
    int64_t row[3] = {0, 0, 0};
    int cell[3] = {0, 0, 0};
    double ctr[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    const double *pts[3] = {p->point_a, p->point_b, p->point_c};
    for (int k = 0; k < 3; ++k) {
        if (k == 1 && !p->rotate) continue;
        if (k == 2 && p->rho_max[1] <= 0.0) continue;
        if (!find_cell(t, pts[k], row[k], cell[k], ctr[k]))
            return scf_fail(FMM_ERR_INVALID_ARG, "a surface point lies outside every leaf node");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int32_t *leaves = t->dev.lists + t->plan.leaves.off;
    const ScfGeo g{{t->cfg.box_lo[0], t->cfg.box_lo[1], t->cfg.box_lo[2]}, t->cfg.box_size};
    // 1. centre of mass; the potential at the surface cells
    scf_com_kernel<<<unsigned(nl), kScfThreads, 0, s>>>(t->dev.info, leaves, t->dev.levels, rho,
                                                         t->dev.partials, g);
    cudaError_t e = cudaGetLastError();
    std::vector<double> part(size_t(nl) * 8);
    double phis[3] = {0.0, 0.0, 0.0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(part.data(), t->dev.partials, part.size() * sizeof(double),
                            cudaMemcpyDeviceToHost, s);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(&phis[k], phi + row[k] * NCELL + cell[k], sizeof(double),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return scf_fail(FMM_ERR_CUDA, cudaGetErrorString(e));
    double msum = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for (int64_t r = 0; r < nl; ++r) {        // fixed order
        msum += part[size_t(r) * 8];
        mx += part[size_t(r) * 8 + 1];
        my += part[size_t(r) * 8 + 2];
        mz += part[size_t(r) * 8 + 3];
    }
    if (!(msum > 0.0)) return scf_fail(FMM_ERR_INVALID_ARG, "the density has no positive mass");
    ScfStars st{};
    st.com[0] = mx / msum;
    st.com[1] = my / msum;
    auto w2 = [&](const double *q) {
        const double dx = q[0] - st.com[0], dy = q[1] - st.com[1];
        return dx * dx + dy * dy;
    };
    // 2. the iteration's scalars from H = 0 at the surface points
    st.omega2 = 0.0;
    if (p->rotate) {
        const double den = w2(ctr[0]) - w2(ctr[1]);
        if (den == 0.0) return scf_fail(FMM_ERR_INVALID_ARG, "points A and B are equally far from the axis");
        st.omega2 = 2.0 * (phis[0] - phis[1]) / den;
    }
    st.C[0] = phis[0] - 0.5 * st.omega2 * w2(ctr[0]);
    st.C[1] = p->rho_max[1] > 0.0 ? phis[2] - 0.5 * st.omega2 * w2(ctr[2]) : 0.0;
    st.x_split = p->x_split;
    for (int i = 0; i < 2; ++i) {
        for (int a = 0; a < 3; ++a) st.centre[i][a] = p->centre[i][a];
        st.r2lim[i] = p->r_lim[i] * p->r_lim[i];
        st.live[i] = p->rho_max[i] > 0.0;
    }
    // 3. each star's largest enthalpy
    scf_hmax_kernel<<<unsigned(nl), kScfThreads, 0, s>>>(t->dev.info, leaves, t->dev.levels, phi,
                                                          t->dev.partials, g, st);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(part.data(), t->dev.partials, part.size() * sizeof(double),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return scf_fail(FMM_ERR_CUDA, cudaGetErrorString(e));
    double hmax[2] = {-1e300, -1e300};
    for (int64_t r = 0; r < nl; ++r)
        for (int i = 0; i < 2; ++i) hmax[i] = std::fmax(hmax[i], part[size_t(r) * 8 + 4 + i]);
    for (int i = 0; i < 2; ++i)
        if (st.live[i] && !(hmax[i] > 0.0))
            return scf_fail(FMM_ERR_INVALID_ARG, "a star has no cell with positive enthalpy");
    // 4. the new density
    scf_density_kernel<<<unsigned(nl), kScfThreads, 0, s>>>(
        t->dev.info, leaves, t->dev.levels, phi, rho_out, g, st, p->n, p->rho_max[0],
        p->rho_max[1], 1.0 / hmax[0], st.live[1] ? 1.0 / hmax[1] : 0.0, p->rho_floor);
    e = cudaGetLastError();
    if (e != cudaSuccess) return scf_fail(FMM_ERR_CUDA, cudaGetErrorString(e));
    out->omega2 = st.omega2;
    out->C[0] = st.C[0];
    out->C[1] = st.C[1];
    out->com[0] = st.com[0];
    out->com[1] = st.com[1];
    out->com[2] = mz / msum;
    out->H_max[0] = hmax[0];
    out->H_max[1] = st.live[1] ? hmax[1] : 0.0;
    out->phi_points[0] = phis[0];
    out->phi_points[1] = phis[1];
    out->phi_points[2] = phis[2];
    out->mass = msum;
    return FMM_OK;
}
