// Time derivative of the gravitational potential and field, for total-energy
// conservation (Sec. 2: besides angular momentum, the solver needs the time
// derivative of the gravitational field, coupled to the hydrodynamics, so
// that total energy is conserved).  The paper gives no formula; the reading
// here is the exact time derivative of the discrete solve along the
// density's rate of change,
//   phi_dot = d/dt phi_FMM(rho + t rho_dot) at t = 0,  g_dot likewise,
// which includes the motion of every refined cell's centre of mass.  It is
// formed from four solves of the same tree by the fourth-order central
// difference
//   f'(0) ~ [8 (f(e) - f(-e)) - (f(2e) - f(-2e))] / (12 e),
// truncation O(e^4), rounding about (unit roundoff of the solve) / e.
#include <string>

#include "fmm_internal.h"

namespace fmm {
namespace {

// rho_work = rho + a rho_dot (the density at time a)
__global__ void shifted_density_kernel(const double *__restrict__ rho,
                                       const double *__restrict__ rho_dot, double a, int64_t n,
                                       double *__restrict__ out)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        out[i] = fma(a, rho_dot[i], rho[i]);
}

// out = w in (first) or out += w in
__global__ void weighted_sum_kernel(const double *__restrict__ in, double w, int64_t n, int first,
                                    double *__restrict__ out)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        out[i] = first ? w * in[i] : fma(w, in[i], out[i]);
}

unsigned grid_for(int64_t n)
{
    const int64_t blocks = (n + 255) / 256;
    const int64_t cap = int64_t(sm_count_of_current_device()) * 8;
    return unsigned(blocks < cap ? blocks : cap);
}

}  // namespace
}  // namespace fmm

extern "C" int fmm_field_time_derivative(fmm_tree_t t, const double *rho, const double *rho_dot,
                                         double eps, double *rho_work, double *M, double *com,
                                         void *L, float *L_comp, double *dL1, double *L64,
                                         double *dL1_acc, double *phi, double *g, double *totals,
                                         double *phi_dot, double *g_dot, fmm_stream_t stream)
{
    using namespace fmm;
    if (!t) {
        record_error("fmm_field_time_derivative: tree is NULL");
        return FMM_ERR_INVALID_ARG;
    }
    if (!rho || !rho_dot || !rho_work || !phi_dot || !g_dot) {
        record_error("fmm_field_time_derivative: NULL buffer");
        return FMM_ERR_INVALID_ARG;
    }
    if (!(eps > 0.0) || !(eps < 1e300)) {
        record_error("fmm_field_time_derivative: eps must be positive and finite");
        return FMM_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t nrho = t->n_leaf * NCELL, ng = t->n_leaf * 3 * NCELL;
    // the four solves, in a fixed order (deterministic)
    const double a[4] = {eps, -eps, 2.0 * eps, -2.0 * eps};
    const double w[4] = {8.0 / (12.0 * eps), -8.0 / (12.0 * eps), -1.0 / (12.0 * eps),
                         1.0 / (12.0 * eps)};
    for (int k = 0; k < 4; ++k) {
        shifted_density_kernel<<<grid_for(nrho), 256, 0, s>>>(rho, rho_dot, a[k], nrho, rho_work);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            record_error(std::string("fmm_field_time_derivative: ") + cudaGetErrorString(e));
            return FMM_ERR_CUDA;
        }
        int rc = fmm_step(t, rho_work, M, com, L, L_comp, dL1, L64, dL1_acc, phi, g, totals, stream);
        if (rc) return rc;
        weighted_sum_kernel<<<grid_for(nrho), 256, 0, s>>>(phi, w[k], nrho, k == 0, phi_dot);
        weighted_sum_kernel<<<grid_for(ng), 256, 0, s>>>(g, w[k], ng, k == 0, g_dot);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            record_error(std::string("fmm_field_time_derivative: ") + cudaGetErrorString(e));
            return FMM_ERR_CUDA;
        }
    }
    return FMM_OK;
}
