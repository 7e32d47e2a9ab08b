// Diagnostic: the integer-pipe float <-> double conversions of
// fmm_convert.cuh against the hardware conversion instructions.
#include <string>

#include "fmm_convert.cuh"
#include "fmm_internal.h"

namespace {

// per input: round-to-nearest, truncation and the exact widening of the
// rounded value, each compared bit for bit with the hardware's result
__global__ void check_kernel(const double *__restrict__ in, int64_t n, int32_t *__restrict__ bad)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const double d = in[i];
        // the helpers' domain: zeros, infinities, NaNs and magnitudes from
        // the smallest normal float up
        const bool in_domain = d == 0.0 || isinf(d) || isnan(d) || fabs(d) >= 1.1754943508222875e-38;
        if (!in_domain) continue;
        const float rn = __double2float_rn(d);
        const float rz = __double2float_rz(d);
        int32_t b = 0;
        if (isnan(d) ? !isnan(fmm::d2f_rn(d)) : __float_as_uint(fmm::d2f_rn(d)) != __float_as_uint(rn))
            b |= 1;
        // truncation of a finite value beyond the float range saturates to
        // infinity in the helper (the hardware gives the largest float): only
        // values inside the range are compared
        if (!isnan(d) && fabs(d) < 3.4028234663852886e38 &&
            __float_as_uint(fmm::d2f_trunc(d)) != __float_as_uint(rz))
            b |= 2;
        if (!isnan(rn) && __double_as_longlong(fmm::f2d_bits(rn)) != __double_as_longlong(double(rn)))
            b |= 4;
        if (b) atomicOr(bad, b);
    }
}

}  // namespace

extern "C" int fmm_check_conversions(const double *values, int64_t n, int32_t *mismatch,
                                     fmm_stream_t stream)
{
    if (!values || !mismatch || n < 0) {
        fmm::record_error("fmm_check_conversions: NULL buffer or negative count");
        return FMM_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(mismatch, 0, sizeof(int32_t), s);
    if (e == cudaSuccess && n > 0) {
        const int64_t blocks = (n + 255) / 256;
        check_kernel<<<unsigned(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(values, n, mismatch);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        fmm::record_error(std::string("fmm_check_conversions: ") + cudaGetErrorString(e));
        return FMM_ERR_CUDA;
    }
    return FMM_OK;
}
