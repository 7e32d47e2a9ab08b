// Diagnostics: the integer-pipe float <-> double conversions of
// fmm_convert.cuh against the hardware conversion instructions, and the
// arithmetic-pipe peak rates of this GPU (the roofline denominators of the
// FP32- and FP64-bound kernels).
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

// Peak-rate loop: every thread runs kChains independent fused multiply-add
// chains, kUnroll steps per loop iteration, so the loop's own instructions
// take about 1 % of the issue slots.  KIND 0: fmaf; 1: the paired FP32 form
// (fma.rn.f32x2, two lanes per instruction); 2: FP64 fma.  The multiplier
// and addend keep every value finite and normal for any iteration count.
// The final values reach memory only through a comparison the compiler cannot
// decide, so no chain is dead code.
constexpr int kPeakThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) peak_kernel(int64_t iters, float seed,
                                                            float *__restrict__ sink)
{
    if constexpr (KIND == 0) {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = seed * float(threadIdx.x + k + 1);
        const float m = 0.9999999f, c = 1e-7f;
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) t += a[k];
        if (t == -1.f) sink[0] = t;
    } else if constexpr (KIND == 1) {
        float2 a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k)
            a[k] = make_float2(seed * float(threadIdx.x + k + 1), seed * float(threadIdx.x + k + 2));
        const float2 m = make_float2(0.9999999f, 0.9999998f), c = make_float2(1e-7f, 2e-7f);
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], m, c);
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) t += a[k].x + a[k].y;
        if (t == -1.f) sink[0] = t;
    } else {
        double a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = double(seed) * double(threadIdx.x + k + 1);
        const double m = 0.9999999999, c = 1e-10;
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) t += a[k];
        if (t == -1.0) sink[0] = float(t);
    }
}

}  // namespace

extern "C" int fmm_peak_rate(int32_t kind, int64_t iters, int32_t blocks_per_sm, float *sink,
                             double *flops, fmm_stream_t stream)
{
    if (kind < 0 || kind > 2 || iters < 1 || iters > (int64_t(1) << 40) || blocks_per_sm < 1 ||
        blocks_per_sm > 32 || !sink || !flops) {
        fmm::record_error("fmm_peak_rate: kind must be 0..2, iters 1..2^40, blocks_per_sm 1..32, "
                          "sink and flops non-NULL");
        return FMM_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        fmm::record_error(std::string("fmm_peak_rate: ") + cudaGetErrorString(e));
        return FMM_ERR_CUDA;
    }
    const unsigned grid = unsigned(sms) * unsigned(blocks_per_sm);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (kind == 0) peak_kernel<0><<<grid, kPeakThreads, 0, s>>>(iters, 1e-3f, sink);
    else if (kind == 1) peak_kernel<1><<<grid, kPeakThreads, 0, s>>>(iters, 1e-3f, sink);
    else peak_kernel<2><<<grid, kPeakThreads, 0, s>>>(iters, 1e-3f, sink);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        fmm::record_error(std::string("fmm_peak_rate: ") + cudaGetErrorString(e));
        return FMM_ERR_CUDA;
    }
    // two flops per fused multiply-add lane
    const double lanes = kind == 1 ? 2.0 : 1.0;
    *flops = double(grid) * kPeakThreads * double(iters) * kUnroll * kChains * lanes * 2.0;
    return FMM_OK;
}

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
