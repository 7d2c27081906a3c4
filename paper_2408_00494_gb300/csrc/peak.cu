// FP32 arithmetic peak of the device, measured: the roofline denominator for kernels bound by FP32
// issue (the rollout kernel's ALU roofline). Every thread of a full-occupancy grid runs 16
// independent fused multiply-add chains, so the FMA pipes never wait on a result; a packed variant
// runs the same 16 chains as 8 register pairs through the .f32x2 form. Each multiply-add counts as
// two FP32 operations.
#include "../../include/bssmppi.h"
#include "internal.h"

#include <algorithm>

namespace bss {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 16;

template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads) fp32_peak_kernel(float* sink, int iters, float a, float b)
{
    float x[kPeakChains];
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    if constexpr (PACKED) {
        float2 y[kPeakChains / 2];
#pragma unroll
        for (int j = 0; j < kPeakChains / 2; ++j) y[j] = make_float2(x[2 * j], x[2 * j + 1]);
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 4
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kPeakChains / 2; ++j) y[j] = __ffma2_rn(y[j], a2, b2);
        }
#pragma unroll
        for (int j = 0; j < kPeakChains / 2; ++j) {
            x[2 * j] = y[j].x;
            x[2 * j + 1] = y[j].y;
        }
    } else {
#pragma unroll 4
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kPeakChains; ++j) x[j] = fmaf(x[j], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) s += x[j];
    if (s == -1.0f) sink[0] = s;  // never true (the chains stay positive), but keeps every chain live
}

}  // namespace bss

using namespace bss;

extern "C" int bssmppi_fp32_peak(int32_t packed, int32_t iters, void* cuda_stream, float* h_ms, double* h_tflops,
                                 int32_t* h_sms)
{
    if (iters < 1 || iters > (1 << 24) || !h_ms || !h_tflops || !h_sms) {
        set_thread_error("fp32_peak: iters out of range [1, 2^24] or NULL output");
        return BSSMPPI_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = packed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp32_peak_kernel<true>, kPeakThreads, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp32_peak_kernel<false>, kPeakThreads, 0);
    float* sink = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int grid = std::max(1, per_sm) * sms;
    // a 0.999 x + 1e-3 chain converges to 1 from any start in (0, 1): no overflow, no denormals
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
        e = cudaEventRecord(t0, st);
        if (packed)
            fp32_peak_kernel<true><<<grid, kPeakThreads, 0, st>>>(sink, iters, 0.999f, 1e-3f);
        else
            fp32_peak_kernel<false><<<grid, kPeakThreads, 0, st>>>(sink, iters, 0.999f, 1e-3f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(t1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    }
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return BSSMPPI_ECUDA;
    }
    const double flops = 2.0 * kPeakChains * (double)iters * (double)grid * kPeakThreads;
    *h_ms = ms;
    *h_tflops = flops / (ms * 1e-3) / 1e12;
    *h_sms = sms;
    return BSSMPPI_OK;
}
