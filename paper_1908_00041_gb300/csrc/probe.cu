// Device throughput probes used as roofline denominators for the FP64 pipe (the
// measured HBM and tensor peaks come from elsewhere): dependent-free FMA streams,
// 8 independent chains per thread, 4 CTAs of 256 threads per SM, timed with events.
#include "favest_internal.h"

namespace {

constexpr int kIters = 2048;

__global__ void __launch_bounds__(256) k_probe_dfma(double *out, double a, double b)
{
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5,
           x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < kIters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == 12345.0) out[0] = s;   // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(256) k_probe_ffma(float *out, float a, float b)
{
    float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5,
          x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < 8 * kIters; ++i) {
        x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
        x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
    }
    float s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == 12345.0f) out[0] = s;
}

}  // namespace

extern "C" int favest_probe_peaks(double *fp64_tflops, double *fp32_tflops)
{
    if (!fp64_tflops || !fp32_tflops) return FAVEST_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FAVEST_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void *buf = nullptr;
    if (cudaMalloc(&buf, 64) != cudaSuccess) return FAVEST_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = sms * 4, block = 256;
    float ms = 0.f;
    k_probe_dfma<<<grid, block>>>((double *)buf, 1.0000001, 1e-9);
    cudaEventRecord(e0);
    for (int r = 0; r < 3; ++r) k_probe_dfma<<<grid, block>>>((double *)buf, 1.0000001, 1e-9);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *fp64_tflops = 3.0 * 2.0 * grid * block * 8.0 * kIters / (ms * 1e-3) / 1e12;
    k_probe_ffma<<<grid, block>>>((float *)buf, 1.0000001f, 1e-9f);
    cudaEventRecord(e0);
    for (int r = 0; r < 3; ++r) k_probe_ffma<<<grid, block>>>((float *)buf, 1.0000001f, 1e-9f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *fp32_tflops = 3.0 * 2.0 * grid * block * 8.0 * 8.0 * kIters / (ms * 1e-3) / 1e12;
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return err == cudaSuccess ? FAVEST_OK : FAVEST_ECUDA;
}
