// Measured FP32 lane rate: the denominator of the rooflines of this library's
// kernels, which are bound by FP32 issue rather than by HBM or tensor cores.
//
// A grid of sm_count x 8 CTAs of 256 threads runs a loop of independent fused
// multiply-adds (8 chains per thread, so that no chain waits on its own
// latency) and is timed with CUDA events on the caller's stream.  One FMA on
// one lane counts as one lane-operation, the unit the kernels' algorithmic
// counts use.
#include "af_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 8192;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_rate_kernel(float a, float b, float *__restrict__ sink)
{
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (float)(threadIdx.x + c);
#pragma unroll 4
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == 1234.5f) sink[0] = s;     // keeps the loop; never true for the a, b used
}

}  // namespace

extern "C" af_status af_fp32_lane_rate(float *d_sink, void *stream, double *h_rate)
{
    if (!d_sink || !h_rate) return af_set_error(AF_ERR_ARG, "af_fp32_lane_rate: NULL argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return af_set_error(AF_ERR_CUDA, "af_fp32_lane_rate: %s", cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    const int blocks = sms * 8;
    // a = 1 - 2^-20, b = 2^-10: the chains stay finite and never reach the sink value
    const float a = 0.99999905f, b = 0.0009765625f;
    float ms = 0.0f;
    if (e == cudaSuccess) {
        fma_rate_kernel<<<blocks, kThreads, 0, st>>>(a, b, d_sink);          // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) {
        for (int r = 0; r < 4; ++r) fma_rate_kernel<<<blocks, kThreads, 0, st>>>(a, b, d_sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return af_set_error(AF_ERR_CUDA, "af_fp32_lane_rate: %s", cudaGetErrorString(e));
    const double lane_ops = 4.0 * blocks * (double)kThreads * kIters * kChains;
    *h_rate = ms > 0.0f ? lane_ops / (ms * 1e-3) : 0.0;
    return af_set_error(AF_OK, "");
}
