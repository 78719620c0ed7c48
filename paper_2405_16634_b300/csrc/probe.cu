// probe.cu -- measured FP32 FMA throughput of the device, the denominator
// against which the pair kernels (bound by FP32 issue) can be read besides the
// nominal SMs x 128 lanes x 2 x clock.
//
// Every thread runs eight independent FMA chains (enough to cover the FMA
// latency at full occupancy), so the only limit is the FMA pipe.
#include "common.cuh"

namespace wnnc {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, float seed, float* out) {
    float a[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
    const float m = 0.999999f, d = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) a[c] = fmaf(a[c], m, d);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += a[c];
    if (s == 12345.678f) out[0] = s;   // keeps the chains live; never true in practice
}

}  // namespace

// FP32 TFLOP/s of an FMA stream over all SMs, timed with CUDA events on `s`.
double probe_fp32(cudaStream_t s) {
    int dev = 0, sms = 0;
    WNNC_CUDA(cudaGetDevice(&dev));
    WNNC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;   // 2048 threads per SM
    const int iters = 1 << 14;
    float* sink = dalloc<float>(1);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    WNNC_CUDA(cudaEventCreate(&e0));
    WNNC_CUDA(cudaEventCreate(&e1));
    k_fma_probe<<<blocks, kProbeThreads, 0, s>>>(iters, 1.f, sink);   // warm-up
    WNNC_LAUNCH_CHECK();
    WNNC_CUDA(cudaEventRecord(e0, s));
    k_fma_probe<<<blocks, kProbeThreads, 0, s>>>(iters, 2.f, sink);
    WNNC_LAUNCH_CHECK();
    WNNC_CUDA(cudaEventRecord(e1, s));
    WNNC_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    WNNC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pool_free(sink);
    const double flops = 2.0 * kProbeChains * (double)iters * (double)blocks * kProbeThreads;
    return flops / (ms * 1e-3) / 1e12;
}

}  // namespace wnnc
