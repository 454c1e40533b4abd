// Arithmetic peak probe: FP64 FMA throughput of the device, used as the
// denominator of the roofline of the kernels bound by FP64 arithmetic (the
// Gram-Schmidt passes: about one FP64 FMA per 8 bytes streamed, which on this
// GPU is below the memory ridge).
#include "rte_internal.h"

namespace rte {
namespace {

// Eight independent FMA chains per thread, kIters rounds; the result is
// written only if it is exactly zero so the compiler keeps every FMA.
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) k_dfma(double seed, double* sink) {
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed + 1e-3 * (threadIdx.x + j);
    const double m = 0.999999, c = 1e-7;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 0.0) sink[0] = s;
}

__global__ void __launch_bounds__(256) k_ffma(float seed, float* sink) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed + 1e-3f * (threadIdx.x + j);
    const float m = 0.9999f, c = 1e-7f;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 0.f) sink[0] = s;
}

template <typename K, typename T>
rte_status time_rate(K kern, T seed, void* stream, double* gflops, const char* what) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(nullptr, e, "device query");
    T* sink = nullptr;
    e = cudaMallocAsync(&sink, sizeof(T), st);
    if (e != cudaSuccess) return cuda_status(nullptr, e, "cudaMallocAsync");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int blocks = sms * 8;
    kern<<<blocks, 256, 0, st>>>(seed, sink);          // warm-up
    cudaEventRecord(a, st);
    for (int r = 0; r < 5; ++r) kern<<<blocks, 256, 0, st>>>(seed + (T)r, sink);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFreeAsync(sink, st);
    if (e != cudaSuccess) return cuda_status(nullptr, e, what);
    const double flops = 5.0 * blocks * 256.0 * 8.0 * kIters * 2.0;
    *gflops = flops / (ms * 1e-3) / 1e9;
    return RTE_OK;
}

}  // namespace
}  // namespace rte

extern "C" RTE_API rte_status rte_fp32_fma_rate(void* stream, double* gflops) {
    if (!gflops) { rte::set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    return rte::time_rate(rte::k_ffma, 1.0f, stream, gflops, "rte_fp32_fma_rate");
}

extern "C" RTE_API rte_status rte_fp64_fma_rate(void* stream, double* gflops) {
    using namespace rte;
    if (!gflops) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(nullptr, e, "device query");
    double* sink = nullptr;
    e = cudaMallocAsync(&sink, sizeof(double), st);
    if (e != cudaSuccess) return cuda_status(nullptr, e, "cudaMallocAsync");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int blocks = sms * 8;
    k_dfma<<<blocks, 256, 0, st>>>(1.0, sink);          // warm-up
    cudaEventRecord(a, st);
    for (int r = 0; r < 5; ++r) k_dfma<<<blocks, 256, 0, st>>>(1.0 + r, sink);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFreeAsync(sink, st);
    if (e != cudaSuccess) return cuda_status(nullptr, e, "rte_fp64_fma_rate");
    const double flops = 5.0 * blocks * 256.0 * 8.0 * kIters * 2.0;
    *gflops = flops / (ms * 1e-3) / 1e9;
    return RTE_OK;
}
