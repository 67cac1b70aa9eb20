// peaks.cu -- measured FP32 and FP64 FMA throughput of the current GPU, the
// denominators of the ALU rooflines of the on-the-fly Legendre kernels.
// Every thread runs 8 independent FMA chains; the chains' sum goes to a
// device word that nothing reads, so the arithmetic cannot be removed.
#include <cuda_runtime.h>

#include "sht_internal.h"

namespace sht {
namespace {

__device__ float g_sink32;
__device__ double g_sink64;

template <typename T, int ITERS>
__global__ void __launch_bounds__(256) k_fma_chain(T seed, T mul, T add)
{
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed + T(threadIdx.x + i);
#pragma unroll 16
    for (int it = 0; it < ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], mul, add);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == T(-1.2345)) {
        if (sizeof(T) == 4) g_sink32 = (float)s;
        else g_sink64 = (double)s;
    }
}

template <typename T, int ITERS>
int time_chain(int blocks, cudaStream_t s, double &tflops)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SHT_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return SHT_ECUDA; }
    // mul slightly below 1 keeps the chains finite
    k_fma_chain<T, ITERS><<<blocks, 256, 0, s>>>(T(1), T(0.999999), T(1e-3));   // warm-up
    cudaEventRecord(e0, s);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) k_fma_chain<T, ITERS><<<blocks, 256, 0, s>>>(T(1), T(0.999999), T(1e-3));
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0.f) return SHT_ECUDA;
    const double flops = 2.0 * 8.0 * ITERS * 256.0 * blocks * reps;
    tflops = flops / (ms * 1e-3) / 1e12;
    return SHT_OK;
}

}  // namespace
}  // namespace sht

extern "C" SHT_API int sht_alu_peaks(double *fp32_tflops, double *fp64_tflops, void *stream)
{
    if (!fp32_tflops || !fp64_tflops) return sht::set_error(SHT_EINVAL, "sht_alu_peaks: null output pointer");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return sht::set_error(SHT_ECUDA, "sht_alu_peaks: no CUDA device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = sht::time_chain<float, 4096>(sms * 8, s, *fp32_tflops);
    if (rc == SHT_OK) rc = sht::time_chain<double, 256>(sms * 8, s, *fp64_tflops);
    if (rc != SHT_OK) return sht::set_error(rc, "sht_alu_peaks: timing failed");
    return SHT_OK;
}
