// probe.cu -- FMA throughput probe (instrumentation; no counterpart in the paper).
// Eight independent FMA chains per thread, 8 CTAs of 256 threads per SM, so the
// FP32 or FP64 pipe is the only limit. Used by the benchmark to report the
// ALU-bound kernels against the rate this GPU actually delivers.
#include "../../include/stokes.h"
#include "internal.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T a, T b, T* out) {
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = x[c] * a + b;
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    out[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

template <typename T>
stokes_status probe(int iters, double* tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return STOKES_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return STOKES_ECUDA;
    const int blocks = sms * 8, threads = 256;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * size_t(blocks) * threads) != cudaSuccess) return STOKES_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_probe<T><<<blocks, threads>>>(16, T(0.999), T(1e-4), out);   // warm-up
    cudaEventRecord(e0);
    k_fma_probe<T><<<blocks, threads>>>(iters, T(0.999), T(1e-4), out);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0.0f) return STOKES_ECUDA;
    *tflops = 2.0 * 8.0 * double(blocks) * threads * iters / (double(ms) * 1e-3) / 1e12;
    return STOKES_OK;
}

}  // namespace

extern "C" stokes_status stokes_probe_fma(double* fp32_tflops, double* fp64_tflops) {
    if (!fp32_tflops || !fp64_tflops) return STOKES_EINVAL;
    stokes_status s = probe<float>(65536, fp32_tflops);
    if (s != STOKES_OK) return s;
    return probe<double>(2048, fp64_tflops);
}
