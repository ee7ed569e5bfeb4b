// Measured arithmetic peaks of the device the library runs on: FP32 and FP64
// fused multiply-add throughput (the ALU ceilings of the FP32-mixed and plain
// FP64 paths), timed with CUDA events. Changes no device setting.
#include <cuda_runtime.h>

#include "ad_pic.h"

namespace {

// Each thread runs ILP independent FMA chains of `iters` steps; the chains
// are kept live by one store per thread, so nothing is optimised away.
template <typename T, int ILP>
__global__ void __launch_bounds__(256) fma_chain_kernel(int iters, T a, T b, T* out) {
    T x[ILP];
#pragma unroll
    for (int j = 0; j < ILP; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < ILP; ++j) x[j] = fma(x[j], a, b);
    }
    T s = (T)0;
#pragma unroll
    for (int j = 0; j < ILP; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int fma_peak(double* tflops) {
    constexpr int ILP = 8;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
        return AD_PIC_ERR_CUDA;
    const int blocks = sms * 8, threads = 256;
    const int iters = sizeof(T) == 4 ? 4096 : 256;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) { cudaGetLastError(); return AD_PIC_ERR_OOM; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = (T)0.999999, b = (T)1e-7;
    float best = 1e30f;
    for (int rep = 0; rep < 6; ++rep) {                 // the first launch is a warm-up
        cudaEventRecord(e0, nullptr);
        fma_chain_kernel<T, ILP><<<blocks, threads>>>(iters, a, b, out);
        cudaEventRecord(e1, nullptr);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return AD_PIC_ERR_CUDA;
    const double flops = 2.0 * ILP * (double)iters * blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return AD_PIC_OK;
}

}  // namespace

extern "C" int ad_pic_fma_peak(int precision, double* tflops) {
    if (!tflops) return AD_PIC_ERR_INVALID_ARG;
    if (cudaPeekAtLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
    if (precision == AD_PIC_FP32_MIXED) return fma_peak<float>(tflops);
    if (precision == AD_PIC_FP64) return fma_peak<double>(tflops);
    return AD_PIC_ERR_INVALID_ARG;
}
