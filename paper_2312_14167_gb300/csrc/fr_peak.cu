// Arithmetic peak of this GPU's FMA pipes, measured (fr_alu_peak): the
// roofline denominator of an ALU-bound kernel (the plain FP64 path).  Every
// thread runs independent FMA chains with operands in registers; the rate
// is 2 flops per FMA over the CUDA-event time of one launch sized to keep
// every SM busy for a few milliseconds.  The result sink is a fixed device
// array inside the library, so nothing is allocated.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "fr_internal.h"

namespace frk {

constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 256;

__device__ double g_peak_sink[64];

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int iters, T m, T c) {
    T x[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) x[k] = fma(x[k], m, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += x[k];
    // m and c keep the chains bounded; the store only keeps them alive
    if (s == (T)-1.2345e30) g_peak_sink[threadIdx.x & 63] = (double)s;
}

}  // namespace frk

extern "C" fr_status fr_alu_peak(int precision, double *flops_per_s) {
    if (!flops_per_s || (precision != FR_FP64 && precision != FR_FP32)) {
        fr::set_error("invalid fr_alu_peak arguments");
        return FR_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int blocks = sms * 8;
    const int iters = precision == FR_FP64 ? 2048 : 16384;
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first is a warm-up
        cudaEventRecord(a, 0);
        if (precision == FR_FP64)
            frk::k_fma_peak<double><<<blocks, frk::kPeakThreads>>>(iters, 0.999999, 1e-7);
        else
            frk::k_fma_peak<float><<<blocks, frk::kPeakThreads>>>(iters, 0.9999f, 1e-5f);
        cudaEventRecord(b, 0);
        e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess || !(best > 0.f)) {
        fr::set_error(std::string("fr_alu_peak: ") + cudaGetErrorString(e));
        return FR_ERR_CUDA;
    }
    const double flops = 2.0 * frk::kPeakChains * (double)iters * frk::kPeakThreads * (double)blocks;
    *flops_per_s = flops / (best * 1e-3);
    return FR_OK;
}
