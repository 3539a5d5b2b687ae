// probe.cu -- measured FP64 throughput of the device: the denominator of the roofline of the
// FP64-bound evolution kernels.  Independent fused multiply-add chains on every SM, timed with
// CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include "adscl.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(512) dfma_chains(double *out, int iters, double a, double c)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * threadIdx.x + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" adscl_status adscl_probe_fp64(int32_t device, void *stream_, double *tflops)
{
    if (!tflops) return ADSCL_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_;
    int sms = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return ADSCL_ECUDA;
    const int blocks = 2 * sms, threads = 512, iters = 8192;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    adscl_status st = ADSCL_OK;
    float best = 1e30f;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return ADSCL_ENOMEM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = ADSCL_ECUDA;
    for (int rep = 0; rep < 4 && st == ADSCL_OK; ++rep) {
        cudaEventRecord(e0, stream);
        dfma_chains<<<blocks, threads, 0, stream>>>(out, iters, 0.999999, 1e-9);
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = ADSCL_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    if (st == ADSCL_OK)
        *tflops = 2.0 * (double)blocks * threads * iters * kChains / (best * 1e-3) / 1e12;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}
