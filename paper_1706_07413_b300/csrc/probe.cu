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

// ---------------------------------------------------------------------------------------------
// The solver's e^{-x} (expneg.cuh) on an array, for verification against a reference exp.

#include <cmath>
#include <vector>

#include "expneg.cuh"

namespace {

template <bool SCALED>
__global__ void exp_neg_kernel(const double *x, double *y, long long n, const double *tab_g)
{
    __shared__ double tab[adscl::kExpTableSize];
    for (int i = threadIdx.x; i < adscl::kExpTableSize; i += blockDim.x) tab[i] = tab_g[i];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = SCALED ? adscl::a_exp_neg_scaled(1.0, x[i], tab) : adscl::a_exp_neg(1.0, x[i], tab);
}

template <bool SCALED>
adscl_status exp_neg_host(int32_t device, const double *x, double *y, int64_t n)
{
    if (!x || !y || n < 0) return ADSCL_EINVAL;
    if (n == 0) return ADSCL_OK;
    if (cudaSetDevice(device) != cudaSuccess) return ADSCL_ECUDA;
    std::vector<double> tab(adscl::kExpTableSize);
    for (int j = 0; j < adscl::kExpTableSize; ++j) tab[j] = (double)std::exp2l((long double)j / 256.0L);
    double *dx = nullptr, *dy = nullptr, *dt = nullptr;
    adscl_status st = ADSCL_OK;
    const size_t nb = (size_t)n * sizeof(double);
    if (cudaMalloc(&dx, nb) != cudaSuccess || cudaMalloc(&dy, nb) != cudaSuccess ||
        cudaMalloc(&dt, tab.size() * sizeof(double)) != cudaSuccess) {
        st = ADSCL_ENOMEM;
    } else if (cudaMemcpy(dx, x, nb, cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemcpy(dt, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        st = ADSCL_ECUDA;
    } else {
        exp_neg_kernel<SCALED><<<256, 256>>>(dx, dy, n, dt);
        if (cudaGetLastError() != cudaSuccess || cudaMemcpy(y, dy, nb, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = ADSCL_ECUDA;
    }
    if (dx) cudaFree(dx);
    if (dy) cudaFree(dy);
    if (dt) cudaFree(dt);
    return st;
}

}  // namespace

extern "C" adscl_status adscl_exp_neg(int32_t device, const double *x, double *y, int64_t n)
{
    return exp_neg_host<false>(device, x, y, n);
}

extern "C" adscl_status adscl_exp_neg_scaled(int32_t device, const double *X, double *y, int64_t n)
{
    return exp_neg_host<true>(device, X, y, n);
}
