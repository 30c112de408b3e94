// lbm_calib.cu -- lbm_measure_fp64_fma: the FP64 fused multiply-add throughput of
// the GPU, measured with a kernel of independent DFMA chains. It is the peak the
// FP64 storage form's arithmetic roofline is set against (that form is bound by
// the FP64 pipe, not by memory); the paper has no counterpart.
#include <cuda_runtime.h>

#include "lbm.h"

namespace {

constexpr int kChains = 8;        // independent FMA chains a thread (latency hiding)
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) dfma_chains(double* __restrict__ out, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-9 * threadIdx.x + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[(long long)blockIdx.x * kThreads + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" lbm_status lbm_measure_fp64_fma(void* cuda_stream, double* tflops) {
    if (!tflops) return LBM_EINVAL;
    *tflops = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return LBM_ECUDA;
    const int blocks = sms * 8, iters = 4096;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lbm_status st = LBM_ECUDA;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(double)) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        dfma_chains<<<blocks, kThreads, 0, s>>>(out, iters, 0.9999999, 1e-7);   // warm-up
        cudaEventRecord(e0, s);
        dfma_chains<<<blocks, kThreads, 0, s>>>(out, iters, 0.9999999, 1e-7);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            cudaGetLastError() == cudaSuccess && ms > 0.f) {
            const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
            *tflops = flops / (ms * 1e-3) / 1e12;
            st = LBM_OK;
        }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}
