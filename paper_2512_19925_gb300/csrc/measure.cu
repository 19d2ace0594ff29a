// measure.cu -- the device's FP64 fused multiply-add rate, measured by the
// library's own loop (the denominator of the FP64 path's ALU roofline).
//
// Every thread runs eight independent chains x <- x a + b (one DFMA each per
// iteration, two floating-point operations), so that the FP64 pipe, not the
// chains' latency, bounds the loop; a grid of eight blocks of 256 threads
// per SM keeps every SM's pipe busy.
#include "../../include/hww.h"
#include "hww_internal.cuh"

namespace {

constexpr int DFMA_CHAINS = 8;
constexpr int DFMA_BLOCK = 256;

__global__ void __launch_bounds__(DFMA_BLOCK) dfma_loop_kernel(double* sink, long long iters, double a, double b) {
    double x[DFMA_CHAINS];
#pragma unroll
    for (int k = 0; k < DFMA_CHAINS; ++k) x[k] = (double)(threadIdx.x + k) * 1e-9;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < DFMA_CHAINS; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < DFMA_CHAINS; ++k) s += x[k];
    if (s == 1234.5) sink[0] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" hww_status hww_dfma_rate(int64_t iters, double* flops_per_s) {
    if (!flops_per_s || iters < 1) return HWW_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HWW_ERR_NO_DEVICE;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return hww::record_cuda_error(e);
    double* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&sink, sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int grid = 8 * nsm;
    float ms = 0.f;
    if (e == cudaSuccess) {
        dfma_loop_kernel<<<grid, DFMA_BLOCK>>>(sink, iters / 8 + 1, 0.999999, 1e-7);  // warm-up
        cudaEventRecord(e0);
        dfma_loop_kernel<<<grid, DFMA_BLOCK>>>(sink, iters, 0.999999, 1e-7);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return hww::record_cuda_error(e);
    const double flops = 2.0 * (double)DFMA_CHAINS * (double)iters * (double)grid * (double)DFMA_BLOCK;
    *flops_per_s = ms > 0.f ? flops / (ms * 1e-3) : 0.0;
    return HWW_OK;
}
