// Test helper: cuRAND's device Philox4x32-10 on given counters and key, to
// pin the two independent Philox implementations (library and CPU checker)
// against a library routine.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void curand_philox_kernel(const uint4* ctr, uint2 key, uint4* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key);
}

extern "C" int curand_philox_ref(const uint32_t* ctr, uint32_t k0, uint32_t k1, int n, uint32_t* out) {
    if (n <= 0) return 0;
    uint4 *dc = nullptr, *dout = nullptr;
    if (cudaMalloc(&dc, sizeof(uint4) * n) != cudaSuccess) return 1;
    if (cudaMalloc(&dout, sizeof(uint4) * n) != cudaSuccess) { cudaFree(dc); return 1; }
    cudaError_t e = cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        curand_philox_kernel<<<(n + 255) / 256, 256>>>(dc, make_uint2(k0, k1), dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dout);
    return e == cudaSuccess ? 0 : 1;
}
