// Test helper: Philox4x32-10 outputs from cuRAND (curand_Philox4x32_10, a
// public device function of the CUDA toolkit) for given counters and keys,
// as an independent implementation to check the oracle's generator against.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void k(const uint4 *ctr, const uint2 *key, uint4 *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_philox_ref(const unsigned *ctr, const unsigned *key, unsigned *out, int n) {
    uint4 *dc = nullptr, *dout = nullptr;
    uint2 *dk = nullptr;
    if (cudaMalloc(&dc, sizeof(uint4) * n) || cudaMalloc(&dk, sizeof(uint2) * n) ||
        cudaMalloc(&dout, sizeof(uint4) * n))
        return 1;
    cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dk, key, sizeof(uint2) * n, cudaMemcpyHostToDevice);
    k<<<(n + 127) / 128, 128>>>(dc, dk, dout, n);
    int err = cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost) != cudaSuccess;
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return err;
}
