// Test helper: rcp_nr (the channel functions' reciprocal) beside the IEEE
// division 1.0 / x, both on the device, for tests/test_gpu_rcp.py.
#include <cuda_runtime.h>

#include "../../paper_1909_07321_gb300/csrc/rcp.cuh"

__global__ void rcp_pair_kernel(const double *x, int n, double *r_nr, double *r_div)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    r_nr[i] = rmgb::rcp_nr(x[i]);
    r_div[i] = 1.0 / x[i];
}

// Host arrays in and out; returns a cudaError_t code.
extern "C" int rcp_pair(const double *x, int n, double *r_nr, double *r_div)
{
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 3 * (size_t)n * sizeof(double));
    if (e != cudaSuccess) return (int)e;
    cudaMemcpy(d, x, (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
    rcp_pair_kernel<<<(n + 255) / 256, 256>>>(d, n, d + n, d + 2 * (size_t)n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
        cudaMemcpy(r_nr, d + n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(r_div, d + 2 * (size_t)n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
    }
    cudaFree(d);
    return (int)e;
}
