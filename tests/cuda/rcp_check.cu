// Test helper: rcp_nr (the channel functions' reciprocal) beside the IEEE
// division 1.0 / x, and rcp_nr_f (the FP32 solve's) beside the correctly
// rounded FP32 reciprocal, on the device, for tests/test_gpu_rcp.py.
#include <cuda_runtime.h>

#include "../../paper_1909_07321_gb300/csrc/rcp.cuh"

__global__ void rcp_pair_kernel(const double *x, int n, double *r_nr, double *r_div)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    r_nr[i] = rmgb::rcp_nr(x[i]);
    r_div[i] = 1.0 / x[i];
}

__global__ void rcp_pair_f32_kernel(const float *x, int n, float *r_nr, float *r_rn)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    r_nr[i] = rmgb::rcp_nr_f(x[i]);
    r_rn[i] = __frcp_rn(x[i]);
}

// FP32: rcp_nr_f (the FP32 solve's pivot reciprocal) beside the correctly
// rounded reciprocal; host arrays in and out; returns a cudaError_t code.
extern "C" int rcp_pair_f32(const float *x, int n, float *r_nr, float *r_rn)
{
    float *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 3 * (size_t)n * sizeof(float));
    if (e != cudaSuccess) return (int)e;
    cudaMemcpy(d, x, (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
    rcp_pair_f32_kernel<<<(n + 255) / 256, 256>>>(d, n, d + n, d + 2 * (size_t)n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
        cudaMemcpy(r_nr, d + n, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
        cudaMemcpy(r_rn, d + 2 * (size_t)n, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
    }
    cudaFree(d);
    return (int)e;
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
