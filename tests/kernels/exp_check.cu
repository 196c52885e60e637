// Test harness: evaluates exp_tab (the step kernel's FP64 exp) on host-given points.
#include <cuda_runtime.h>

#include "fp64_exp.cuh"

__global__ void k_exp(const double *x, double *y, long long n)
{
    __shared__ double e2[32];
    if (threadIdx.x < 32) e2[threadIdx.x] = m2m::kExp2j[threadIdx.x];
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = m2m::exp_tab(x[i], e2);
}

extern "C" int exp_check(const double *x, double *y, long long n)
{
    double t[32];
    m2m::exp2_table(t);
    if (cudaMemcpyToSymbol(m2m::kExp2j, t, sizeof t) != cudaSuccess) return 1;
    double *d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(double) * (n > 0 ? n : 1)) != cudaSuccess) return 2;
    cudaMemcpy(d, x, sizeof(double) * n, cudaMemcpyHostToDevice);
    k_exp<<<256, 256>>>(d, d + n, n);
    cudaMemcpy(y, d + n, sizeof(double) * n, cudaMemcpyDeviceToHost);
    const cudaError_t e = cudaDeviceSynchronize();
    cudaFree(d);
    return e == cudaSuccess ? 0 : 3;
}
