// Test probe: error of the step kernel's FP64 reciprocal and square root against
// the correctly rounded CUDA operations, over log-uniform arguments.
#include <cstdio>
#include <cuda_runtime.h>
#include "ark_step.cuh"
__device__ double ulps(double a, double b)
{
    if (a == b) return 0.0;
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    return (double)(ia > ib ? ia - ib : ib - ia);
}
__global__ void probe(long long n, double* res)   // res[0..2] max ulp, res[3..5] count of non-exact
{
    __shared__ double m[6][256];
    double e0 = 0, e1 = 0, e2 = 0, c0 = 0, c1 = 0, c2 = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        // log-uniform in [2^-40, 2^40] from a counter hash
        unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ull;
        h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29;
        const double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
        const double x = exp2(80.0 * u - 40.0);
        const double r = ark::rcp(x);
        double c, rc;
        ark::sqrt_rsqrt(x, c, rc);
        const double d0 = ulps(r, 1.0 / x), d1 = ulps(c, sqrt(x)), d2 = ulps(rc, 1.0 / sqrt(x));
        e0 = fmax(e0, d0); e1 = fmax(e1, d1); e2 = fmax(e2, d2);
        c0 += d0 > 0; c1 += d1 > 0; c2 += d2 > 0;
    }
    m[0][threadIdx.x] = e0; m[1][threadIdx.x] = e1; m[2][threadIdx.x] = e2;
    m[3][threadIdx.x] = c0; m[4][threadIdx.x] = c1; m[5][threadIdx.x] = c2;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < 256; ++t) {
            for (int k = 0; k < 3; ++k) m[k][0] = fmax(m[k][0], m[k][t]);
            for (int k = 3; k < 6; ++k) m[k][0] += m[k][t];
        }
        for (int k = 0; k < 3; ++k) atomicMax((unsigned long long*)&res[k], (unsigned long long)__double_as_longlong(m[k][0]));
        for (int k = 3; k < 6; ++k) atomicAdd(&res[k], m[k][0]);
    }
}
int main()
{
    double* d;
    if (cudaMalloc(&d, 6 * sizeof(double)) != cudaSuccess) return 1;
    cudaMemset(d, 0, 6 * sizeof(double));
    const long long n = 1ll << 26;
    probe<<<152 * 8, 256>>>(n, d);
    double h[6];
    cudaError_t e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    printf("n=%lld  max ulp: rcp %.0f  sqrt %.0f  rsqrt %.0f   not correctly rounded: rcp %.0f sqrt %.0f rsqrt %.0f  (%s)\n",
           n, h[0], h[1], h[2], h[3], h[4], h[5], cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 2;
}
