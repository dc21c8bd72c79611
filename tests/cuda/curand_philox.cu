// Test helper: draws from cuRAND's device Philox4_32_10 generator, so that the
// project's Philox4x32-10 implementations can be compared with a library that
// is run, not copied.  Built by the GPU test that uses it.
#include <cstdint>
#include <curand_kernel.h>

__global__ void draw_kernel(unsigned long long seed, unsigned long long subsequence, unsigned long long offset,
                            uint32_t *out, int n)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subsequence, offset, &st);
    for (int k = 0; k < n; ++k) {
        const uint4 v = curand4(&st);
        out[4 * k + 0] = v.x;
        out[4 * k + 1] = v.y;
        out[4 * k + 2] = v.z;
        out[4 * k + 3] = v.w;
    }
}

extern "C" int curand_philox_draw(unsigned long long seed, unsigned long long subsequence,
                                  unsigned long long offset, uint32_t *host_out, int n)
{
    uint32_t *d = nullptr;
    if (cudaMalloc(&d, sizeof(uint32_t) * 4 * n) != cudaSuccess) return -1;
    draw_kernel<<<1, 1>>>(seed, subsequence, offset, d, n);
    cudaError_t e = cudaMemcpy(host_out, d, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : -2;
}
