// Test helper: cuRAND's device Philox4x32-10 (curand_kernel.h) for raw
// counters, as a reference for the library's generator. curand_init(seed,
// subsequence, 0) starts at counter (0, 0, subsequence low, subsequence high)
// with key (seed low, seed high); skipping 4 c outputs (c = ctr.x | ctr.y << 32)
// moves it to (ctr.x, ctr.y, ctr.z, ctr.w), and curand4 returns that block.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void curand_philox_kernel(unsigned long long seed, const uint4 *ctr, long long n, uint4 *out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = ctr[i];
    curandStatePhilox4_32_10_t st;
    const unsigned long long sub = (unsigned long long)c.z | ((unsigned long long)c.w << 32);
    const unsigned long long pos = (unsigned long long)c.x | ((unsigned long long)c.y << 32);
    curand_init(seed, sub, 0ull, &st);
    // skip `pos` blocks of four outputs: 4 pos overflows 64 bits for pos >= 2^62,
    // so the top three bits of pos are skipped 2^61 blocks at a time
    skipahead((pos & ((1ull << 61) - 1ull)) * 4ull, &st);
    for (unsigned long long k = 0; k < (pos >> 61); ++k) skipahead(1ull << 63, &st);
    out[i] = curand4(&st);
}

extern "C" int curand_philox(unsigned long long seed, const uint32_t *ctr, long long n, uint32_t *out) {
    uint4 *d_c = nullptr, *d_o = nullptr;
    if (cudaMalloc(&d_c, n * 16) != cudaSuccess || cudaMalloc(&d_o, n * 16) != cudaSuccess) return 1;
    cudaMemcpy(d_c, ctr, n * 16, cudaMemcpyHostToDevice);
    curand_philox_kernel<<<(unsigned)((n + 255) / 256), 256>>>(seed, d_c, n, d_o);
    cudaMemcpy(out, d_o, n * 16, cudaMemcpyDeviceToHost);
    const cudaError_t e = cudaGetLastError();
    cudaFree(d_c);
    cudaFree(d_o);
    return e == cudaSuccess ? 0 : 2;
}
