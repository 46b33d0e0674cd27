// curand_ref.cu -- test helper: Philox4_32_10 outputs from cuRAND's device
// API for arbitrary counters, to pin the oracle's generator on all four
// counter words.  curand_init(seed, subsequence = c2 | c3 << 32, 0) sets the
// upper counter words; skipping 4n elements advances words 0-1 by n blocks,
// done in four steps of 4 (n >> 2) plus 4 (n & 3) so that no element count
// overflows 64 bits.  curand4 then returns the 4 words at counter
// (c0, c1, c2, c3).
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include <cstdint>

__global__ void k_ref(const uint4* ctr, size_t n, unsigned long long seed, uint4* out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = ctr[i];
    curandStatePhilox4_32_10_t st;
    const unsigned long long subseq = (unsigned long long)c.z | ((unsigned long long)c.w << 32);
    const unsigned long long block = (unsigned long long)c.x | ((unsigned long long)c.y << 32);
    curand_init(seed, subseq, 0ull, &st);
    for (int k = 0; k < 4; ++k) skipahead(4ull * (block >> 2), &st);
    skipahead(4ull * (block & 3ull), &st);
    out[i] = curand4(&st);
}

extern "C" int curand_philox_ref(const uint32_t* ctr, size_t n, unsigned long long seed, uint32_t* out)
{
    uint4 *dc = nullptr, *dout = nullptr;
    if (cudaMalloc(&dc, n * sizeof(uint4)) != cudaSuccess) return 1;
    if (cudaMalloc(&dout, n * sizeof(uint4)) != cudaSuccess) return 1;
    cudaMemcpy(dc, ctr, n * sizeof(uint4), cudaMemcpyHostToDevice);
    k_ref<<<(unsigned)((n + 255) / 256), 256>>>(dc, n, seed, dout);
    const cudaError_t e = cudaMemcpy(out, dout, n * sizeof(uint4), cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dout);
    return e == cudaSuccess ? 0 : 2;
}
