// curand_philox.cu -- test helper: Philox-4x32-10 words from cuRAND's device
// API, the library implementation the oracle's Philox is checked against.
//
// cuRAND's Philox state holds a 128-bit counter (x, y, z, w) and a 64-bit key:
// curand_init(seed, subsequence, offset) sets key = (seed lo, seed hi), adds
// subsequence to the counter's upper half (z, w) and offset / 4 to its lower
// half (x, y).  With offset = 4 g the first curand4() therefore returns the
// block of counter (g lo, g hi, c2, c3), which is the counter layout of the
// walks' draws.
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_curand_words(unsigned long long start, unsigned long long n, uint32_t c2, uint32_t c3,
                               unsigned long long key, uint4 *out) {
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    const unsigned long long g = start + i;
    curand_init(key, ((unsigned long long)c3 << 32) | c2, 4ull * g, &st);
    out[i] = curand4(&st);
}

extern "C" int curand_philox_words(unsigned long long start, unsigned long long n, uint32_t c2, uint32_t c3,
                                   unsigned long long key, void *out_dev) {
    if (n == 0) return 0;
    const unsigned long long blocks = (n + 255) / 256;
    k_curand_words<<<(unsigned)blocks, 256>>>(start, n, c2, c3, key, (uint4 *)out_dev);
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}
