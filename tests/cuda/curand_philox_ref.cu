// Test helper: raw Philox4x32-10 words from cuRAND's device API, used to pin
// the oracle's Philox at counters whose words 0, 1 and 3 are non-zero
// (cuRAND's host generator only reaches word 2).  curand_init(seed,
// subsequence, offset) starts the counter at (offset/4 lo, offset/4 hi,
// subsequence lo, subsequence hi) with key (seed lo, seed hi).
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_curand_words(unsigned long long seed, unsigned long long subseq0,
                               unsigned long long offset, uint4* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed, subseq0 + (unsigned long long)i, offset, &st);
  out[i] = curand4(&st);
}

extern "C" int curand_ref_words(unsigned long long seed, unsigned long long subseq0,
                                unsigned long long offset, void* out_dev, int n) {
  k_curand_words<<<(n + 127) / 128, 128>>>(seed, subseq0, offset, static_cast<uint4*>(out_dev), n);
  if (cudaGetLastError() != cudaSuccess) return 1;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}
