// Test helper: the product's device Box-Muller (sk::box_muller_x2, the
// transform every Gaussian sketch kernel applies to a Philox call) on caller
// words, so that a test can run it on every input it can ever see and
// compare with the oracle bit for bit.
#include <stdint.h>

#include "../../paper_2603_20966_gb300/csrc/sk_rng.cuh"

__global__ void k_box_muller_all(const uint4* words, float4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = sk::box_muller_x2(words[i]);
}

extern "C" int box_muller_all(const void* words_dev, void* out_dev, int n) {
  k_box_muller_all<<<(n + 255) / 256, 256>>>(static_cast<const uint4*>(words_dev),
                                             static_cast<float4*>(out_dev), n);
  if (cudaGetLastError() != cudaSuccess) return 1;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}
