// Integer throughput probe: a measurement helper that gives the leaf
// networks' instruction counts a measured denominator. The paper has no
// counterpart. Each thread keeps eight independent registers and updates
// each of them `iters` times, so the loop is bound by instruction issue and
// the integer pipes, not by latency or memory.
//
//   kind 0: x = min(x, y_j) ^ i        (32-bit: one min, one xor)
//   kind 1: x = (y_j < x ? y_j : x) ^ i (64-bit: the compare-and-select a
//                                        64-bit code's minimum takes, then
//                                        an xor of both words)
//
// One word per thread goes to d_sink so nothing is optimised away.
#include "../../include/vqsort.h"

#include <cuda_runtime.h>
#include <cstdint>

namespace {

constexpr unsigned PROBE_NT = 256;

__global__ void __launch_bounds__(PROBE_NT) k_probe_min32(unsigned iters, uint32_t seed, uint32_t *sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[8], y[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    x[j] = (t * 0x9E3779B9u) ^ (seed + j);
    y[j] = (t + 0x7F4A7C15u * (j + 1)) ^ seed;
  }
  for (unsigned i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = min(x[j], y[j]) ^ i;
  }
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) r ^= x[j];
  sink[t] = r;
}

__global__ void __launch_bounds__(PROBE_NT) k_probe_min64(unsigned iters, uint32_t seed, uint32_t *sink) {
  const uint64_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t x[8], y[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    x[j] = (t * 0x9E3779B97F4A7C15ull) ^ (seed + (uint64_t)j);
    y[j] = (t + 0xBF58476D1CE4E5B9ull * (j + 1)) ^ ((uint64_t)seed << 32);
  }
  for (unsigned i = 0; i < iters; ++i) {
    const uint64_t m = ((uint64_t)i << 32) | i;
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (y[j] < x[j] ? y[j] : x[j]) ^ m;
  }
  uint64_t r = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) r ^= x[j];
  sink[t] = (uint32_t)(r ^ (r >> 32));
}

}  // namespace

extern "C" vq_status vqsort_probe_int_throughput(int kind, unsigned blocks, unsigned iters, void *d_sink,
                                                 uint64_t *ops_per_thread, void *stream) {
  if ((kind != 0 && kind != 1) || blocks == 0 || !d_sink || !ops_per_thread) return VQ_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == 0) {
    k_probe_min32<<<blocks, PROBE_NT, 0, s>>>(iters, 0x22050598u, (uint32_t *)d_sink);
    *ops_per_thread = 2ull * 8 * iters;
  } else {
    k_probe_min64<<<blocks, PROBE_NT, 0, s>>>(iters, 0x22050598u, (uint32_t *)d_sink);
    *ops_per_thread = 6ull * 8 * iters;
  }
  return cudaGetLastError() == cudaSuccess ? VQ_OK : VQ_ERR_CUDA;
}
