// Stable sort by an appended row id (Sec. 5: a unique row identifier in the
// least significant bits of the key makes Quicksort stable). Each key's
// order-preserving code is packed with its input position below it: keys of
// up to 4 bytes as one 64-bit code (code << 32 | row; n < 2^32), 8-byte keys
// as a 128-bit code {low = row, high = code}. Equal keys then differ only in
// their rows, so the ordinary ascending sort of the packed codes puts them in
// input order; unpacking writes the keys back and the rows out. Descending
// order complements the key code only, never the row.
#include "launch.h"

namespace vq {

namespace {

constexpr int STABLE_NT = 256;

template <int KB>
__global__ void __launch_bounds__(STABLE_NT) k_stable_pack(const void *keys, void *packed, uint64_t n, Codec cd) {
  const uint64_t stride = (uint64_t)gridDim.x * STABLE_NT;
  for (uint64_t i = (uint64_t)blockIdx.x * STABLE_NT + threadIdx.x; i < n; i += stride) {
    const auto c = encode<KB>(load_cg<KB>(keys, i), cd);
    if constexpr (KB == 8) ((U128 *)packed)[i] = U128{i, (uint64_t)c};
    else ((uint64_t *)packed)[i] = ((uint64_t)c << 32) | i;
  }
}

template <int KB>
__global__ void __launch_bounds__(STABLE_NT) k_stable_unpack(const void *packed, void *keys, uint64_t *rows,
                                                             uint64_t n, Codec cd) {
  using C = typename KT<KB>::Code;
  const uint64_t stride = (uint64_t)gridDim.x * STABLE_NT;
  for (uint64_t i = (uint64_t)blockIdx.x * STABLE_NT + threadIdx.x; i < n; i += stride) {
    C c;
    uint64_t row;
    if constexpr (KB == 8) {
      const U128 p = ((const U128 *)packed)[i];
      c = p.hi;
      row = p.lo;
    } else {
      const uint64_t p = ((const uint64_t *)packed)[i];
      c = (C)(p >> 32);
      row = p & 0xFFFFFFFFull;
    }
    store_key<KB>(keys, i, decode<KB>(c, cd));
    rows[i] = row;
  }
}

unsigned stable_grid(uint64_t n) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const uint64_t want = (n + STABLE_NT - 1) / STABLE_NT, cap = (uint64_t)sms * 8;
  return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_stable_pack(int kb, const void *keys, void *packed, uint64_t n, Codec cd, cudaStream_t s) {
  const unsigned g = stable_grid(n);
  switch (kb) {
    case 2: k_stable_pack<2><<<g, STABLE_NT, 0, s>>>(keys, packed, n, cd); break;
    case 4: k_stable_pack<4><<<g, STABLE_NT, 0, s>>>(keys, packed, n, cd); break;
    case 8: k_stable_pack<8><<<g, STABLE_NT, 0, s>>>(keys, packed, n, cd); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_stable_unpack(int kb, const void *packed, void *keys, uint64_t *rows, uint64_t n, Codec cd,
                                 cudaStream_t s) {
  const unsigned g = stable_grid(n);
  switch (kb) {
    case 2: k_stable_unpack<2><<<g, STABLE_NT, 0, s>>>(packed, keys, rows, n, cd); break;
    case 4: k_stable_unpack<4><<<g, STABLE_NT, 0, s>>>(packed, keys, rows, n, cd); break;
    case 8: k_stable_unpack<8><<<g, STABLE_NT, 0, s>>>(packed, keys, rows, n, cd); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace vq
