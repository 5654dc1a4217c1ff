// One Partition that allocates nothing.
//
// Some callers cannot call cudaMalloc at the moment they need a partition:
// cudaMalloc may synchronize the device and can fail under a fixed memory
// budget, which a latency-critical serving loop or code running inside
// another allocator's hooks cannot afford. vqsort_partition gets its
// scratch (counters, the range descriptor and the tile queue) from a
// library-owned allocation made on first use; this variant instead uses a
// fixed array in device memory that is part of the loaded library, so no
// call to an allocator is ever made.
//
// The array holds up to NOALLOC_TILES partition tiles, so one call accepts
// at most NOALLOC_TILES * ((32768 - 16) / key_bytes) keys. Every GPU that
// loads the library keeps the array (528,896 bytes, about 517 KiB) until the
// process exits.
#include <cstring>
#include <mutex>

#include "launch.h"
#include "../../include/vqsort.h"

using namespace vq;

namespace {

constexpr unsigned NOALLOC_TILES = 65536;
constexpr size_t NOALLOC_HDR = 512;                          // Header, rounded up to 256 bytes
constexpr size_t NOALLOC_SEGS = 64 * sizeof(SegDesc);        // the one range (room to spare)
constexpr size_t NOALLOC_BYTES = NOALLOC_HDR + NOALLOC_SEGS + (size_t)NOALLOC_TILES * 8;
static_assert(sizeof(Header) <= NOALLOC_HDR, "header does not fit");
static_assert(NOALLOC_BYTES == 528896, "the size stated above and in the header");

// The scratch shared by every call in the process. Host code must not use
// this name as an address: it is a host-side stand-in. The device address
// comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {};

vq_status noalloc_scratch(void **ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VQ_ERR_CUDA;
  if (dev < 0 || dev >= 64) return VQ_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return VQ_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *ptr = g_noalloc_ptr[dev];
  return VQ_OK;
}

int kbytes(vq_dtype dt) {
  switch (dt) {
    case VQ_I16: case VQ_U16: return 2;
    case VQ_I32: case VQ_U32: case VQ_F32: return 4;
    case VQ_I64: case VQ_U64: case VQ_F64: return 8;
    case VQ_U128: case VQ_KV64: return 16;
  }
  return 0;
}

Codec codec_for(vq_dtype dt, int ascending) {
  Codec c;
  c.desc = ascending ? 0 : 1;
  c.kind = (dt == VQ_I16 || dt == VQ_I32 || dt == VQ_I64) ? 1
           : (dt == VQ_F32 || dt == VQ_F64) ? 2
           : dt == VQ_KV64 ? 3 : 0;
  return c;
}

}  // namespace

extern "C" vq_status vqsort_partition_noalloc(vq_dtype dt, const void *d_in, void *d_out, size_t n,
                                              const void *h_pivot, int ascending, uint64_t *d_left_count,
                                              void *stream) {
  const int kb = kbytes(dt);
  if (!kb || !h_pivot || !d_left_count) return VQ_ERR_INVALID;
  if (n > 0 && (!d_in || !d_out || d_in == d_out)) return VQ_ERR_INVALID;
  if ((uintptr_t)d_in % kb || (uintptr_t)d_out % kb) return VQ_ERR_INVALID;
  const unsigned long long T = part_tile_keys(kb);
  if (n > (unsigned long long)NOALLOC_TILES * T) return VQ_ERR_INVALID;   // beyond the fixed scratch
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
    return VQ_ERR_CUDA;
  if (major != 10 || minor != 3) return VQ_ERR_UNSUPPORTED;
  void *scratch = nullptr;
  vq_status st = noalloc_scratch(&scratch);
  if (st != VQ_OK) return st;
  unsigned char *w = (unsigned char *)scratch;

  SortArgs a{};
  a.keys = const_cast<void *>(d_in);
  a.alt = d_out;
  a.hdr = (Header *)w;
  a.segs = (SegDesc *)(w + NOALLOC_HDR);
  a.items = (unsigned long long *)(w + NOALLOC_HDR + NOALLOC_SEGS);
  a.leaf_warp = a.leaf_block = a.fb = nullptr;   // a partition hands nothing to the leaf kernels
  a.offsets = nullptr;
  a.n_total = n;
  a.num_segments = 1;
  a.out_left = (unsigned long long *)d_left_count;
  a.cap_q = NOALLOC_TILES;
  a.cap_segs = 64;
  a.tile_keys = (unsigned)T;
  a.tile_cpt = PART_CPT;
  a.leaf_cutoff = default_leaf_cutoff(kb);
  a.depth_override = -1;
  a.spin_limit = 1u << 22;
  a.mode = MODE_PARTITION;
  a.codec = codec_for(dt, ascending);
  a.pivot = U128{0, 0};
  switch (kb) {
    case 2: { uint16_t v; memcpy(&v, h_pivot, 2); a.pivot.lo = encode<2>(v, a.codec); break; }
    case 4: { uint32_t v; memcpy(&v, h_pivot, 4); a.pivot.lo = encode<4>(v, a.codec); break; }
    case 8: { uint64_t v; memcpy(&v, h_pivot, 8); a.pivot.lo = encode<8>(v, a.codec); break; }
    case 16: { U128 v; memcpy(&v, h_pivot, 16); a.pivot = encode<16>(v, a.codec); break; }
  }
  // The prep kernel clears the counters and the tile queue of the shared
  // scratch, so a call never sees the previous call's state.
  cudaStream_t s = (cudaStream_t)stream;
  if (launch_prep(a, s) != cudaSuccess) return VQ_ERR_CUDA;
  if (launch_seed(kb, a, s) != cudaSuccess) return VQ_ERR_CUDA;
  if (launch_partition(kb, a, s) != cudaSuccess) return VQ_ERR_CUDA;
  return VQ_OK;
}
