// Depth-bound fallback (Sec. 2.2): a range that is still unsorted after
// 2*floor(log2 n)+4 partition levels is finished here with O(m log m) work.
// The paper switches to Heapsort, which is sequential; the GPU form is a
// merge sort: chunks of 2048 keys are sorted by the block network, then
// merge passes double the run length, each output element placed by a
// merge-path binary search. Passes are separated by a grid barrier, so the
// kernel is launched cooperatively; every barrier wait is bounded.
#include "launch.h"
#include "sortnet.cuh"

namespace vq {

namespace {

constexpr unsigned ERR_TIMEOUT = 5;

__device__ bool grid_sync(const SortArgs &a) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long gen = ld_acquire(&a.hdr->bar_gen);
    const unsigned long long arrived = atomicAdd(&a.hdr->bar_count, 1ull) + 1;
    int ok = 1;
    if (arrived == gridDim.x) {
      atomicExch(&a.hdr->bar_count, 0ull);
      st_release(&a.hdr->bar_gen, gen + 1);
    } else {
      for (unsigned it = 0; ld_acquire(&a.hdr->bar_gen) == gen; ++it) {
        if (aborted(a)) { ok = 0; break; }
        if (it >= a.spin_limit) {
          raise_error(a, ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int KB> __device__ __forceinline__ const void *buf_of(const SortArgs &a, unsigned parity) {
  return parity ? a.alt : a.keys;
}

template <int KB> __global__ void __launch_bounds__(FB_NT) k_fallback(SortArgs a) {
  using C = typename KT<KB>::Code;
  __shared__ C sx[FB_CHUNK];
  const unsigned long long nfb = a.hdr->n_fb;
  if (nfb == 0 || a.hdr->abort) return;
  const unsigned tid = threadIdx.x;
  for (unsigned long long f = 0; f < nfb; ++f) {
    const LeafEntry le = a.fb[f];
    const uint64_t b = le.begin, len = le.len;
    if (b + len > a.n_total) {   // guard (uniform across the grid)
      if (blockIdx.x == 0 && threadIdx.x == 0) guard_failed(a, GUARD_LEAF);
      return;
    }
    const unsigned par = le.flags & SEG_PARITY;
    const bool raw = le.flags & SEG_RAW;
    void *bufA = (void *)buf_of<KB>(a, par), *bufB = (void *)buf_of<KB>(a, par ^ 1u);

    // chunk sort: bufA -> bufB
    const uint64_t nch = (len + FB_CHUNK - 1) / FB_CHUNK;
    for (uint64_t c = blockIdx.x; c < nch; c += gridDim.x) {
      const uint64_t cb = b + c * FB_CHUNK;
      const unsigned clen = (unsigned)min((uint64_t)FB_CHUNK, b + len - cb);
      C k[FB_R];
#pragma unroll
      for (int r = 0; r < FB_R; ++r) {
        const unsigned j = r * FB_NT + tid;
        if (j < clen) {
          const C v = load_cg<KB>(bufA, cb + j);
          k[r] = raw ? encode<KB>(v, a.codec) : v;
        } else {
          k[r] = KT<KB>::max_code();
        }
      }
      group_sort<C, FB_R, FB_NT>(k, tid, sx);
#pragma unroll
      for (int r = 0; r < FB_R; ++r) {
        const unsigned i = tid * FB_R + r;
        if (i < clen) store_key<KB>(bufB, cb + i, k[r]);
      }
      __syncthreads();
    }
    if (!grid_sync(a)) return;

    // merge passes
    void *cur = bufB, *nxt = bufA;
    for (uint64_t w = FB_CHUNK; w < len; w *= 2) {
      for (uint64_t o = blockIdx.x; o * FB_CHUNK < len; o += gridDim.x) {
        const uint64_t ob = o * FB_CHUNK;
        const uint64_t pb = (ob / (2 * w)) * (2 * w);           // pair start (range-relative)
        const uint64_t la = min(w, len - pb);
        const uint64_t lb = min(w, len - pb - la);
        const uint64_t k0 = ob - pb + (uint64_t)tid * FB_R;      // diagonal of this thread
        if (k0 >= la + lb) continue;
        const unsigned cnt = (unsigned)min((uint64_t)FB_R, la + lb - k0);
        const uint64_t A0 = b + pb, B0 = b + pb + la;
        uint64_t lo = k0 > lb ? k0 - lb : 0, hi = min(k0, la);
        while (lo < hi) {
          const uint64_t mid = (lo + hi) / 2;
          // A[mid] <= B[k0-1-mid]: the split is after mid (ties take A first)
          if (!lt(load_cg<KB>(cur, B0 + (k0 - 1 - mid)), load_cg<KB>(cur, A0 + mid))) lo = mid + 1;
          else hi = mid;
        }
        uint64_t ia = lo, ib = k0 - lo;
        for (unsigned q = 0; q < cnt; ++q) {
          C out;
          if (ib >= lb) {
            out = load_cg<KB>(cur, A0 + ia++);
          } else if (ia >= la) {
            out = load_cg<KB>(cur, B0 + ib++);
          } else {
            const C x = load_cg<KB>(cur, A0 + ia), y = load_cg<KB>(cur, B0 + ib);
            if (!lt(y, x)) { out = x; ++ia; } else { out = y; ++ib; }
          }
          store_key<KB>(nxt, b + pb + k0 + q, out);
        }
      }
      if (!grid_sync(a)) return;
      void *t = cur;
      cur = nxt;
      nxt = t;
    }

    // decode into the user's buffer
    const uint64_t gt = (uint64_t)blockIdx.x * FB_NT + tid, stride = (uint64_t)gridDim.x * FB_NT;
    for (uint64_t j = gt; j < len; j += stride)
      store_key<KB>(a.out, b + j, decode<KB>(load_cg<KB>(cur, b + j), a.codec));
    if (!grid_sync(a)) return;
  }
}

template <int KB> cudaError_t fallback_impl(const SortArgs &a, cudaStream_t s) {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fallback<KB>, FB_NT, 0);
    grid = sms * (per > 0 ? per : 1);
    if (grid > 64) grid = 64;   // few blocks: cheap to co-schedule, the path is rare
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(FB_NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fallback<KB>, a);
}

}  // namespace

cudaError_t launch_fallback(int kb, const SortArgs &a, cudaStream_t s) {
  switch (kb) {
    case 2: return fallback_impl<2>(a, s);
    case 4: return fallback_impl<4>(a, s);
    case 8: return fallback_impl<8>(a, s);
    case 16: return fallback_impl<16>(a, s);
    // key-only pairs: the merge sort pads with the all-ones code, which ties
    // with a real key of all ones; it sorts them in the (key, value) order,
    // one of the orders by key (same bits, same codec)
    case KV_KEYONLY: return fallback_impl<16>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace vq
