// Base case of the recursion (Sec. 2.3): ranges of at most the leaf cutoff
// are sorted by transpose-free sorting networks (Sec. 3) and written, in
// input form, straight into the user's buffer.
//
//   - k_leaf_warp: one warp per range of <= 512 keys; each lane holds R keys
//     (R = 1..16, the smallest that fits), padded with the all-ones code,
//     which is the last value in sort order (Sec. 2.3 padding rule).
//   - k_leaf_mid: 128 threads per range of up to 2048 keys (16-byte keys:
//     1024), 8 or 16 keys per thread.
//   - k_leaf_block: cutoff/16 threads per range of up to the cutoff;
//     cross-warp merge steps exchange registers through shared memory, and
//     the sorted keys are staged in shared memory for coalesced stores.
//     Ranges flagged all-equal are only decoded and copied.
#include "launch.h"
#include "sortnet.cuh"

namespace vq {

namespace {

template <int KB> __device__ __forceinline__ typename KT<KB>::Code load_key(const void *b, uint64_t i) {
  if constexpr (KB == 2) return ((const uint16_t *)b)[i];
  else if constexpr (KB == 4) return ((const uint32_t *)b)[i];
  else if constexpr (KB == 8) return ((const uint64_t *)b)[i];
  else {
    const ulonglong2 v = ((const ulonglong2 *)b)[i];
    return typename KT<KB>::Code{v.x, v.y};
  }
}

// Key-only pairs (KV) tie on equal keys with different values, so the
// padding slots and the merge sentinels (all-ones and all-zero codes) must
// not tie with a real key: a leaf holding a key equal to 0 or 2^64 - 1 is
// sorted in the (key, value) order instead (the same bits read as a
// 128-bit code), which is one of the orders by key.
__device__ __forceinline__ bool edge_key(const KV &c) { return c.hi == 0 || c.hi == ~0ull; }
template <class C> __device__ __forceinline__ bool edge_key(const C &) { return false; }
template <int R> __device__ __forceinline__ void as_u128(const KV (&k)[R], U128 (&q)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) q[r] = U128{k[r].lo, k[r].hi};
}

// Compare-exchanges of the bitonic sorting network on P = G*R keys (G threads
// of R keys, P a power of two): P/2 per stage, L(L+1)/2 stages, L = log2 P.
template <int G, int R> __device__ __forceinline__ unsigned long long network_ce() {
  constexpr unsigned long long P = (unsigned long long)G * R;
  constexpr unsigned L = ilog2((unsigned)P);
  return P / 2 * L * (L + 1) / 2;
}

template <int KB, int R>
__device__ __forceinline__ void warp_leaf(const SortArgs &a, const void *src, uint64_t b, unsigned len, bool raw,
                                          unsigned lane) {
  using C = typename KT<KB>::Code;
  C k[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const unsigned j = r * 32 + lane;
    if (j < len) {
      C c = load_key<KB>(src, b + j);
      k[r] = raw ? encode<KB>(c, a.codec) : c;
    } else {
      k[r] = KT<KB>::max_code();
    }
  }
  if constexpr (KB == KV_KEYONLY) {
    bool edge = false;
#pragma unroll
    for (int r = 0; r < R; ++r) edge |= r * 32 + lane < len && edge_key(k[r]);
    if (__any_sync(0xFFFFFFFFu, edge)) {
      U128 q[R];
      as_u128<R>(k, q);
      warp_sort<U128, R>(q, lane);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const unsigned i = lane * R + r;
        if (i < len) store_key<16>(a.out, b + i, decode<16>(q[r], a.codec));
      }
      if (lane == 0) atomicAdd(&a.hdr->leaf_ce, network_ce<32, R>());
      return;
    }
  }
  warp_sort<C, R>(k, lane);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const unsigned i = lane * R + r;
    if (i < len) store_key<KB>(a.out, b + i, decode<KB>(k[r], a.codec));
  }
  if (lane == 0) atomicAdd(&a.hdr->leaf_ce, network_ce<32, R>());
}

template <int KB> __global__ void __launch_bounds__(256) k_leaf_warp(SortArgs a) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned long long n = a.hdr->n_leaf_warp;
  if (a.hdr->abort) return;
  for (;;) {
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(&a.hdr->cur_leaf_warp, 1ull);
    idx = __shfl_sync(0xFFFFFFFFu, idx, 0);
    if (idx >= n) break;
    const LeafEntry le = a.leaf_warp[idx];
    if (le.begin + le.len > a.n_total || le.len > WARP_LEAF_MAX) {   // guard
      if (lane == 0) guard_failed(a, GUARD_LEAF);
      continue;
    }
    const void *src = (le.flags & SEG_PARITY) ? a.alt : a.keys;
    const bool raw = le.flags & SEG_RAW;
    const unsigned len = le.len;
    if (len <= 32) warp_leaf<KB, 1>(a, src, le.begin, len, raw, lane);
    else if (len <= 64) warp_leaf<KB, 2>(a, src, le.begin, len, raw, lane);
    else if (len <= 128) warp_leaf<KB, 4>(a, src, le.begin, len, raw, lane);
    else if (len <= 256) warp_leaf<KB, 8>(a, src, le.begin, len, raw, lane);
    else warp_leaf<KB, 16>(a, src, le.begin, len, raw, lane);
  }
}

// Runs the register networks build before merge-path rounds take over. A
// bitonic phase joining runs of L keys costs log2(2L) steps of a shuffle and
// a compare-and-select per key; a merge round costs about twenty
// instructions per output key for 64-bit codes plus a binary search per
// thread (about a dozen probes, shared by its R keys). The phases stay in
// registers while they are the cheaper of the two: longest for 32-bit codes
// (one min or max instruction per exchange), shortest for 128-bit codes,
// and longer with fewer keys per thread (the search is shared by fewer).
template <int KB, int R> __host__ __device__ constexpr unsigned leaf_run0() {
  return KB <= 4 ? 256u : KB == 8 ? (R >= 16 ? 64u : 128u) : (R >= 8 ? 32u : 64u);
}

// The keys of one leaf in registers (ns slots on the first nta threads) are
// sorted by merge_sort_block, staged in shared memory and stored decoded,
// coalesced, at ob.
template <int KB, int R, int NT, unsigned L0>
__device__ __forceinline__ void sort_and_store(const SortArgs &a, typename KT<KB>::Code (&k)[R], unsigned t,
                                               unsigned len, unsigned ns, unsigned nta,
                                               typename KT<KB>::Code *sx, void *ob) {
  using C = typename KT<KB>::Code;
  merge_sort_block<C, R, NT, L0>(k, t, ns, sx);
  if (t < nta) {
#pragma unroll
    for (int r = 0; r < R; ++r) sx[spad<R>(t * R + r)] = k[r];
  }
  __syncthreads();
  const C *__restrict__ st = sx;
  if (KB != KV_KEYONLY && a.codec.kind == 0 && !a.codec.desc) {   // unsigned ascending: codes are the keys
#pragma unroll 4
    for (unsigned j = t; j < len; j += NT) store_key<KB>(ob, j, st[spad<R>(j)]);
  } else {
#pragma unroll 4
    for (unsigned j = t; j < len; j += NT) store_key<KB>(ob, j, decode<KB>(st[spad<R>(j)], a.codec));
  }
  if (t == 0) atomicAdd(&a.hdr->leaf_ce, merge_sort_cmps<R, NT, L0>(ns));
  __syncthreads();
}

// NT threads sort one range of len <= NT*R keys: the first ns/R threads load
// the keys (coalesced; ns = len rounded up to the register-stage run),
// padded with the all-ones code, the last value in sort order (Sec. 2.3);
// merge_sort_block sorts them; the result is staged in shared memory and
// stored decoded, coalesced.
template <int KB, int R, int NT>
__device__ __forceinline__ void block_leaf(const SortArgs &a, const void *src, uint64_t b, unsigned len, bool raw,
                                           typename KT<KB>::Code *sx) {
  using C = typename KT<KB>::Code;
  constexpr unsigned L0 = leaf_run0<KB, R>() < 32u * R ? leaf_run0<KB, R>() : 32u * R;
  const unsigned t = threadIdx.x;
  const unsigned ns = (len + L0 - 1) / L0 * L0;
  const unsigned nta = ns / R;
  C k[R];
  const void *sb = (const unsigned char *)src + b * kmem(KB);
  if (t < nta && !raw) {   // keys written by a partition level are codes already
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const unsigned j = r * nta + t;
      k[r] = j < len ? load_key<KB>(sb, j) : KT<KB>::max_code();
    }
  } else if (t < nta) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const unsigned j = r * nta + t;
      k[r] = j < len ? encode<KB>(load_key<KB>(sb, j), a.codec) : KT<KB>::max_code();
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) k[r] = KT<KB>::max_code();
  }
  void *ob = (unsigned char *)a.out + b * kmem(KB);
  if constexpr (KB == KV_KEYONLY) {
    bool edge = false;
#pragma unroll
    for (int r = 0; r < R; ++r) edge |= t < nta && r * nta + t < len && edge_key(k[r]);
    if (__syncthreads_or(edge)) {
      U128 q[R];
      as_u128<R>(k, q);
      sort_and_store<16, R, NT, L0>(a, q, t, len, ns, nta, (U128 *)sx, ob);
      return;
    }
  }
  sort_and_store<KB, R, NT, L0>(a, k, t, len, ns, nta, sx, ob);
}

// Starts pulling the keys of leaf `idx` (if it exists) from HBM into L2 with
// one bulk prefetch, so that its loads, issued after the current leaf is
// sorted, hit L2. The 16-byte aligned span around the keys stays within the
// memory pages of the array.
template <int KB>
__device__ __forceinline__ void prefetch_leaf_l2(const SortArgs &a, const LeafEntry *list, unsigned long long idx,
                                                 unsigned long long n) {
  if (idx >= n) return;
  const LeafEntry le = list[idx];
  if (le.len == 0 || le.begin + le.len > a.n_total) return;
  const uintptr_t src = (uintptr_t)((le.flags & SEG_PARITY) ? a.alt : a.keys);
  const uintptr_t g0 = (src + le.begin * kmem(KB)) & ~(uintptr_t)15;
  const uintptr_t g1 = (src + (le.begin + le.len) * kmem(KB) + 15) & ~(uintptr_t)15;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g0), "r"((unsigned)(g1 - g0)) : "memory");
}

// NT threads sort one range of up to RMAX*NT keys at a time.
template <int KB, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 && KB <= 8 ? 4 : NT <= 512 ? 2 : 1) k_leaf_block(SortArgs a) {
  constexpr int RMAX = leaf_rmax(KB, NT);
  using C = typename KT<KB>::Code;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_idx, s_next;
  C *sx = (C *)smem;
  const unsigned long long n = a.hdr->n_leaf_block;
  if (a.hdr->abort) return;
  if (threadIdx.x == 0) s_idx = atomicAdd(&a.hdr->cur_leaf_block, 1ull);
  __syncthreads();
  unsigned long long idx = s_idx;
  while (idx < n) {
    if (threadIdx.x == 0) {
      const unsigned long long nx = atomicAdd(&a.hdr->cur_leaf_block, 1ull);
      s_next = nx;
      prefetch_leaf_l2<KB>(a, a.leaf_block, nx, n);
    }
    const LeafEntry le = a.leaf_block[idx];
    // guard: inside the array, and no longer than the cutoff the shared
    // memory was sized for
    if (le.begin + le.len > a.n_total || le.len > (unsigned)(RMAX * NT) ||
        le.len > (a.leaf_cutoff < 1024 ? 1024u : a.leaf_cutoff)) {
      if (threadIdx.x == 0) guard_failed(a, GUARD_LEAF);
    } else {
      const void *src = (le.flags & SEG_PARITY) ? a.alt : a.keys;
      const bool raw = le.flags & SEG_RAW;
      const unsigned len = le.len;
      if (le.flags & LEAF_COPY) {
        for (unsigned j = threadIdx.x; j < len; j += NT) {
          const C c = load_key<KB>(src, le.begin + j);
          store_key<KB>(a.out, le.begin + j, decode<KB>(raw ? encode<KB>(c, a.codec) : c, a.codec));
        }
      } else {
        switch (leaf_r_for(len, NT, RMAX)) {
          case 4: block_leaf<KB, 4, NT>(a, src, le.begin, len, raw, sx); break;
          case 8: block_leaf<KB, (RMAX < 8 ? RMAX : 8), NT>(a, src, le.begin, len, raw, sx); break;
          default: block_leaf<KB, RMAX, NT>(a, src, le.begin, len, raw, sx); break;
        }
      }
    }
    __syncthreads();
    idx = s_next;
    __syncthreads();
  }
}

// Mid-size leaves: one MID_NT-thread block per range of (WARP_LEAF_MAX,
// mid_max_keys(KB)] keys, 16 keys per thread (16-byte keys: 8).
template <int KB> __global__ void __launch_bounds__(MID_NT, kmem(KB) == 16 ? 4 : 8) k_leaf_mid(SortArgs a) {
  using C = typename KT<KB>::Code;
  constexpr unsigned MAXK = mid_max_keys(KB);
  __shared__ C sx[MAXK + MAXK / 8];
  __shared__ unsigned long long s_idx, s_next;
  const unsigned long long n = a.hdr->n_leaf_mid;
  if (a.hdr->abort) return;
  if (threadIdx.x == 0) s_idx = atomicAdd(&a.hdr->cur_leaf_mid, 1ull);
  __syncthreads();
  unsigned long long idx = s_idx;
  while (idx < n) {
    if (threadIdx.x == 0) {
      const unsigned long long nx = atomicAdd(&a.hdr->cur_leaf_mid, 1ull);
      s_next = nx;
      prefetch_leaf_l2<KB>(a, a.leaf_mid, nx, n);
    }
    const LeafEntry le = a.leaf_mid[idx];
    if (le.begin + le.len > a.n_total || le.len > MAXK) {   // guard
      if (threadIdx.x == 0) guard_failed(a, GUARD_LEAF);
    } else {
      const void *src = (le.flags & SEG_PARITY) ? a.alt : a.keys;
      const bool raw = le.flags & SEG_RAW;
      const unsigned len = le.len;
      // one register count per key size: a second instantiation of the
      // sort doubled the code the instruction cache has to hold
      block_leaf<KB, (kmem(KB) == 16 ? 8 : 16), MID_NT>(a, src, le.begin, len, raw, sx);
    }
    __syncthreads();
    idx = s_next;
    __syncthreads();
  }
}

template <int KB> int leaf_mid_grid() {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_leaf_mid<KB>, MID_NT, 0);
    grid = sms * (per > 0 ? per : 1);
  }
  return grid;
}

template <int KB, int NT> int leaf_block_grid(size_t smem) {
  static int grid = 0;
  static size_t last = 0;
  if (!grid || last != smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_leaf_block<KB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)leaf_block_smem(KB, max_leaf_cutoff(KB), NT));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_leaf_block<KB, NT>, NT, smem);
    grid = sms * (per > 0 ? per : 1);
    last = smem;
  }
  return grid;
}

template <int KB> int leaf_warp_grid() {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_leaf_warp<KB>, 256, 0);
    grid = sms * (per > 0 ? per : 1);
  }
  return grid;
}

template <int KB> cudaError_t leaf_block_impl(const SortArgs &a, cudaStream_t s) {
  const unsigned C = a.leaf_cutoff < 1024 ? 1024 : a.leaf_cutoff;
  if constexpr (kmem(KB) == 16) {   // cutoff <= 4096: at most 8 keys per thread at 512 threads
    if (a.leaf_threads == 256) {
      const size_t smem = leaf_block_smem(KB, C, 256);
      k_leaf_block<KB, 256><<<leaf_block_grid<KB, 256>(smem), 256, smem, s>>>(a);
    } else {
      const size_t smem = leaf_block_smem(KB, C, 512);
      k_leaf_block<KB, 512><<<leaf_block_grid<KB, 512>(smem), 512, smem, s>>>(a);
    }
  } else {
    const int nt = leaf_nt_for(C, a.leaf_threads);
    const size_t smem = leaf_block_smem(KB, C, nt);
    switch (nt) {
      case 1024: k_leaf_block<KB, 1024><<<leaf_block_grid<KB, 1024>(smem), 1024, smem, s>>>(a); break;
      case 512: k_leaf_block<KB, 512><<<leaf_block_grid<KB, 512>(smem), 512, smem, s>>>(a); break;
      default: k_leaf_block<KB, 256><<<leaf_block_grid<KB, 256>(smem), 256, smem, s>>>(a); break;
    }
  }
  return cudaGetLastError();
}

template <int KB> cudaError_t leaf_mid_impl(const SortArgs &a, cudaStream_t s) {
  k_leaf_mid<KB><<<leaf_mid_grid<KB>(), MID_NT, 0, s>>>(a);
  return cudaGetLastError();
}

template <int KB> cudaError_t leaf_warp_impl(const SortArgs &a, cudaStream_t s) {
  k_leaf_warp<KB><<<leaf_warp_grid<KB>(), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_leaf_warp(int kb, const SortArgs &a, cudaStream_t s) {
  switch (kb) {
    case 2: return leaf_warp_impl<2>(a, s);
    case 4: return leaf_warp_impl<4>(a, s);
    case 8: return leaf_warp_impl<8>(a, s);
    case 16: return leaf_warp_impl<16>(a, s);
    case KV_KEYONLY: return leaf_warp_impl<KV_KEYONLY>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_leaf_mid(int kb, const SortArgs &a, cudaStream_t s) {
  switch (kb) {
    case 2: return leaf_mid_impl<2>(a, s);
    case 4: return leaf_mid_impl<4>(a, s);
    case 8: return leaf_mid_impl<8>(a, s);
    case 16: return leaf_mid_impl<16>(a, s);
    case KV_KEYONLY: return leaf_mid_impl<KV_KEYONLY>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_leaf_block(int kb, const SortArgs &a, cudaStream_t s) {
  switch (kb) {
    case 2: return leaf_block_impl<2>(a, s);
    case 4: return leaf_block_impl<4>(a, s);
    case 8: return leaf_block_impl<8>(a, s);
    case 16: return leaf_block_impl<16>(a, s);
    case KV_KEYONLY: return leaf_block_impl<KV_KEYONLY>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace vq
