// Transpose-free sorting networks in registers (Sec. 3 of the paper).
//
// A group of threads sorts G*R keys: thread t holds the "column" of R keys
// k[0..R) in registers, the keys' logical index is t*R + r. First every
// column is sorted by a small optimal network (networks.h), applied to all
// columns at once. Then sorted runs are joined by bitonic merges whose
// modules are brought into vertical alignment by exchanging whole
// registers between threads (warp shuffles inside a warp, shared memory
// across warps) or by pairing registers inside a thread; the key matrix is
// never transposed.
#pragma once

#include "common.cuh"
#include "networks.h"

namespace vq {

template <class C, int R> __device__ __forceinline__ void column_sort(C (&k)[R]) {
#define VQ_CE(a, b) cas(k[a], k[b]);
  if constexpr (R == 2) { VQ_NET2(VQ_CE) }
  if constexpr (R == 4) { VQ_NET4(VQ_CE) }
  if constexpr (R == 8) { VQ_NET8(VQ_CE) }
  if constexpr (R == 16) { VQ_NET16(VQ_CE) }
#undef VQ_CE
}

// One side of a compare-exchange whose partner lives in another thread: the
// lower position keeps the minimum, the upper one the maximum. Equal codes
// are identical bit patterns, so either choice is right on ties.
__device__ __forceinline__ uint32_t keep(uint32_t mine, uint32_t other, bool lower) {
  const uint32_t mn = umin(mine, other), mx = umax(mine, other);
  return lower ? mn : mx;
}
template <class C> __device__ __forceinline__ C keep(const C &mine, const C &other, bool lower) {
  const bool take = lt(other, mine) != !lower;
  return take ? other : mine;
}

// One merge step. `t` is the thread's index in the sorting group; steps whose
// partner thread is in another warp go through `sx` (R*NT codes, layout
// [register][thread]) and need the whole group (NT threads) at the barrier.
template <class C, int R, int NT>
__device__ __forceinline__ void merge_step(C (&k)[R], const VqMergeStep &m, unsigned t, C *sx) {
  if (m.lane_xor == 0) {
#pragma unroll
    for (int r = 0; r < R; ++r)
      if ((r & m.reg_xor) == 0) cas(k[r], k[r ^ m.reg_xor]);
    return;
  }
  const bool lower = (t & m.lower_bit) == 0;
  if (m.lane_xor < 32) {
    if (m.reverse) {
#pragma unroll
      for (int r = 0; r < (R + 1) / 2; ++r) {
        C o1 = shfl_xor(k[R - 1 - r], (int)m.lane_xor);
        C o2 = shfl_xor(k[r], (int)m.lane_xor);
        k[r] = keep(k[r], o1, lower);
        if (R - 1 - r != r) k[R - 1 - r] = keep(k[R - 1 - r], o2, lower);
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) k[r] = keep(k[r], shfl_xor(k[r], (int)m.lane_xor), lower);
    }
    return;
  }
  // partner thread in another warp: exchange through shared memory
#pragma unroll
  for (int r = 0; r < R; ++r) sx[r * NT + t] = k[r];
  __syncthreads();
  const unsigned pt = t ^ m.lane_xor;
#pragma unroll
  for (int r = 0; r < R; ++r) k[r] = keep(k[r], sx[(m.reverse ? R - 1 - r : r) * NT + pt], lower);
  __syncthreads();
}

__host__ __device__ constexpr unsigned ilog2(unsigned x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// Merge phase joining sorted runs of L keys into runs of 2L, then the next
// phase. Fully unrolled so every step's lane mask and register pairing are
// compile-time constants and the keys stay in registers.
template <class C, int R, int NT, unsigned L>
__device__ __forceinline__ void merge_phases(C (&k)[R], unsigned t, C *sx) {
  constexpr unsigned steps = ilog2(L) + 1;
#pragma unroll
  for (unsigned s = 0; s < steps; ++s) merge_step<C, R, NT>(k, vq_merge_step(L, R, s), t, sx);
  if constexpr (2 * L < (unsigned)(NT * R)) merge_phases<C, R, NT, 2 * L>(k, t, sx);
}

// Sorts NT*R keys held by NT threads (NT = 32: one warp, no shared memory).
// The result: thread t holds the keys of logical indices t*R .. t*R+R-1.
template <class C, int R, int NT>
__device__ __forceinline__ void group_sort(C (&k)[R], unsigned t, C *sx) {
  if constexpr (R > 1) column_sort<C, R>(k);
  if constexpr (NT * R > R) merge_phases<C, R, NT, (unsigned)R>(k, t, sx);
}

// Warp-only variant with fully unrolled loops (NT = 32).
template <class C, int R> __device__ __forceinline__ void warp_sort(C (&k)[R], unsigned lane) {
  group_sort<C, R, 32>(k, lane, nullptr);
}

}  // namespace vq
