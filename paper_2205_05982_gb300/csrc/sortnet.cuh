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
// Key-only pairs tie on equal keys with different values: on a tie both
// partners keep their own pair, so no pair is lost or duplicated.
__device__ __forceinline__ KV keep(const KV &mine, const KV &other, bool lower) {
  const uint64_t x = lower ? other.hi : mine.hi, y = lower ? mine.hi : other.hi;
  return x < y ? other : mine;
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

// ---------------------------------------------------------------------------
// Block sorts for leaves of more than a few hundred keys: the register
// networks above build sorted runs of L0 keys inside each warp, then
// merge-path merges in shared memory join runs pairwise (L0 -> 2 L0 -> ...).
// A bitonic merge of two runs of L keys costs log2(2L) compare-exchange
// steps per key; a merge-path merge costs one comparison per key plus a
// binary search per thread, so past a few dozen keys per run merging is the
// cheaper way to finish the base case. Runs need not be powers of two: only
// the slots up to the leaf length rounded up to L0 take part.
// ---------------------------------------------------------------------------

// Shared-memory slot of logical index i: one spare slot per R keys, so that
// the R keys of consecutive threads (stride R + 1) fall in distinct banks.
template <int R> __device__ __forceinline__ unsigned spad(unsigned i) { return i + i / (unsigned)R; }

// A code above or equal to every code of the key type: read past the end of
// a run, so the other run's keys are taken first.
template <class C> __device__ __forceinline__ C ones_code();
template <> __device__ __forceinline__ uint32_t ones_code<uint32_t>() { return ~0u; }
template <> __device__ __forceinline__ uint64_t ones_code<uint64_t>() { return ~0ull; }
template <> __device__ __forceinline__ U128 ones_code<U128>() { return U128{~0ull, ~0ull}; }
template <> __device__ __forceinline__ KV ones_code<KV>() { return KV{~0ull, ~0ull}; }

// Bitonic phases joining runs of L keys up to runs of LEND keys; a run of
// LEND keys spans LEND/R <= 32 lanes, so every step is a register pairing
// or a shuffle.
//
// The phases run as a loop over three step bodies, not unrolled per phase
// (which multiplied the code and made the leaves wait on the instruction
// cache): a phase joining runs of L keys is one mirrored exchange with the
// lane 2L/R - 1 away (register r against R - 1 - r), exchanges with the
// lanes L/(2R), ..., 1 away, and the log2(R) steps inside each thread's
// registers (vq_merge_step gives the same schedule).
template <class C, int R, unsigned L, unsigned LEND>
__device__ __forceinline__ void warp_phases(C (&k)[R], unsigned lane) {
#pragma unroll 1
  for (unsigned l = L; l < LEND; l *= 2) {
    {   // step 0: mirrored partner, lower half of each 2l block keeps the minimum
      const unsigned lx = 2 * l / R - 1;
      const bool lower = (lane & (l / R)) == 0;
#pragma unroll
      for (int r = 0; r < (R + 1) / 2; ++r) {
        const C o1 = shfl_xor(k[R - 1 - r], (int)lx);
        const C o2 = shfl_xor(k[r], (int)lx);
        k[r] = keep(k[r], o1, lower);
        if (R - 1 - r != r) k[R - 1 - r] = keep(k[R - 1 - r], o2, lower);
      }
    }
#pragma unroll 1
    for (unsigned d = l / 2; d >= (unsigned)R; d /= 2) {   // partners d/R lanes away
      const unsigned lx = d / R;
      const bool lower = (lane & lx) == 0;
#pragma unroll
      for (int r = 0; r < R; ++r) k[r] = keep(k[r], shfl_xor(k[r], (int)lx), lower);
    }
#pragma unroll
    for (int dr = R / 2; dr >= 1; dr /= 2) {   // partners inside the thread
#pragma unroll
      for (int r = 0; r < R; ++r)
        if ((r & dr) == 0) cas(k[r], k[r ^ dr]);
    }
  }
}

// A code below or equal to every code: read before the start of a run.
template <class C> __device__ __forceinline__ C zero_code();
template <> __device__ __forceinline__ uint32_t zero_code<uint32_t>() { return 0u; }
template <> __device__ __forceinline__ uint64_t zero_code<uint64_t>() { return 0ull; }
template <> __device__ __forceinline__ U128 zero_code<U128>() { return U128{0ull, 0ull}; }
template <> __device__ __forceinline__ KV zero_code<KV>() { return KV{0ull, 0ull}; }

// One merge-path round: the ns slots form sorted runs of L keys; afterwards
// they form sorted runs of 2L. Thread t holds logical slots t*R .. t*R+R-1
// before and after. A pair whose second run is empty is already merged.
//
// Each thread finds where its first output splits the two runs (binary
// search, ties: the first run's key first) and takes the split of its last
// output + 1 from the next thread (a shuffle, or shared memory across
// warps). It then fills its R outputs with two independent chains, one
// taking the smaller head from the front, one the larger tail from the
// back, R/2 steps each: the front chain yields the R/2 smallest keys after
// the first split, the back chain the R/2 largest before the last one, and
// the two chains overlap their shared-memory latencies. Reads past a run's
// end (front) or before its start (back) give a code no key passes; where a
// key equals it, the bits are the same either way. Rounds of runs within one
// warp synchronise the warp only.
template <class C, int R, int NT, bool WARP>
__device__ __forceinline__ void mp_round(C (&k)[R], unsigned t, unsigned ns, C *sx, const unsigned L) {
  constexpr int H = R / 2;
  static_assert(R >= 2 && R % 2 == 0, "two chains of R/2 outputs");
  const unsigned o = t * R, lane = t & 31u;
  const bool act = o < ns;
  if (act) {
#pragma unroll
    for (int r = 0; r < R; ++r) sx[spad<R>(o + r)] = k[r];
  }
  if constexpr (WARP) __syncwarp(); else __syncthreads();
  const unsigned base = o & ~(2 * L - 1);
  const bool merge = act && ns - base > L;
  // runs A = [base, base + L) (full) and B = [base + L, base + L + lb)
  const unsigned d = o - base, lb = merge ? min(L, ns - base - L) : 0u;
  const unsigned da = spad<R>(base), db = spad<R>(base + L);
  const C *A = sx + da, *B = sx + db;
  unsigned lo = 0;
  if (merge) {
    // merge path: how many of the first d outputs come from A
    lo = d > lb ? d - lb : 0;
    unsigned hi = min(d, L);
    while (lo < hi) {
      const unsigned mid = (lo + hi) >> 1;
      if (lt(B[spad<R>(d - 1 - mid)], A[spad<R>(mid)])) hi = mid;
      else lo = mid + 1;
    }
  }
  // the next thread's split is where this thread's outputs end
  unsigned lo_next = __shfl_down_sync(0xFFFFFFFFu, lo, 1);
  if constexpr (!WARP) {
    __shared__ unsigned s_first[NT / 32];
    if (lane == 0) s_first[t >> 5] = lo;
    __syncthreads();
    if (lane == 31 && t + 1 < (unsigned)NT) lo_next = s_first[(t >> 5) + 1];
  }
  if (merge) {
    const unsigned ja = d + R == L + lb ? L : lo_next;   // the pair's last thread ends at (L, lb)
    // ea, eb: keys of A and B not yet taken by the back chain; signed, as a
    // tie with the sentinel below a run takes the sentinel and steps past 0
    unsigned ia = lo, ib = d - lo;
    int ea = (int)ja, eb = (int)(d + R - ja);
    C x = ia < L ? A[spad<R>(ia)] : ones_code<C>();
    C y = ib < lb ? B[spad<R>(ib)] : ones_code<C>();
    C u = ea > 0 ? A[spad<R>((unsigned)ea - 1)] : zero_code<C>();
    C w = eb > 0 ? B[spad<R>((unsigned)eb - 1)] : zero_code<C>();
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const bool tb = lt(y, x);   // front: B's head strictly smaller
      const bool ta = lt(w, u);   // back: A's tail strictly larger
      k[r] = tb ? y : x;
      k[R - 1 - r] = ta ? u : w;
      if (r + 1 < H) {
        ia += tb ? 0u : 1u;
        ib += tb ? 1u : 0u;
        ea -= ta ? 1 : 0;
        eb -= ta ? 0 : 1;
        const unsigned i = tb ? ib : ia, lim = tb ? lb : L, d0 = tb ? db : da;
        const int e = ta ? ea : eb;
        const unsigned d1 = ta ? da : db;
        const C v = i < lim ? sx[d0 + spad<R>(i)] : ones_code<C>();
        const C v2 = e > 0 ? sx[d1 + spad<R>((unsigned)e - 1)] : zero_code<C>();
        x = tb ? x : v;
        y = tb ? v : y;
        u = ta ? v2 : u;
        w = ta ? w : v2;
      }
    }
  }
  if constexpr (WARP) __syncwarp(); else __syncthreads();
}

// Rounds for run lengths L0, 2 L0, ... while runs are shorter than ns (the
// test is uniform over the block, so every thread takes the same barriers):
// first the rounds whose run pairs fit one warp, then the block-wide ones.
// The rounds are loops, not unrolled: one body of each kind keeps the code
// small enough for the instruction cache.
template <class C, int R, int NT, unsigned L0>
__device__ __forceinline__ void mp_rounds(C (&k)[R], unsigned t, unsigned ns, C *sx) {
  unsigned L = L0;
#pragma unroll 1
  for (; L < ns && 2 * L <= 32u * R; L *= 2) mp_round<C, R, NT, true>(k, t, ns, sx, L);
#pragma unroll 1
  for (; L < ns; L *= 2) mp_round<C, R, NT, false>(k, t, ns, sx, L);
}

// Sorts the ns = (leaf length rounded up to L0) slots held by the first
// ns/R of NT threads (the others hold nothing and only take the barriers).
// Afterwards thread t holds logical slots t*R .. t*R+R-1. sx: spad<R>(NT*R)
// codes of shared memory.
template <class C, int R, int NT, unsigned L0>
__device__ __forceinline__ void merge_sort_block(C (&k)[R], unsigned t, unsigned ns, C *sx) {
  static_assert(L0 >= (unsigned)R && L0 <= 32u * R, "runs of the register stage fit one warp");
  if ((t & ~31u) * R < ns) {   // warps holding slots
    if constexpr (R > 1) column_sort<C, R>(k);
    warp_phases<C, R, (unsigned)R, L0>(k, t & 31u);
  }
  mp_rounds<C, R, NT, L0>(k, t, ns, sx);
}

// Comparisons made by merge_sort_block on ns slots (statistics): the
// column networks, the bitonic phases and, per merge round, one per output
// key plus the binary searches.
template <int R, int NT, unsigned L0> __device__ __forceinline__ unsigned long long merge_sort_cmps(unsigned ns) {
  constexpr unsigned col = R == 2 ? 1 : R == 4 ? 5 : R == 8 ? 19 : R == 16 ? 60 : 0;
  unsigned long long c = (unsigned long long)(ns / R) * col;
  for (unsigned L = R; L < L0; L *= 2) c += (unsigned long long)(ns / 2) * (ilog2(L) + 1);
  for (unsigned L = L0; L < ns; L *= 2) {
    const unsigned full = ns / (2 * L) * (2 * L), rest = ns - full;   // keys in pairs with a second run
    const unsigned merged = full + (rest > L ? rest : 0);
    c += merged + (unsigned long long)(merged / R) * (ilog2(L) + 1);
  }
  return c;
}

}  // namespace vq
