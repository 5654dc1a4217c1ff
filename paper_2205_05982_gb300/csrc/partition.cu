// The Quicksort recursion on the device: pivot sampling (Sec. 2.2), the
// partition level (Sec. 2.1) and the recursion driver (Algorithm 1) as one
// persistent kernel pulling tiles from an on-device work queue.
//
// A live range ("segment") [begin, end) of the recursion is cut into tiles of
// T keys; each tile is one queue item. A thread block claims the next item,
// loads the tile with one TMA bulk copy into shared memory, compares every
// key with the pivot, compacts left and right keys inside the block with
// warp ballots, learns how many left keys all earlier tiles of the range
// produced by decoupled look-back, and writes both runs to the other
// (ping-pong) buffer: left keys grow from `begin`, right keys from `end`
// downwards. The block that finishes the last tile of a range performs the
// rest of Algorithm 1 for it: the degenerate-partition rule, leaf routing of
// small children, the depth bound, pivot sampling of large children, and
// publication of their tiles as new queue items. No step needs the host.
#include "launch.h"
#include "sortnet.cuh"

namespace vq {

namespace {

constexpr int NT = PART_NT;
constexpr int NWARP = NT / 32;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr unsigned ERR_INVALID = 1, ERR_TIMEOUT = 5, ERR_INTERNAL = 6;

// ---------------------------------------------------------------------------
// SFC64 (Doty-Humphrey) with its published seeding, and the multiply-high
// bounded draw of Sec. 2.2.
// ---------------------------------------------------------------------------
struct Sfc64 {
  uint64_t a, b, c, n;
};
__device__ __forceinline__ uint64_t sfc_next(Sfc64 &s) {
  const uint64_t out = s.a + s.b + s.n++;
  s.a = s.b ^ (s.b >> 11);
  s.b = s.c + (s.c << 3);
  s.c = ((s.c << 24) | (s.c >> 40)) + out;
  return out;
}
__device__ __forceinline__ void sfc_seed(Sfc64 &s, uint64_t seed) {
  s.a = s.b = s.c = seed;
  s.n = 1;
  for (int i = 0; i < 12; ++i) sfc_next(s);
}

// ---------------------------------------------------------------------------
// Keys inside a 16-byte chunk (V = 16 / KB keys).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t word(const uint4 &q, unsigned i) {
  return i == 0 ? q.x : i == 1 ? q.y : i == 2 ? q.z : q.w;
}
__device__ __forceinline__ void set_word(uint4 &q, unsigned i, uint32_t w) {
  if (i == 0) q.x = w; else if (i == 1) q.y = w; else if (i == 2) q.z = w; else q.w = w;
}

template <int KB> __device__ __forceinline__ typename KT<KB>::Code key_at(const uint4 &q, unsigned v);
template <> __device__ __forceinline__ uint32_t key_at<2>(const uint4 &q, unsigned v) {
  const uint32_t w = word(q, v >> 1);
  return (v & 1) ? (w >> 16) : (w & 0xFFFFu);
}
template <> __device__ __forceinline__ uint32_t key_at<4>(const uint4 &q, unsigned v) { return word(q, v); }
template <> __device__ __forceinline__ uint64_t key_at<8>(const uint4 &q, unsigned v) {
  return ((uint64_t)word(q, 2 * v + 1) << 32) | word(q, 2 * v);
}
template <> __device__ __forceinline__ U128 key_at<16>(const uint4 &q, unsigned) {
  return U128{((uint64_t)q.y << 32) | q.x, ((uint64_t)q.w << 32) | q.z};
}

template <int KB> __device__ __forceinline__ void set_key(uint4 &q, unsigned v, typename KT<KB>::Code c);
template <> __device__ __forceinline__ void set_key<2>(uint4 &q, unsigned v, uint32_t c) {
  const uint32_t w = word(q, v >> 1);
  set_word(q, v >> 1, (v & 1) ? ((w & 0xFFFFu) | (c << 16)) : ((w & 0xFFFF0000u) | (c & 0xFFFFu)));
}
template <> __device__ __forceinline__ void set_key<4>(uint4 &q, unsigned v, uint32_t c) { set_word(q, v, c); }
template <> __device__ __forceinline__ void set_key<8>(uint4 &q, unsigned v, uint64_t c) {
  set_word(q, 2 * v, (uint32_t)c);
  set_word(q, 2 * v + 1, (uint32_t)(c >> 32));
}
template <> __device__ __forceinline__ void set_key<16>(uint4 &q, unsigned, U128 c) {
  q = make_uint4((uint32_t)c.lo, (uint32_t)(c.lo >> 32), (uint32_t)c.hi, (uint32_t)(c.hi >> 32));
}

template <int KB> __device__ __forceinline__ typename KT<KB>::Code code_of(uint64_t lo, uint64_t hi) {
  if constexpr (KB == 16) return U128{lo, hi};
  else return (typename KT<KB>::Code)lo;
}
template <int KB> __device__ __forceinline__ void code_words(typename KT<KB>::Code c, uint64_t &lo, uint64_t &hi) {
  if constexpr (KB == 16) { lo = c.lo; hi = c.hi; }
  else { lo = (uint64_t)c; hi = 0; }
}

// Shared scratch used by the range-level helpers (one per thread block).
struct RangeScratch {
  unsigned long long sid, q0, idx;
  int ok;
};

// ---------------------------------------------------------------------------
// Pivot sampling (Sec. 2.2, read for the GPU): 256/kc chunks of 64 bytes
// (kc = 64/KB keys), aligned to 64 bytes in memory, at SFC64-drawn chunk
// indices; the 256 sampled codes are sorted by one warp with the register
// network and the code at rank 127 is the pivot. Whole block participates.
// ---------------------------------------------------------------------------
template <int KB>
__device__ typename KT<KB>::Code sample_pivot(const void *buf, uint64_t b, uint64_t m, bool raw, Codec cd,
                                              uint64_t seed, void *scratch) {
  using C = typename KT<KB>::Code;
  constexpr unsigned kc = 64 / KB, ns = SAMPLE / kc;
  C *s_code = (C *)scratch;
  unsigned long long *s_chunk = (unsigned long long *)(s_code + SAMPLE);
  const uintptr_t addr = (uintptr_t)buf + b * KB;
  const uint64_t off = ((64 - (addr & 63)) & 63) / KB;
  const uint64_t nc = (m - off) / kc;
  if (threadIdx.x == 0) {
    Sfc64 r;
    sfc_seed(r, seed);
    for (unsigned j = 0; j < ns; ++j) s_chunk[j] = __umul64hi(sfc_next(r), nc);
  }
  __syncthreads();
  for (unsigned i = threadIdx.x; i < SAMPLE; i += blockDim.x) {
    const unsigned j = i / kc, t = i % kc;
    C c = load_cg<KB>(buf, b + off + s_chunk[j] * kc + t);
    if (raw) c = encode<KB>(c, cd);
    s_code[i] = c;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const unsigned lane = threadIdx.x;
    C k[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) k[r] = s_code[lane * 8 + r];
    warp_sort<C, 8>(k, lane);
#pragma unroll
    for (int r = 0; r < 8; ++r) s_code[lane * 8 + r] = k[r];
  }
  __syncthreads();
  const C p = s_code[SAMPLE / 2 - 1];
  __syncthreads();
  return p;
}

// ---------------------------------------------------------------------------
// Range bookkeeping (whole block).
// ---------------------------------------------------------------------------

// Creates a range to partition and publishes its tiles as queue items.
template <int KB>
__device__ void make_segment(const SortArgs &a, uint64_t b, uint64_t e, unsigned depth, unsigned flags,
                             typename KT<KB>::Code pivot, unsigned depth_limit, RangeScratch &rs) {
  constexpr unsigned T = part_tile_keys(KB);
  const uint64_t m = e - b;
  const unsigned nt = (unsigned)((m + T - 1) / T);
  if (threadIdx.x == 0) {
    const unsigned long long sid = atomicAdd(&a.hdr->nseg, 1ull);
    const unsigned long long q0 = atomicAdd(&a.hdr->tail, (unsigned long long)nt);
    int ok = sid < a.cap_segs && q0 + nt <= a.cap_q && sid < (1ull << 31);
    if (ok) {
      SegDesc &d = a.segs[sid];
      uint64_t lo, hi;
      code_words<KB>(pivot, lo, hi);
      d.begin = b;
      d.end = e;
      d.piv_lo = lo;
      d.piv_hi = hi;
      d.q0 = (unsigned)q0;
      d.ntiles = nt;
      d.depth = depth;
      d.flags = flags;
      d.tiles_done = 0;
      d.has_lt = 0;
      d.depth_limit = depth_limit;
      d.pad = 0;
    } else {
      raise_error(a, ERR_INTERNAL);
    }
    rs.sid = sid;
    rs.q0 = q0;
    rs.ok = ok;
  }
  __syncthreads();
  if (rs.ok) {
    const unsigned long long q0 = rs.q0, sid = rs.sid;
    for (unsigned k = threadIdx.x; k < nt; k += blockDim.x) st_relaxed(&a.status[q0 + k], 0);
    __threadfence();
    __syncthreads();
    for (unsigned k = threadIdx.x; k < nt; k += blockDim.x)
      st_release(&a.items[q0 + k], ITEM_VALID | (sid << 32) | k);
  }
  __syncthreads();
}

// Appends `count` entries to a leaf list; returns the first index or ~0.
__device__ unsigned long long reserve(const SortArgs &a, unsigned long long *counter, unsigned cap,
                                      unsigned count, RangeScratch &rs) {
  if (threadIdx.x == 0) {
    unsigned long long i = atomicAdd(counter, (unsigned long long)count);
    if (i + count > cap) {
      raise_error(a, ERR_INTERNAL);
      i = ~0ull;
    }
    rs.idx = i;
  }
  __syncthreads();
  const unsigned long long i = rs.idx;
  __syncthreads();
  return i;
}

// A finished range of keys that only needs sorting by a leaf network, or
// only decoding (all equal), or the merge fallback. Returns the keys handed
// over (counted off `remaining` by the caller).
__device__ void emit_leaf(const SortArgs &a, uint64_t b, uint64_t m, unsigned flags, RangeScratch &rs) {
  const bool warp = m <= WARP_LEAF_MAX;
  const unsigned long long i = warp ? reserve(a, &a.hdr->n_leaf_warp, a.cap_leaf_warp, 1, rs)
                                    : reserve(a, &a.hdr->n_leaf_block, a.cap_leaf_block, 1, rs);
  if (i != ~0ull && threadIdx.x == 0) {
    LeafEntry *l = warp ? a.leaf_warp : a.leaf_block;
    l[i] = LeafEntry{b, (unsigned)m, flags};
    atomicAdd(warp ? &a.hdr->leaves_warp : &a.hdr->leaves_block, 1ull);
    atomicAdd(&a.hdr->leaf_keys, m);
  }
}

__device__ void emit_equal(const SortArgs &a, uint64_t b, uint64_t m, unsigned flags, RangeScratch &rs) {
  const unsigned C = a.leaf_cutoff;
  const unsigned n = (unsigned)((m + C - 1) / C);
  const unsigned long long i = reserve(a, &a.hdr->n_leaf_block, a.cap_leaf_block, n, rs);
  if (i == ~0ull) return;
  for (unsigned k = threadIdx.x; k < n; k += blockDim.x) {
    const uint64_t cb = b + (uint64_t)k * C;
    const uint64_t len = min((uint64_t)C, b + m - cb);
    a.leaf_block[i + k] = LeafEntry{cb, (unsigned)len, flags | LEAF_COPY};
  }
  if (threadIdx.x == 0) {
    atomicAdd(&a.hdr->equal_ranges, 1ull);
    atomicAdd(&a.hdr->equal_keys, m);
  }
}

__device__ void emit_fallback(const SortArgs &a, uint64_t b, uint64_t m, unsigned flags, RangeScratch &rs) {
  const unsigned long long i = reserve(a, &a.hdr->n_fb, a.cap_fb, 1, rs);
  if (i != ~0ull && threadIdx.x == 0) {
    a.fb[i] = LeafEntry{b, (unsigned)m, flags};
    atomicAdd(&a.hdr->fallback_ranges, 1ull);
    atomicAdd(&a.hdr->fallback_keys, m);
  }
}

// A child of a partitioned range: leaf, fallback, or a new range to
// partition (Algorithm 1: BaseCase for small sides, ChoosePivot + Recurse
// otherwise; the depth bound of Sec. 2.2 before recursing). Returns the keys
// handed to a leaf list or the fallback.
template <int KB>
__device__ uint64_t child_range(const SortArgs &a, uint64_t b, uint64_t e, unsigned depth, unsigned parity,
                                unsigned depth_limit, void *scratch, RangeScratch &rs) {
  const uint64_t m = e - b;
  if (m == 0) return 0;
  if (m <= a.leaf_cutoff) {
    emit_leaf(a, b, m, parity, rs);
    return m;
  }
  if (depth >= depth_limit) {
    emit_fallback(a, b, m, parity, rs);
    return m;
  }
  const void *buf = parity ? a.alt : a.keys;
  const auto p = sample_pivot<KB>(buf, b, m, false, a.codec, range_seed(a.seed, b, depth), scratch);
  make_segment<KB>(a, b, e, depth, parity, p, depth_limit, rs);
  return 0;
}

// Everything Algorithm 1 does after Partition returned, for range `sd`.
template <int KB>
__device__ void finish_range(const SortArgs &a, const SegDesc &sd, unsigned sid, void *scratch,
                             RangeScratch &rs) {
  using C = typename KT<KB>::Code;
  const uint64_t b = sd.begin, e = sd.end, m = e - b;
  const uint64_t L = ld_relaxed(&a.status[sd.q0 + sd.ntiles - 1]) & ST_VAL;
  if (a.mode == MODE_PARTITION) {
    if (threadIdx.x == 0) {
      *a.out_left = L;
      st_release(&a.hdr->remaining, 0);
    }
    return;
  }
  const unsigned parity = (sd.flags & SEG_PARITY) ^ 1u;   // keys now live in the other buffer
  const unsigned d1 = sd.depth + 1;
  if (threadIdx.x == 0) {
    atomicAdd(&a.hdr->keys_partitioned, m);
    atomicAdd(&a.hdr->tiles, (unsigned long long)sd.ntiles);
    atomicAdd(&a.hdr->segments, 1ull);
    atomicMax(&a.hdr->max_depth, (unsigned long long)d1);
  }
  uint64_t handed = 0;
  if (sd.flags & SEG_EXCL) {
    // pivot was one below the repeated maximum p: the right side is all p
    handed += child_range<KB>(a, b, b + L, d1, parity, sd.depth_limit, scratch, rs);
    emit_equal(a, b + L, e - (b + L), parity, rs);
    handed += e - (b + L);
  } else if (L == m) {
    // Degenerate partition (Algorithm 1): every key <= pivot.
    if (threadIdx.x == 0) atomicAdd(&a.hdr->degenerate, 1ull);
    const unsigned has_lt = ld_relaxed32(&a.segs[sid].has_lt);
    if (!has_lt) {
      emit_equal(a, b, m, parity, rs);   // min == max: already sorted
      handed += m;
    } else if (d1 >= sd.depth_limit) {
      emit_fallback(a, b, m, parity, rs);
      handed += m;
    } else {
      // The pivot p is an input key and the maximum of the range. Split off
      // the keys equal to p with pivot p-1 (keys < p go left): both sides are
      // non-empty, so the recursion makes progress.
      const C p = code_of<KB>(sd.piv_lo, sd.piv_hi);
      make_segment<KB>(a, b, e, d1, parity | SEG_EXCL, pred(p), sd.depth_limit, rs);
    }
  } else {
    handed += child_range<KB>(a, b, b + L, d1, parity, sd.depth_limit, scratch, rs);
    handed += child_range<KB>(a, b + L, e, d1, parity, sd.depth_limit, scratch, rs);
  }
  __syncthreads();
  if (threadIdx.x == 0 && handed) atomicAdd(&a.hdr->remaining, (unsigned long long)(0ull - handed));
}

// ---------------------------------------------------------------------------
// Work claiming and look-back.
// ---------------------------------------------------------------------------

// Thread 0: claims the next ticket and waits (bounded) for its item. Returns
// 0 when all keys are placed, on abort, or on a timeout.
__device__ int claim(const SortArgs &a, unsigned long long &item) {
  const unsigned long long t = atomicAdd(&a.hdr->head, 1ull);
  for (unsigned it = 0;; ++it) {
    if (t < a.cap_q) {
      const unsigned long long v = ld_acquire(&a.items[t]);
      if (v & ITEM_VALID) {
        item = v;
        return 1;
      }
    }
    if (ld_acquire(&a.hdr->remaining) == 0) return 0;
    if (aborted(a)) return 0;
    if (it >= a.spin_limit) {
      raise_error(a, ERR_TIMEOUT);
      return 0;
    }
    __nanosleep(it < 32 ? 32 : 256);
  }
}

// Warp 0: publishes the tile's left count and returns the left keys of all
// earlier tiles of the range (decoupled look-back over a 32-tile window).
// Returns ~0 if the wait gave up.
__device__ uint64_t lookback(const SortArgs &a, unsigned long long *st, unsigned i, uint64_t tileL,
                             bool stall) {
  const unsigned lane = threadIdx.x & 31;
  if (i == 0) {
    if (lane == 0 && !stall) st_relaxed(&st[0], ST_PFX | tileL);
    return 0;
  }
  if (lane == 0) st_relaxed(&st[i], ST_AGG | tileL);
  uint64_t excl = 0;
  long long j = (long long)i - 1;
  for (;;) {
    const long long idx = j - (long long)lane;
    uint64_t v = ST_PFX;   // before tile 0: an empty inclusive prefix
    for (unsigned it = 0;; ++it) {
      if (idx >= 0) v = ld_relaxed(&st[idx]);
      if (__all_sync(FULL, (v >> 62) != 0)) break;
      const int give_up = it >= a.spin_limit || aborted(a);
      if (__any_sync(FULL, give_up)) {
        if (lane == 0 && it >= a.spin_limit) raise_error(a, ERR_TIMEOUT);
        return ~0ull;
      }
      if (it > 8) __nanosleep(64);
    }
    const unsigned pm = __ballot_sync(FULL, (v >> 62) == 2);
    const unsigned first = pm ? (unsigned)(__ffs(pm) - 1) : 31u;
    uint64_t val = lane <= first ? (v & ST_VAL) : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) val += __shfl_xor_sync(FULL, val, o);
    excl += val;
    if (pm) break;
    j -= 32;
  }
  if (lane == 0) st_relaxed(&st[i], ST_PFX | (excl + tileL));
  return excl;
}

// Writes `len` keys from shared memory (key index s, placed so that its byte
// offset matches `gdst` modulo 16) to global memory: 16-byte stores for the
// aligned body, single keys for the ragged ends.
template <int KB>
__device__ __forceinline__ void store_run(void *gdst, const unsigned char *smem, unsigned s, unsigned len) {
  using M = typename KT<KB>::Mem;
  constexpr unsigned V = 16 / KB;
  const uintptr_t ga = (uintptr_t)gdst;
  const unsigned head = min(len, (unsigned)(((16 - (ga & 15)) & 15) / KB));
  const unsigned body = (len - head) / V;
  const unsigned tail = len - head - body * V;
  const M *sm = (const M *)smem + s;
  M *g = (M *)gdst;
  if (threadIdx.x < head) g[threadIdx.x] = sm[threadIdx.x];
  const uint4 *sb = (const uint4 *)(sm + head);
  uint4 *gb = (uint4 *)(g + head);
  for (unsigned c = threadIdx.x; c < body; c += NT) gb[c] = sb[c];
  if (threadIdx.x < tail) g[head + body * V + threadIdx.x] = sm[head + body * V + threadIdx.x];
}

template <int KB> __device__ __forceinline__ typename KT<KB>::Mem to_mem(typename KT<KB>::Code c) {
  if constexpr (KB == 16) return c;
  else return (typename KT<KB>::Mem)c;
}

// ---------------------------------------------------------------------------
// Kernels.
// ---------------------------------------------------------------------------

// Resets the counters and clears the work queue.
__global__ void k_prep(SortArgs a) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (unsigned long long i = i0; i < a.cap_q; i += stride) a.items[i] = 0;
  unsigned long long *h = (unsigned long long *)a.hdr;
  for (unsigned long long i = i0; i < sizeof(Header) / 8; i += stride) h[i] = 0;
}

// Roots of the recursion: one range per segment (or the whole array).
template <int KB> __global__ void __launch_bounds__(NT) k_seed(SortArgs a) {
  __shared__ RangeScratch rs;
  __shared__ __align__(16) unsigned char scratch[SAMPLE * sizeof(typename KT<KB>::Code) + 64 * 8];
  for (unsigned long long sg = blockIdx.x; sg < a.num_segments; sg += gridDim.x) {
    uint64_t b = 0, e = a.n_total;
    if (a.offsets) {
      b = a.offsets[sg];
      e = a.offsets[sg + 1];
      if (b > e || e > a.n_total) {
        if (threadIdx.x == 0) raise_error(a, ERR_INVALID);
        return;
      }
    }
    const uint64_t m = e - b;
    if (a.mode == MODE_PARTITION) {
      if (m == 0) {
        if (threadIdx.x == 0) *a.out_left = 0;
        return;
      }
      if (threadIdx.x == 0) atomicAdd(&a.hdr->remaining, m);
      make_segment<KB>(a, b, e, 0, SEG_RAW, code_of<KB>(a.pivot.lo, a.pivot.hi), 1, rs);
      continue;
    }
    if (m <= 1) continue;   // one key in input form is already its own output
    const unsigned limit =
        a.depth_override >= 0 ? (unsigned)a.depth_override : 2 * floor_log2_u64(m) + 4;
    if (m <= a.leaf_cutoff) {
      emit_leaf(a, b, m, SEG_RAW, rs);
    } else if (limit == 0) {
      emit_fallback(a, b, m, SEG_RAW, rs);
    } else {
      if (threadIdx.x == 0) atomicAdd(&a.hdr->remaining, m);
      const auto p = sample_pivot<KB>(a.keys, b, m, true, a.codec, range_seed(a.seed, b, 0), scratch);
      make_segment<KB>(a, b, e, 0, SEG_RAW, p, limit, rs);
    }
    __syncthreads();
  }
}

// The persistent partition kernel.
template <int KB> __global__ void __launch_bounds__(NT, 3) k_partition(SortArgs a) {
  using C = typename KT<KB>::Code;
  using M = typename KT<KB>::Mem;
  constexpr unsigned V = 16 / KB;
  constexpr unsigned T = part_tile_keys(KB);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t s_bar;
  __shared__ SegDesc s_seg;
  __shared__ unsigned long long s_item;
  __shared__ int s_go, s_fin;
  __shared__ unsigned s_wL[NWARP], s_wV[NWARP], s_bL[NWARP], s_bR[NWARP];
  __shared__ unsigned long long s_pfx, s_dstR;
  __shared__ unsigned s_tileL, s_tileR, s_sL, s_sR;
  __shared__ RangeScratch rs;

  const unsigned tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) mbar_init(&s_bar, 1);
  __syncthreads();
  uint32_t phase = 0;

  for (;;) {
    if (tid == 0) {
      unsigned long long item = 0;
      const int go = claim(a, item);
      s_go = go;
      if (go) {
        s_item = item;
        const unsigned sid = (unsigned)((item >> 32) & 0x7FFFFFFFu);
        const unsigned long long *src = (const unsigned long long *)&a.segs[sid];
        unsigned long long *dstw = (unsigned long long *)&s_seg;
#pragma unroll
        for (int w = 0; w < 8; ++w) dstw[w] = __ldcg(src + w);
      }
    }
    __syncthreads();
    if (!s_go) break;

    const unsigned sid = (unsigned)((s_item >> 32) & 0x7FFFFFFFu);
    const unsigned i = (unsigned)(s_item & 0xFFFFFFFFu);
    const uint64_t b = s_seg.begin, e = s_seg.end;
    const bool par = s_seg.flags & SEG_PARITY, raw = s_seg.flags & SEG_RAW;
    const C piv = code_of<KB>(s_seg.piv_lo, s_seg.piv_hi);
    const unsigned char *src = (const unsigned char *)(par ? a.alt : a.keys);
    unsigned char *dst = (unsigned char *)(par ? a.keys : a.alt);
    const uint64_t t0 = b + (uint64_t)i * T;
    const unsigned cnt = (unsigned)min((uint64_t)T, e - t0);
    const uintptr_t g0 = (uintptr_t)(src + t0 * KB), g1 = g0 + (uintptr_t)cnt * KB;
    const uintptr_t w0 = g0 & ~(uintptr_t)15;
    const uintptr_t a0 = (g0 + 15) & ~(uintptr_t)15, a1 = g1 & ~(uintptr_t)15;
    const bool body = a0 < a1;

    // ---- load the tile: TMA bulk copy of the aligned body, plain loads of the ragged ends
    if (tid == 0) {
      fence_proxy_async();
      if (body) {
        mbar_arrive_expect_tx(&s_bar, (uint32_t)(a1 - a0));
        bulk_load(smem + (a0 - w0), (const void *)a0, (uint32_t)(a1 - a0), &s_bar);
      } else {
        mbar_arrive_expect_tx(&s_bar, 0);
      }
    }
    if constexpr (KB < 16) {
      const uintptr_t hend = body ? a0 : g1;
      const unsigned nh = (unsigned)((hend - g0) / KB);
      const unsigned ntl = body ? (unsigned)((g1 - a1) / KB) : 0u;
      if (tid < nh) {
        *(M *)(smem + (g0 - w0) + tid * KB) = __ldcg((const M *)g0 + tid);
      } else if (tid >= 64 && tid < 64 + ntl) {
        *(M *)(smem + (a1 - w0) + (tid - 64) * KB) = __ldcg((const M *)a1 + (tid - 64));
      }
    }
    {
      unsigned it = 0;
      while (!mbar_try_wait(&s_bar, phase)) {
        if (++it > a.spin_limit) {   // a copy that never lands: give up (cannot happen for valid addresses)
          if (tid == 0) raise_error(a, ERR_TIMEOUT);
          break;
        }
      }
    }
    phase ^= 1;
    __syncthreads();

    // ---- tile chunks into registers (raw root tiles are encoded here)
    const unsigned nwc = (unsigned)((((g1 + 15) & ~(uintptr_t)15) - w0) / 16);
    const unsigned lo = (unsigned)(g0 - w0), hi = (unsigned)(g1 - w0);
    uint4 ch[PART_CPT];
    const uint4 *sw = (const uint4 *)smem;
#pragma unroll
    for (int j = 0; j < PART_CPT; ++j) {
      const unsigned c = tid + j * NT;
      ch[j] = c < nwc ? sw[c] : make_uint4(0, 0, 0, 0);
      if (raw) {
#pragma unroll
        for (unsigned v = 0; v < V; ++v) set_key<KB>(ch[j], v, encode<KB>(key_at<KB>(ch[j], v), a.codec));
      }
    }

    // ---- pass 1: per-warp counts of left and valid keys
    unsigned nL = 0, nV = 0;
    int anyLt = 0;
#pragma unroll
    for (int j = 0; j < PART_CPT; ++j) {
#pragma unroll
      for (unsigned v = 0; v < V; ++v) {
        const unsigned off = 16 * (tid + j * NT) + v * KB;
        const bool valid = off >= lo && off < hi;
        const C c = key_at<KB>(ch[j], v);
        const bool le = !lt(piv, c);
        nL += (valid && le);
        nV += valid;
        anyLt |= (valid && lt(c, piv));
      }
    }
    nL = __reduce_add_sync(FULL, nL);
    nV = __reduce_add_sync(FULL, nV);
    if (lane == 0) {
      s_wL[warp] = nL;
      s_wV[warp] = nV;
    }
    anyLt = __syncthreads_or(anyLt);

    // ---- block scan of warp counts, then look-back across tiles
    if (warp == 0) {
      unsigned xL = lane < NWARP ? s_wL[lane] : 0, xV = lane < NWARP ? s_wV[lane] : 0;
      unsigned iL = xL, iV = xV;
#pragma unroll
      for (int o = 1; o < NWARP; o <<= 1) {
        const unsigned yL = __shfl_up_sync(FULL, iL, o), yV = __shfl_up_sync(FULL, iV, o);
        if (lane >= (unsigned)o) { iL += yL; iV += yV; }
      }
      const unsigned totL = __shfl_sync(FULL, iL, NWARP - 1), totV = __shfl_sync(FULL, iV, NWARP - 1);
      if (lane < NWARP) {
        s_bL[lane] = iL - xL;
        s_bR[lane] = (iV - xV) - (iL - xL);
      }
      const bool stall = a.test_stall && sid == 0;
      const uint64_t excl = lookback(a, a.status + s_seg.q0, i, totL, stall);
      if (lane == 0) {
        s_pfx = excl;
        s_tileL = totL;
        s_tileR = totV - totL;
        if (excl != ~0ull) {
          const uint64_t rightPrefix = (uint64_t)i * T - excl;
          const uint64_t dstR = e - rightPrefix - (totV - totL);
          const uintptr_t gL = (uintptr_t)(dst + (b + excl) * KB), gR = (uintptr_t)(dst + dstR * KB);
          const unsigned sL = (unsigned)((gL & 15) / KB);
          s_sL = sL;
          s_sR = ((sL + totL + V - 1) / V) * V + (unsigned)((gR & 15) / KB);
          s_dstR = dstR;
        }
      }
    }
    __syncthreads();
    if (s_pfx == ~0ull) break;

    // ---- pass 2: ballot compaction into the staging buffer (reuses the window)
    {
      unsigned runL = s_bL[warp], runR = s_bR[warp];
      const unsigned sL = s_sL, sR = s_sR;
      const unsigned ltm = (1u << lane) - 1u;
      M *stage = (M *)smem;
      const bool dec = a.mode == MODE_PARTITION;
#pragma unroll
      for (int j = 0; j < PART_CPT; ++j) {
#pragma unroll
        for (unsigned v = 0; v < V; ++v) {
          const unsigned off = 16 * (tid + j * NT) + v * KB;
          const bool valid = off >= lo && off < hi;
          const C c = key_at<KB>(ch[j], v);
          const bool le = !lt(piv, c);
          const unsigned bl = __ballot_sync(FULL, valid && le), br = __ballot_sync(FULL, valid && !le);
          if (valid) {
            const unsigned pos = le ? sL + runL + __popc(bl & ltm) : sR + runR + __popc(br & ltm);
            stage[pos] = to_mem<KB>(dec ? decode<KB>(c, a.codec) : c);
          }
          runL += __popc(bl);
          runR += __popc(br);
        }
      }
    }
    __syncthreads();

    // ---- write both runs with 16-byte stores
    store_run<KB>(dst + (b + s_pfx) * KB, smem, s_sL, s_tileL);
    store_run<KB>(dst + s_dstR * KB, smem, s_sR, s_tileR);
    fence_proxy_async();   // the next TMA copy reuses the window

    // ---- range completion
    if (anyLt && tid == 0) atomicOr(&a.segs[sid].has_lt, 1u);
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const unsigned prev = atomicAdd(&a.segs[sid].tiles_done, 1u);
      const int fin = prev == s_seg.ntiles - 1;
      if (fin) __threadfence();
      s_fin = fin;
    }
    __syncthreads();
    if (s_fin) {
      __threadfence();
      finish_range<KB>(a, s_seg, sid, smem, rs);
    }
    __syncthreads();
  }
}

// Pivot of one array by the sampling rule (debug/test entry).
template <int KB> __global__ void __launch_bounds__(NT) k_choose_pivot(SortArgs a, const void *keys,
                                                                       unsigned long long n,
                                                                       unsigned long long seed, void *out) {
  __shared__ __align__(16) unsigned char scratch[SAMPLE * sizeof(typename KT<KB>::Code) + 64 * 8];
  const auto p = sample_pivot<KB>(keys, 0, n, true, a.codec, seed, scratch);
  if (threadIdx.x == 0) store_key<KB>(out, 0, decode<KB>(p, a.codec));
}

template <int KB> int partition_grid() {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_partition<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, PART_SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_partition<KB>, NT, PART_SMEM);
    grid = sms * (per > 0 ? per : 1);
  }
  return grid;
}

template <int KB> cudaError_t seed_impl(const SortArgs &a, cudaStream_t s) {
  const unsigned long long g = a.num_segments < 65535ull * 4 ? a.num_segments : 65535ull * 4;
  k_seed<KB><<<(unsigned)(g ? g : 1), NT, 0, s>>>(a);
  return cudaGetLastError();
}

template <int KB> cudaError_t partition_impl(const SortArgs &a, cudaStream_t s) {
  k_partition<KB><<<partition_grid<KB>(), NT, PART_SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prep(const SortArgs &a, cudaStream_t s) {
  unsigned long long work = a.cap_q > sizeof(Header) / 8 ? a.cap_q : sizeof(Header) / 8;
  unsigned blocks = (unsigned)min(4096ull, (work + 1023) / 1024);
  k_prep<<<blocks ? blocks : 1, 1024, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_seed(int kb, const SortArgs &a, cudaStream_t s) {
  switch (kb) {
    case 2: return seed_impl<2>(a, s);
    case 4: return seed_impl<4>(a, s);
    case 8: return seed_impl<8>(a, s);
    case 16: return seed_impl<16>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_partition(int kb, const SortArgs &a, cudaStream_t s) {
  switch (kb) {
    case 2: return partition_impl<2>(a, s);
    case 4: return partition_impl<4>(a, s);
    case 8: return partition_impl<8>(a, s);
    case 16: return partition_impl<16>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_choose_pivot(int kb, const SortArgs &a, const void *keys, unsigned long long n,
                                unsigned long long seed, void *out, cudaStream_t s) {
  switch (kb) {
    case 2: k_choose_pivot<2><<<1, NT, 0, s>>>(a, keys, n, seed, out); break;
    case 4: k_choose_pivot<4><<<1, NT, 0, s>>>(a, keys, n, seed, out); break;
    case 8: k_choose_pivot<8><<<1, NT, 0, s>>>(a, keys, n, seed, out); break;
    case 16: k_choose_pivot<16><<<1, NT, 0, s>>>(a, keys, n, seed, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace vq
