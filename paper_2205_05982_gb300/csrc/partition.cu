// The Quicksort recursion on the device: pivot sampling (Sec. 2.2), the
// partition level (Sec. 2.1) and the recursion driver (Algorithm 1) as one
// persistent kernel pulling work from an on-device queue.
//
// A live range ("segment") [begin, end) of the recursion is cut into tiles;
// each tile is one queue item. A thread block claims the next item and loads
// the tile with one TMA bulk copy into shared memory. A two-way range
// compares every key with the pivot, compacts left and right keys with warp
// ballots, reserves its slots on both sides with one atomic on the range's
// write cursors and writes both runs to the other (ping-pong) buffer: left
// keys grow from `begin`, right keys from `end` downwards. A K-way range (16
// to 256 buckets, the multi-pivot split of Sec. 4.2) runs a counting pass and
// a scatter pass over its tiles. The block that finishes the last tile of a
// range performs the rest of Algorithm 1 for it: the degenerate-partition
// rule, leaf routing of small children, the depth bound, pivot sampling of
// children (large ones through setup items that any block can claim), and
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
template <> __device__ __forceinline__ KV key_at<KV_KEYONLY>(const uint4 &q, unsigned) {
  return KV{((uint64_t)q.y << 32) | q.x, ((uint64_t)q.w << 32) | q.z};
}

template <int KB> __device__ __forceinline__ typename KT<KB>::Code code_of(uint64_t lo, uint64_t hi) {
  if constexpr (kmem(KB) == 16) return typename KT<KB>::Code{lo, hi};
  else return (typename KT<KB>::Code)lo;
}
template <int KB> __device__ __forceinline__ void code_words(typename KT<KB>::Code c, uint64_t &lo, uint64_t &hi) {
  if constexpr (kmem(KB) == 16) { lo = c.lo; hi = c.hi; }
  else { lo = (uint64_t)c; hi = 0; }
}

// Shared scratch used by the range-level helpers (one per thread block).
struct RangeScratch {
  unsigned long long sid, q0, idx;   // q0: first queue slot of a new range
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
  constexpr unsigned kc = 64 / kmem(KB), ns = SAMPLE / kc;
  C *s_code = (C *)scratch;
  unsigned long long *s_chunk = (unsigned long long *)(s_code + SAMPLE);
  const uintptr_t addr = (uintptr_t)buf + b * kmem(KB);
  const uint64_t off = ((64 - (addr & 63)) & 63) / kmem(KB);
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

// Publishes `count` queue items from slot q0 on: item k = bits | k. Each
// thread fences once (ordering the range's descriptor, written before the
// caller's barrier) and then stores its items relaxed.
__device__ __forceinline__ void publish_items(const SortArgs &a, unsigned long long q0, unsigned count,
                                              unsigned long long bits) {
  if (threadIdx.x >= count) return;
  fence_release();
  for (unsigned k = threadIdx.x; k < count; k += blockDim.x) st_relaxed(&a.items[q0 + k], bits | k);
}

// Creates a range to partition and publishes its tiles as queue items.
template <int KB>
__device__ void make_segment(const SortArgs &a, uint64_t b, uint64_t e, unsigned depth, unsigned flags,
                             typename KT<KB>::Code pivot, unsigned depth_limit, RangeScratch &rs) {
  const unsigned T = a.tile_keys;
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
      d.cursor = 0;
      d.depth = depth;
      d.flags = flags;
      d.ntiles = nt;
      d.tiles_done = 0;
      d.has_lt = 0;
      d.depth_limit = depth_limit;
    } else {
      raise_error(a, ERR_INTERNAL);
    }
    rs.sid = sid;
    rs.q0 = q0;
    rs.ok = ok;
  }
  __syncthreads();
  // the descriptor (written by thread 0, ordered by the barrier above) is
  // published with the items
  if (rs.ok) publish_items(a, rs.q0, nt, ITEM_VALID | (rs.sid << 32));
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

// The leaf list for a range of m keys (at most the cutoff): warp leaves up to
// WARP_LEAF_MAX keys, mid-size leaves up to a.mid_max, block leaves above.
struct LeafList {
  unsigned long long *n, *stat, *keys;
  LeafEntry *list;
  unsigned cap;
};
__device__ __forceinline__ LeafList leaf_list(const SortArgs &a, uint64_t m) {
  if (m <= WARP_LEAF_MAX)
    return LeafList{&a.hdr->n_leaf_warp, &a.hdr->leaves_warp, &a.hdr->leaf_keys_warp, a.leaf_warp, a.cap_leaf_warp};
  if (m <= a.mid_max)
    return LeafList{&a.hdr->n_leaf_mid, &a.hdr->leaves_mid, &a.hdr->leaf_keys_mid, a.leaf_mid, a.cap_leaf_mid};
  return LeafList{&a.hdr->n_leaf_block, &a.hdr->leaves_block, &a.hdr->leaf_keys_block, a.leaf_block,
                  a.cap_leaf_block};
}

// A finished range of keys that only needs sorting by a leaf network
// (emit_leaf), or only decoding because all keys are equal (emit_equal), or
// the merge fallback (emit_fallback). The caller counts the keys handed over
// off `remaining`.
__device__ void emit_leaf(const SortArgs &a, uint64_t b, uint64_t m, unsigned flags, RangeScratch &rs) {
  const LeafList L = leaf_list(a, m);
  const unsigned long long i = reserve(a, L.n, L.cap, 1, rs);
  if (i != ~0ull && threadIdx.x == 0) {
    L.list[i] = LeafEntry{b, (unsigned)m, flags};
    atomicAdd(L.stat, 1ull);
    atomicAdd(&a.hdr->leaf_keys, m);
    atomicAdd(L.keys, m);
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

// ---------------------------------------------------------------------------
// K-way ranges. The paper tried a K > 2 partition only as a prototype (Sec.
// 4.2); on the GPU a split into K = 2^kbits buckets (16..256) costs one
// counting pass and one scatter pass, where two-way levels would need kbits
// passes. Splitters come from a sorted random sample; bucket j holds the keys
// above splitter j and at most splitter j+1 (keys equal to a splitter take
// the lower bucket, the "<=" rule of the two-way partition). When the
// splitters repeat values, the range switches to equality mode: 2d + 1
// buckets around its d distinct splitters, every second one holding the keys
// equal to one splitter (build_splitters). A key's bucket
// is found through a table indexed by the KW_TABLE_BITS code bits that follow
// the prefix shared by the first and the last splitter: the table gives the
// splitters certainly below the key and the few (usually none or one) that
// share its table bits, which are then compared.
// ---------------------------------------------------------------------------

// Exclusive scan of one value per thread over the block; `total` gets the sum.
__device__ unsigned long long block_excl_scan(unsigned long long x, unsigned long long *s_w,
                                              unsigned long long &total) {
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(FULL, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  unsigned long long pre = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < NWARP; ++w) {
    const unsigned long long v = s_w[w];
    if (w < (int)warp) pre += v;
    tot += v;
  }
  __syncthreads();
  total = tot;
  return pre + incl - x;
}

// Keys per thread of the splitter sample: as many as the scratch holds.
template <int KB, int CPT> __host__ __device__ constexpr unsigned kw_sample_r() {
  return kmem(KB) == 16 ? (CPT >= 8 ? 4u : 2u) : (CPT >= 8 ? 8u : 4u);
}
template <int KB, unsigned R> __host__ __device__ constexpr unsigned kw_scratch_bytes() {
  return R * NT * (unsigned)sizeof(typename KT<KB>::Code) + R * NT / (64 / kmem(KB)) * 8u;
}

// Leading bits shared by two codes (the code width when they are equal).
__device__ __forceinline__ unsigned common_prefix(uint32_t x, uint32_t y) { return x == y ? 32u : __clz(x ^ y); }
__device__ __forceinline__ unsigned common_prefix(uint64_t x, uint64_t y) { return x == y ? 64u : __clzll(x ^ y); }
__device__ __forceinline__ unsigned common_prefix(const U128 &x, const U128 &y) {
  return x.hi != y.hi ? (unsigned)__clzll(x.hi ^ y.hi) : x.lo != y.lo ? 64u + __clzll(x.lo ^ y.lo) : 128u;
}
__device__ __forceinline__ unsigned common_prefix(const KV &x, const KV &y) { return common_prefix(x.hi, y.hi); }

// The KW_TABLE_BITS bits of code k that follow its first `sh` bits (zeros
// past the end of the code); sh is below the code width.
__device__ __forceinline__ unsigned table_bits(uint32_t k, unsigned sh) {
  return (k << (sh & 31)) >> (32 - KW_TABLE_BITS);
}
__device__ __forceinline__ unsigned table_bits(uint64_t k, unsigned sh) {
  return (unsigned)((k << (sh & 63)) >> (64 - KW_TABLE_BITS));
}
__device__ __forceinline__ unsigned table_bits(const KV &k, unsigned sh) { return table_bits(k.hi, sh); }
__device__ __forceinline__ unsigned table_bits(const U128 &k, unsigned sh) {
  const unsigned s = sh & 127;
  const uint64_t top = s == 0 ? k.hi : s < 64 ? (k.hi << s) | (k.lo >> (64 - s)) : k.lo << (s - 64);
  return (unsigned)(top >> (64 - KW_TABLE_BITS));
}

// Bucket of code k: the number of splitters strictly below it. split[1..K-1]
// ascending, s1 = split[1], sk = split[K-1], sh = their shared prefix.
template <class C>
__device__ __forceinline__ unsigned classify(const C &k, const C *split, const unsigned short *table,
                                             const C &s1, const C &sk, unsigned sh, unsigned K) {
  if (!lt(s1, k)) return 0;
  if (lt(sk, k)) return K - 1;
  // s1 < k <= sk: k shares the prefix, so every splitter with smaller
  // table bits is below k and every one with larger bits above it
  const unsigned e = table[table_bits(k, sh)];
  unsigned b = e & 255u, n = e >> 8;
  // Count the splitters with equal table bits that are below k. Most keys
  // have none or one: the first candidate is compared without a branch
  // (loaded even when there is none, from a valid slot), and only a key above
  // it with more candidates left enters the search loop.
  {
    const bool below = lt(split[b < KW_MAX - 1 ? b + 1 : KW_MAX - 1], k);
    if (n) {
      if (below) {
        ++b;
        --n;
      } else {
        n = 0;
      }
    }
  }
  while (n) {
    const unsigned h = n >> 1;
    if (lt(split[b + h + 1], k)) {
      b += h + 1;
      n -= h + 1;
    } else {
      n = h;
    }
  }
  return b;
}

// The bucket lookup of one K-way range, staged in shared memory: nsp
// splitters split[1..nsp]; in equality mode (eqb) bucket 2b holds the keys
// strictly between splitters b and b+1 and bucket 2b+1 the keys equal to
// splitter b+1.
template <class C> struct KwLookup {
  const C *split;
  const unsigned short *table;
  C s1, sk;
  unsigned sh, nsp, eqb;
  __device__ __forceinline__ unsigned operator()(const C &k) const {
    const unsigned b = classify(k, split, table, s1, sk, sh, nsp + 1);
    if (!eqb) return b;
    return 2 * b + ((b < nsp && eq(k, split[b + 1])) ? 1u : 0u);
  }
};

// Buckets for a range of m keys: about kw_target keys each, 16..256 of them.
__device__ __forceinline__ unsigned kway_bits(const SortArgs &a, uint64_t m) {
  unsigned bits = KW_MIN_BITS;
  while (bits < KW_MAX_BITS && ((uint64_t)a.kw_target << bits) < m) ++bits;
  return bits;
}

// Samples R*NT keys of [b, b+m) (whole 64-byte chunks at random positions,
// as in sample_pivot, but drawn independently per chunk),
// sorts them with the block network and takes splitter i = sample rank
// i*S/K - 1 (i = 1..K-1). When those repeat a value (heavy duplicates) and
// the distinct values d number at most 127, the range switches to equality
// mode: the d distinct values split it into 2d + 1 buckets, every second one
// holding the keys equal to one splitter, which need no further sorting (the
// K-way form of a three-way partition). Writes the splitters and the lookup
// table to `kw` and returns the bucket count, or 0, writing nothing, when
// every sampled code is the same (such ranges are split in two).
template <int KB, unsigned R>
__device__ unsigned build_splitters(const void *buf, uint64_t b, uint64_t m, bool raw, Codec cd, uint64_t seed,
                                    unsigned kbits, KwayDesc &kw, void *scratch) {
  using C = typename KT<KB>::Code;
  constexpr unsigned S = R * NT, kc = 64 / kmem(KB), ns = S / kc;
  static_assert(S >= 2 * KW_MAX, "sample holds the splitters and their distinct values");
  constexpr unsigned WIDTH = KB == KV_KEYONLY ? 64u : 8 * sizeof(C);   // bits the order reads
  C *sx = (C *)scratch;
  unsigned long long *s_chunk = (unsigned long long *)(sx + S);
  __shared__ int s_same;
  __shared__ unsigned long long s_wb[NWARP];
  const uintptr_t addr = (uintptr_t)buf + b * kmem(KB);
  const uint64_t off = ((64 - (addr & 63)) & 63) / kmem(KB);
  const uint64_t nc = (m - off) / kc;
  // one draw per thread: the SplitMix64 finaliser of the range seed and the
  // draw index (counter-based, so no thread waits on a sequential stream),
  // bounded by multiply-high
  for (unsigned j = threadIdx.x; j < ns; j += NT)
    s_chunk[j] = __umul64hi(mix64(seed + 0x9E3779B97F4A7C15ull * (j + 1)), nc);
  __syncthreads();
  C k[R];
#pragma unroll
  for (unsigned r = 0; r < R; ++r) {
    const unsigned i = threadIdx.x + r * NT;
    const C c = load_cg<KB>(buf, b + off + s_chunk[i / kc] * kc + i % kc);
    k[r] = raw ? encode<KB>(c, cd) : c;
  }
  group_sort<C, R, NT>(k, threadIdx.x, sx);   // thread t: sample ranks R*t .. R*t+R-1
  if (threadIdx.x == 0) sx[0] = k[0];
  __syncthreads();
  if (threadIdx.x == NT - 1) s_same = eq(sx[0], k[R - 1]);
  __syncthreads();
  const bool same = s_same;
  if (same) return 0;   // uniform across the block
  const unsigned K = 1u << kbits, step = S >> kbits;
  C *sp = sx;   // splitters 1..K-1
#pragma unroll
  for (unsigned r = 0; r < R; ++r) {
    const unsigned rank1 = R * threadIdx.x + r + 1;
    const unsigned i = rank1 / step;
    if (rank1 % step == 0 && i < K) sp[i] = k[r];
  }
  __syncthreads();
  // distinct splitter values, compacted to dv[1..nd]
  const unsigned i = threadIdx.x + 1;
  const bool first = i < K && (i == 1 || !eq(sp[i], sp[i - 1]));
  unsigned long long nd;
  const unsigned long long pos = block_excl_scan(first ? 1ull : 0ull, s_wb, nd);
  const bool eqm = nd < K - 1 && 2 * nd + 1 <= KW_MAX;
  C *dv = sx + KW_MAX;
  if (eqm && first) dv[pos + 1] = sp[i];
  __syncthreads();
  const C *use = eqm ? dv : sp;
  const unsigned nsp = eqm ? (unsigned)nd : K - 1;
  for (unsigned j = threadIdx.x + 1; j <= nsp; j += NT) {
    uint64_t lo, hi;
    code_words<KB>(use[j], lo, hi);
    kw.split_lo[j] = lo;
    kw.split_hi[j] = hi;
  }
  const unsigned sh = common_prefix(use[1], use[nsp]);
  if (threadIdx.x == 0) {
    kw.shift = sh;
    kw.nsplit = nsp;
    kw.eqmode = eqm;
  }
  // table[p]: splitters (all sharing the prefix, so their table bits ascend
  // with the index) whose table bits are below p, and how many equal p
  for (unsigned p = threadIdx.x; p < KW_TABLE; p += NT) {
    unsigned below = 0, upto = 0;
    if (sh < WIDTH) {
      unsigned lo = 1, n = nsp;   // first j with bits(use[j]) >= p
      while (n) {
        const unsigned h = n >> 1;
        if (table_bits(use[lo + h], sh) < p) { lo += h + 1; n -= h + 1; } else n = h;
      }
      below = lo - 1;
      unsigned lo2 = lo, n2 = nsp + 1 - lo;   // first j with bits(use[j]) > p
      while (n2) {
        const unsigned h = n2 >> 1;
        if (table_bits(use[lo2 + h], sh) <= p) { lo2 += h + 1; n2 -= h + 1; } else n2 = h;
      }
      upto = lo2 - 1;
    }
    kw.table[p] = (unsigned short)(below | ((upto - below) << 8));
  }
  __syncthreads();
  return eqm ? 2 * (unsigned)nd + 1 : K;
}

// Counting-pass tiles of a K-way range with `nt` scatter-pass tiles: a
// counting tile needs no staging half, so it covers two scatter tiles' keys
// (the whole window) and keeps one histogram for each.
__device__ __forceinline__ unsigned kw_count_items(unsigned nt) { return (nt + 1) / 2; }

// Creates a K-way range on record `kid` (splitters already written) and
// publishes its counting-pass tiles.
__device__ void make_kway_segment(const SortArgs &a, uint64_t b, uint64_t e, unsigned depth, unsigned flags,
                                  unsigned depth_limit, unsigned long long kid, unsigned K,
                                  RangeScratch &rs) {
  const unsigned T = a.kw_tile_keys;
  const uint64_t m = e - b;
  const unsigned nt = (unsigned)((m + T - 1) / T), nc = kw_count_items(nt);
  KwayDesc &kw = a.kw[kid];
  for (unsigned j = threadIdx.x; j < K; j += NT)
#pragma unroll
    for (unsigned st = 0; st < KW_STRIPES; ++st) kw.cnt[st][j] = 0;
  if (threadIdx.x == 0) {
    const unsigned long long sid = atomicAdd(&a.hdr->nseg, 1ull);
    const unsigned long long q0 = atomicAdd(&a.hdr->tail, (unsigned long long)nc);
    const int ok = sid < a.cap_segs && q0 + nc <= a.cap_q && sid < (1ull << 31);
    if (ok) {
      SegDesc &d = a.segs[sid];
      d.begin = b;
      d.end = e;
      d.piv_lo = kid;
      d.piv_hi = K;
      d.cursor = 0;
      d.depth = depth;
      d.flags = flags | SEG_KWAY;
      d.ntiles = nt;
      d.tiles_done = 0;
      d.has_lt = 0;
      d.depth_limit = depth_limit;
    } else {
      raise_error(a, ERR_INTERNAL);
    }
    rs.sid = sid;
    rs.q0 = q0;
    rs.ok = ok;
  }
  __syncthreads();
  // the counters (zeroed above) and the descriptor are published with the items
  if (rs.ok) publish_items(a, rs.q0, nc, ITEM_VALID | (rs.sid << 32));
  __syncthreads();
}

// Starts partitioning [b, e) (more than a leaf, depth below its bound):
// a K-way range when it is large enough and its sample has two values or
// more, else a two-way range around a sampled pivot (Algorithm 1's
// ChoosePivot). `scratch` holds kw_scratch_bytes<KB, R>() bytes.
template <int KB, unsigned R>
__device__ void start_range(const SortArgs &a, uint64_t b, uint64_t e, unsigned depth, unsigned flags,
                            unsigned depth_limit, bool allow_kway, void *scratch, RangeScratch &rs) {
  const uint64_t m = e - b;
  const bool raw = flags & SEG_RAW;
  const void *buf = (flags & SEG_PARITY) ? a.alt : a.keys;
  const uint64_t seed = range_seed(a.seed, b, depth);
  if (allow_kway && a.kw && m >= a.kw_min_keys) {
    if (threadIdx.x == 0) {
      const unsigned long long kid = atomicAdd(&a.hdr->nkw, 1ull);
      rs.idx = kid < a.cap_kw ? kid : ~0ull;   // no record left: split in two
    }
    __syncthreads();
    const unsigned long long kid = rs.idx;
    __syncthreads();
    if (kid != ~0ull) {
      const unsigned K = build_splitters<KB, R>(buf, b, m, raw, a.codec, seed, kway_bits(a, m), a.kw[kid], scratch);
      if (K) {
        make_kway_segment(a, b, e, depth, flags, depth_limit, kid, K, rs);
        return;
      }
    }
  }
  const auto p = sample_pivot<KB>(buf, b, m, raw, a.codec, seed, scratch);
  make_segment<KB>(a, b, e, depth, flags | (allow_kway ? 0u : SEG_NOKWAY), p, depth_limit, rs);
}

// Thread 0: queues the setup of child j of range psid (sampled later by
// whichever block claims the item).
__device__ void publish_setup(const SortArgs &a, unsigned psid, unsigned j, bool nokway) {
  const unsigned long long q = atomicAdd(&a.hdr->tail, 1ull);
  if (q >= a.cap_q) {
    raise_error(a, ERR_INTERNAL);
    return;
  }
  st_release(&a.items[q], ITEM_VALID | ((unsigned long long)psid << 32) | ITEM_SETUP |
                              (nokway ? ITEM_NOKWAY : 0ull) | j);
}

// A child [b, e) of two-way range psid (j = 0 left, 1 right): leaf,
// fallback, or a new range to partition (Algorithm 1: BaseCase for small
// sides, ChoosePivot + Recurse otherwise; the depth bound of Sec. 2.2
// before recursing). Children large enough for a K-way split are queued as
// setup items, whose larger sample does not fit this block's free scratch.
// Returns the keys handed to a leaf list or the fallback.
template <int KB>
__device__ uint64_t child_range(const SortArgs &a, uint64_t b, uint64_t e, unsigned depth, unsigned parity,
                                unsigned depth_limit, void *scratch, RangeScratch &rs, unsigned psid,
                                unsigned j) {
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
  if (a.kw && m >= a.kw_min_keys) {
    if (threadIdx.x == 0) publish_setup(a, psid, j, false);
    return 0;
  }
  const auto p = sample_pivot<KB>(parity ? a.alt : a.keys, b, m, false, a.codec, range_seed(a.seed, b, depth),
                                  scratch);
  make_segment<KB>(a, b, e, depth, parity, p, depth_limit, rs);
  return 0;
}

// After the counting pass of a K-way range: bucket bounds from the counts,
// each stripe's write cursor at its share of the bucket, then the
// scatter-pass tiles.
__device__ void finish_kway_count(const SortArgs &a, const SegDesc &sd, unsigned sid, RangeScratch &rs,
                                  unsigned long long *s_w) {
  KwayDesc &kw = a.kw[sd.piv_lo];
  const unsigned K = (unsigned)sd.piv_hi;
  const unsigned tid = threadIdx.x;
  unsigned c[KW_STRIPES];
  unsigned long long cnt = 0;
#pragma unroll
  for (unsigned st = 0; st < KW_STRIPES; ++st) {
    c[st] = tid < K ? __ldcg(&kw.cnt[st][tid]) : 0u;
    cnt += c[st];
  }
  unsigned long long total;
  const unsigned long long excl = block_excl_scan(cnt, s_w, total);
  if (tid < K) {
    kw.start[tid] = sd.begin + excl;
    unsigned run = (unsigned)excl;
#pragma unroll
    for (unsigned st = 0; st < KW_STRIPES; ++st) {
      kw.cnt[st][tid] = run;
      run += c[st];
    }
  }
  if (tid == 0) {
    kw.start[K] = sd.begin + total;
    if (sd.begin + total != sd.end) guard_failed(a, GUARD_BOUNDS);
    a.segs[sid].tiles_done = 0;
    atomicAdd(&a.hdr->keys_counted, sd.end - sd.begin);
    const unsigned long long q0 = atomicAdd(&a.hdr->tail, (unsigned long long)sd.ntiles);
    rs.q0 = q0;
    rs.ok = q0 + sd.ntiles <= a.cap_q && sd.begin + total == sd.end;
    if (q0 + sd.ntiles > a.cap_q) raise_error(a, ERR_INTERNAL);
  }
  __syncthreads();
  if (rs.ok) publish_items(a, rs.q0, sd.ntiles, ITEM_VALID | ((unsigned long long)sid << 32) | ITEM_PHASE);
  __syncthreads();
}

// After the scatter pass of a K-way range: its buckets are the children, one
// per thread. Leaves and fallback ranges are listed here; every larger child
// becomes a setup item, so up to 256 children are sampled by as many blocks.
__device__ void finish_kway_scatter(const SortArgs &a, const SegDesc &sd, unsigned sid,
                                    unsigned long long *s_w) {
  if (a.test_stall && sid == 0) return;   // test hook: children never appear
  const KwayDesc &kw = a.kw[sd.piv_lo];
  const unsigned K = (unsigned)sd.piv_hi;
  const bool eqm = __ldcg(&kw.eqmode) != 0;
  const unsigned tid = threadIdx.x;
  const unsigned parity = (sd.flags & SEG_PARITY) ^ 1u;
  const unsigned d1 = sd.depth + 1;
  const uint64_t m = sd.end - sd.begin;
  if (tid == 0) {
    atomicAdd(&a.hdr->keys_partitioned, m);
    atomicAdd(&a.hdr->tiles, (unsigned long long)(sd.ntiles + kw_count_items(sd.ntiles)));
    atomicAdd(&a.hdr->segments, 1ull);
    atomicAdd(&a.hdr->kway_ranges, 1ull);
    atomicMax(&a.hdr->max_depth, (unsigned long long)d1);
  }
  unsigned long long handed = 0, setup = 0;
  bool nokway = false;
  if (tid < K) {
    const uint64_t cb = __ldcg(&kw.start[tid]), ce = __ldcg(&kw.start[tid + 1]);
    if (ce < cb || cb < sd.begin || ce > sd.end) {
      guard_failed(a, GUARD_BOUNDS);
    } else if (ce > cb) {
      const uint64_t mc = ce - cb;
      if (eqm && (tid & 1)) {
        // keys equal to one splitter: only decoded and copied, in pieces of
        // at most the cutoff
        const unsigned C = a.leaf_cutoff;
        const unsigned ne = (unsigned)((mc + C - 1) / C);
        const unsigned long long i0 = atomicAdd(&a.hdr->n_leaf_block, (unsigned long long)ne);
        if (i0 + ne <= a.cap_leaf_block) {
          for (unsigned q = 0; q < ne; ++q) {
            const uint64_t pb = cb + (uint64_t)q * C;
            a.leaf_block[i0 + q] = LeafEntry{pb, (unsigned)min((uint64_t)C, ce - pb), parity | LEAF_COPY};
          }
          atomicAdd(&a.hdr->equal_ranges, 1ull);
          atomicAdd(&a.hdr->equal_keys, mc);
        } else {
          raise_error(a, ERR_INTERNAL);
        }
        handed = mc;
      } else if (mc <= a.leaf_cutoff) {
        const LeafList L = leaf_list(a, mc);
        const unsigned long long i = atomicAdd(L.n, 1ull);
        if (i < L.cap) {
          L.list[i] = LeafEntry{cb, (unsigned)mc, parity};
          atomicAdd(L.stat, 1ull);
          atomicAdd(&a.hdr->leaf_keys, mc);
          atomicAdd(L.keys, mc);
        } else {
          raise_error(a, ERR_INTERNAL);
        }
        handed = mc;
      } else if (d1 >= sd.depth_limit) {
        const unsigned long long i = atomicAdd(&a.hdr->n_fb, 1ull);
        if (i < a.cap_fb) {
          a.fb[i] = LeafEntry{cb, (unsigned)mc, parity};
          atomicAdd(&a.hdr->fallback_ranges, 1ull);
          atomicAdd(&a.hdr->fallback_keys, mc);
        } else {
          raise_error(a, ERR_INTERNAL);
        }
        handed = mc;
      } else {
        setup = 1;
        nokway = mc == m;   // the split made no progress: split this one in two
      }
    }
  }
  unsigned long long nsetup, handed_total;
  const unsigned long long pos = block_excl_scan(setup, s_w, nsetup);
  block_excl_scan(handed, s_w, handed_total);
  __shared__ unsigned long long s_q0;
  if (tid == 0) {
    unsigned long long q0 = nsetup ? atomicAdd(&a.hdr->tail, nsetup) : 0ull;
    if (nsetup && q0 + nsetup > a.cap_q) {
      raise_error(a, ERR_INTERNAL);
      q0 = ~0ull;
    }
    s_q0 = q0;
  }
  __syncthreads();
  if (setup && s_q0 != ~0ull)
    st_release(&a.items[s_q0 + pos], ITEM_VALID | ((unsigned long long)sid << 32) | ITEM_SETUP |
                                         (nokway ? ITEM_NOKWAY : 0ull) | tid);
  __syncthreads();
  if (tid == 0 && handed_total) atomicAdd(&a.hdr->remaining, 0ull - handed_total);
}

// A setup item: child j of range pd (id psid) becomes a partitioned range.
template <int KB, unsigned R>
__device__ void setup_child(const SortArgs &a, const SegDesc &pd, unsigned psid, unsigned j, bool allow_kway,
                            void *scratch, RangeScratch &rs) {
  uint64_t cb, ce;
  if (pd.flags & SEG_KWAY) {
    const KwayDesc &kw = a.kw[pd.piv_lo];
    cb = __ldcg(&kw.start[j]);
    ce = __ldcg(&kw.start[j + 1]);
  } else {
    const uint64_t L = ld_relaxed(&a.segs[psid].cursor) & 0xFFFFFFFFull;
    cb = j ? pd.begin + L : pd.begin;
    ce = j ? pd.end : pd.begin + L;
  }
  const unsigned parity = (pd.flags & SEG_PARITY) ^ 1u;
  const unsigned d1 = pd.depth + 1, limit = pd.depth_limit;
  if (ce <= cb || ce > a.n_total) {   // guard (uniform: every thread read the same bounds)
    if (threadIdx.x == 0) guard_failed(a, GUARD_BOUNDS);
    return;
  }
  start_range<KB, R>(a, cb, ce, d1, parity, limit, allow_kway, scratch, rs);
}

// Everything Algorithm 1 does after Partition returned, for range `sd`.
template <int KB>
__device__ void finish_range(const SortArgs &a, const SegDesc &sd, unsigned sid, void *scratch,
                             RangeScratch &rs) {
  using C = typename KT<KB>::Code;
  const uint64_t b = sd.begin, e = sd.end, m = e - b;
  const uint64_t L = ld_relaxed(&a.segs[sid].cursor) & 0xFFFFFFFFull;
  if (a.mode == MODE_PARTITION) {
    if (threadIdx.x == 0) {
      *a.out_left = L;
      st_release(&a.hdr->remaining, 0);
    }
    return;
  }
  if (a.test_stall && sid == 0) return;   // test hook: children never appear
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
    handed += child_range<KB>(a, b, b + L, d1, parity, sd.depth_limit, scratch, rs, sid, 0);
    emit_equal(a, b + L, e - (b + L), parity, rs);
    handed += e - (b + L);
  } else if (L == m) {
    // Degenerate partition (Algorithm 1): every key <= pivot.
    if (threadIdx.x == 0) atomicAdd(&a.hdr->degenerate, 1ull);
    if (!ld_relaxed32(&a.segs[sid].has_lt)) {
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
    handed += child_range<KB>(a, b, b + L, d1, parity, sd.depth_limit, scratch, rs, sid, 0);
    handed += child_range<KB>(a, b + L, e, d1, parity, sd.depth_limit, scratch, rs, sid, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && handed) atomicAdd(&a.hdr->remaining, (unsigned long long)(0ull - handed));
}

// ---------------------------------------------------------------------------
// Work claiming.
// ---------------------------------------------------------------------------

// Thread 0: waits (bounded) for the item of an already claimed ticket.
// Returns 0 when all keys are placed, on abort, or on a timeout.
__device__ int wait_ticket(const SortArgs &a, unsigned long long t, unsigned long long &item) {
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

// Thread 0: is the item of ticket t already published?
__device__ __forceinline__ bool probe_ticket(const SortArgs &a, unsigned long long t, unsigned long long &item) {
  if (t >= a.cap_q) return false;
  const unsigned long long v = ld_acquire(&a.items[t]);
  if (v & ITEM_VALID) {
    item = v;
    return true;
  }
  return false;
}

template <int KB> __device__ __forceinline__ typename KT<KB>::Mem to_mem(typename KT<KB>::Code c) {
  if constexpr (KB == KV_KEYONLY) return U128{c.lo, c.hi};
  else if constexpr (KB == 16) return c;
  else return (typename KT<KB>::Mem)c;
}

// Pass 1 over the tile window: left keys (code <= pivot), valid keys, and
// whether some key is < pivot. Chunks fully inside the tile skip the
// per-key bounds test.
template <int KB, int CPT, bool RAW>
__device__ __forceinline__ void count_tile(const SortArgs &a, const uint4 *__restrict__ sw, unsigned nwc, unsigned lo,
                                           unsigned hi, typename KT<KB>::Code piv, unsigned &nL,
                                           unsigned &nV, int &anyLt) {
  using C = typename KT<KB>::Code;
  constexpr unsigned V = 16 / kmem(KB);
#pragma unroll 2
  for (int j = 0; j < CPT; ++j) {
    const unsigned c = threadIdx.x + j * NT;
    const uint4 q = c < nwc ? sw[c] : make_uint4(0, 0, 0, 0);
    const bool full = 16 * c >= lo && 16 * c + 16 <= hi;
#pragma unroll
    for (unsigned v = 0; v < V; ++v) {
      const unsigned off = 16 * c + v * kmem(KB);
      const bool valid = full || (off >= lo && off < hi);
      C k = key_at<KB>(q, v);
      if (RAW) k = encode<KB>(k, a.codec);
      nL += (valid && !lt(piv, k));
      nV += valid;
      anyLt |= (valid && lt(k, piv));
    }
  }
}

// Pass 2 over the tile window: every valid key goes to its ballot rank in
// the left run (outL) or the right run (outR).
template <int KB, int CPT, bool RAW, bool DEC>
__device__ __forceinline__ void scatter_tile(const SortArgs &a, const uint4 *__restrict__ sw, unsigned nwc,
                                             unsigned lo, unsigned hi, typename KT<KB>::Code piv,
                                             typename KT<KB>::Mem *__restrict__ outL,
                                             typename KT<KB>::Mem *__restrict__ outR,
                                             unsigned runL, unsigned runR) {
  using C = typename KT<KB>::Code;
  constexpr unsigned V = 16 / kmem(KB);
  const unsigned lane = threadIdx.x & 31;
  const unsigned ltm = (1u << lane) - 1u;
#pragma unroll 2
  for (int j = 0; j < CPT; ++j) {
    const unsigned c = threadIdx.x + j * NT;
    const uint4 q = c < nwc ? sw[c] : make_uint4(0, 0, 0, 0);
    const bool full = 16 * c >= lo && 16 * c + 16 <= hi;
#pragma unroll
    for (unsigned v = 0; v < V; ++v) {
      const unsigned off = 16 * c + v * kmem(KB);
      const bool valid = full || (off >= lo && off < hi);
      C k = key_at<KB>(q, v);
      if (RAW) k = encode<KB>(k, a.codec);
      const bool le = !lt(piv, k);
      const unsigned bl = __ballot_sync(FULL, valid && le), br = __ballot_sync(FULL, valid && !le);
      if (valid) {
        const typename KT<KB>::Mem out = to_mem<KB>(DEC ? decode<KB>(k, a.codec) : k);
        if (le) outL[runL + __popc(bl & ltm)] = out;
        else outR[runR + __popc(br & ltm)] = out;
      }
      runL += __popc(bl);
      runR += __popc(br);
    }
  }
}

// Counting pass over a K-way counting tile, the keys of two scatter tiles
// (2 x KCPT chunks per thread): every key adds one to its bucket in the
// histogram of the scatter tile that will move it (h0 for the first TK keys,
// h1 for the rest), and its bucket is stored for the scatter pass. A scatter
// tile holds TK keys, TK x KB = NT x KCPT x 16 - 16 bytes, so only the chunks
// of j = KCPT - 1 can hold keys of both.
template <int KB, int KCPT, bool RAW>
__device__ __forceinline__ void kw_count_tile(const SortArgs &a, const uint4 *__restrict__ sw, unsigned nwc,
                                              unsigned lo, unsigned hi, const KwLookup<typename KT<KB>::Code> &cl,
                                              unsigned *__restrict__ h0, unsigned *__restrict__ h1,
                                              unsigned char *__restrict__ ids) {
  using C = typename KT<KB>::Code;
  constexpr unsigned V = 16 / kmem(KB);
  constexpr unsigned TK = kw_tile_keys(KB, 2 * KCPT);
  static_assert(TK * kmem(KB) == NT * KCPT * 16 - 16, "scatter tile size");
  const unsigned split = lo + TK * kmem(KB);   // first byte of the second scatter tile
#pragma unroll
  for (int j = 0; j < 2 * KCPT; ++j) {
    const unsigned c = threadIdx.x + j * NT;
    if (c < nwc) {
      const uint4 q = sw[c];
      const bool full = 16 * c >= lo && 16 * c + 16 <= hi;
#pragma unroll
      for (unsigned v = 0; v < V; ++v) {
        const unsigned off = 16 * c + v * kmem(KB);
        if (full || (off >= lo && off < hi)) {
          C k = key_at<KB>(q, v);
          if (RAW) k = encode<KB>(k, a.codec);
          const unsigned bk = cl(k);
          unsigned *h = j < KCPT - 1 ? h0 : j >= KCPT ? h1 : (off < split ? h0 : h1);
          atomicAdd(&h[bk], 1u);
          ids[(off - lo) / kmem(KB)] = (unsigned char)bk;   // for the scatter pass
        }
      }
    }
  }
}

// Scatter pass over a K-way tile window. (1) Each key takes the next rank in
// its bucket (stored by the counting pass, copied to s_ids) from the shared
// histogram. (2) One thread per bucket turns the
// tile's counts into offsets of the bucket-ordered tile and reserves the
// bucket's slots in the range with one atomic. (3) Keys are staged in bucket
// order in the second half of the window. (4) The staged tile is written out
// with consecutive threads on consecutive keys, so each bucket's keys leave
// as one contiguous run.
template <int KB, int KCPT, bool RAW>
__device__ __forceinline__ void kw_scatter_tile(const SortArgs &a, const uint4 *__restrict__ sw, unsigned nwc,
                                                unsigned lo, unsigned hi, const unsigned char *__restrict__ s_ids,
                                                unsigned K, KwayDesc &kw, unsigned stripe, uint64_t rbegin,
                                                typename KT<KB>::Mem *__restrict__ dst,
                                                typename KT<KB>::Mem *__restrict__ stage,
                                                unsigned char *__restrict__ sb, unsigned *__restrict__ s_hist,
                                                unsigned short *__restrict__ s_tstart,
                                                unsigned *__restrict__ s_off, unsigned long long *s_w) {
  using C = typename KT<KB>::Code;
  constexpr unsigned V = 16 / kmem(KB), Q = KCPT * V;
  const unsigned tid = threadIdx.x;
  uint32_t pk[Q];   // rank << 8 | bucket, ~0 for no key
#pragma unroll
  for (int j = 0; j < KCPT; ++j) {
    const unsigned c = tid + j * NT;
#pragma unroll
    for (unsigned v = 0; v < V; ++v) pk[j * V + v] = ~0u;
    if (c < nwc) {
      const bool full = 16 * c >= lo && 16 * c + 16 <= hi;
#pragma unroll
      for (unsigned v = 0; v < V; ++v) {
        const unsigned off = 16 * c + v * kmem(KB);
        if (full || (off >= lo && off < hi)) {
          const unsigned bk = s_ids[(off - lo) / kmem(KB)];
          pk[j * V + v] = (atomicAdd(&s_hist[bk], 1u) << 8) | bk;
        }
      }
    }
  }
  __syncthreads();
  const unsigned cnt = tid < K ? s_hist[tid] : 0u;
  unsigned long long nkeys;
  const unsigned long long excl = block_excl_scan(cnt, s_w, nkeys);
  // the bucket's slots are reserved now; the atomic's result is first used
  // after the staging below, so its round trip overlaps the staging
  unsigned rel = 0;
  unsigned long long lim = 0;
  if (tid < K) {
    s_tstart[tid] = (unsigned short)excl;
    if (cnt) {
      rel = atomicAdd(&kw.cnt[stripe][tid], cnt);
      lim = __ldcg(&kw.start[tid + 1]);   // the bucket's end, for the guard below
    }
    s_hist[tid] = 0;   // ready for the next tile
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < KCPT; ++j) {
    const unsigned c = tid + j * NT;
    if (c < nwc) {
      const uint4 q = sw[c];
#pragma unroll
      for (unsigned v = 0; v < V; ++v) {
        const uint32_t p = pk[j * V + v];
        if (p != ~0u) {
          C k = key_at<KB>(q, v);
          if (RAW) k = encode<KB>(k, a.codec);
          const unsigned bk = p & 255u, pos = s_tstart[bk] + (p >> 8);
          stage[pos] = to_mem<KB>(k);
          sb[pos] = (unsigned char)bk;
        }
      }
    }
  }
  if (tid < K) {
    // staged position p of this bucket goes to rbegin + off + p
    unsigned off = 0;
    if (cnt) {
      if (rbegin + rel + cnt > lim) {   // guard: stay inside the bucket
        guard_failed(a, GUARD_BUCKET);
        off = ~0u;
      } else {
        off = rel - (unsigned)excl;   // rel >= excl: earlier buckets fill the tile's first slots
      }
    }
    s_off[tid] = off;
  }
  __syncthreads();
  typename KT<KB>::Mem *__restrict__ out = dst + rbegin;
#pragma unroll 4
  for (unsigned p = tid; p < (unsigned)nkeys; p += NT) {
    const unsigned off = s_off[sb[p]];
    if (off != ~0u) out[off + p] = stage[p];
  }
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
  constexpr unsigned R = kw_sample_r<KB, 8>();
  __shared__ RangeScratch rs;
  __shared__ __align__(16) unsigned char scratch[kw_scratch_bytes<KB, R>()];
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
    if (m <= 1) {   // one key in input form is already sorted
      if (m == 1 && a.out != a.keys && threadIdx.x == 0) store_key<KB>(a.out, b, load_cg<KB>(a.keys, b));
      continue;
    }
    const unsigned limit =
        a.depth_override >= 0 ? (unsigned)a.depth_override : 2 * floor_log2_u64(m) + 4;
    if (m <= a.leaf_cutoff) {
      emit_leaf(a, b, m, SEG_RAW, rs);
    } else if (limit == 0) {
      emit_fallback(a, b, m, SEG_RAW, rs);
    } else {
      if (threadIdx.x == 0) atomicAdd(&a.hdr->remaining, m);
      start_range<KB, R>(a, b, e, 0, SEG_RAW, limit, true, scratch, rs);
    }
    __syncthreads();
  }
}

// Loads the descriptor of `item`'s range (through L2) into `seg`.
__device__ __forceinline__ void load_desc(const SortArgs &a, unsigned long long item, SegDesc &seg) {
  const unsigned sid = (unsigned)((item >> 32) & 0x7FFFFFFFu);
  const unsigned long long *d = (const unsigned long long *)&a.segs[sid];
  unsigned long long w[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) w[k] = __ldcg(d + k);
  unsigned long long *sw = (unsigned long long *)&seg;
#pragma unroll
  for (int k = 0; k < 8; ++k) sw[k] = w[k];
}

// Keys per tile of a range's item: K-way counting tiles cover two scatter
// tiles.
__device__ __forceinline__ unsigned tile_keys_of(const SortArgs &a, const SegDesc &seg,
                                                 unsigned long long item) {
  if (!(seg.flags & SEG_KWAY)) return a.tile_keys;
  return (item & ITEM_PHASE) ? a.kw_tile_keys : 2 * a.kw_tile_keys;
}

// Starts the TMA bulk copy of the tile's 16-byte-aligned window into `buf`.
// The window may include up to 15 bytes on each side that belong to
// neighbouring ranges; they are never used (and never cross a page). A K-way
// scatter tile also copies its keys' buckets (one byte each, aligned the same
// way) into the second half of the window, which is free until staging.
template <int KB, int CPT>
__device__ __forceinline__ void issue_tile(const SortArgs &a, unsigned long long item, const SegDesc &seg,
                                           unsigned char *buf, uint64_t *bar) {
  const unsigned T = tile_keys_of(a, seg, item);
  const unsigned i = (unsigned)(item & ITEM_INDEX);
  const uint64_t b = seg.begin, e = seg.end;
  const bool par = seg.flags & SEG_PARITY;
  const unsigned char *src = (const unsigned char *)(par ? a.alt : a.keys);
  const uint64_t t0 = b + (uint64_t)i * T;
  if (t0 >= e || e > a.n_total) {   // guard: never copy outside the array
    guard_failed(a, GUARD_TILE);
    mbar_arrive_expect_tx(bar, 0);
    return;
  }
  const unsigned cnt = (unsigned)min((uint64_t)T, e - t0);
  const uintptr_t g0 = (uintptr_t)(src + t0 * kmem(KB)), g1 = g0 + (uintptr_t)cnt * kmem(KB);
  const uintptr_t w0 = g0 & ~(uintptr_t)15, w1 = (g1 + 15) & ~(uintptr_t)15;
  fence_proxy_async_global();
  if ((seg.flags & SEG_KWAY) && (item & ITEM_PHASE)) {
    const uintptr_t i0 = (uintptr_t)(a.kw_ids + t0) & ~(uintptr_t)15;
    const uintptr_t i1 = ((uintptr_t)(a.kw_ids + t0 + cnt) + 15) & ~(uintptr_t)15;
    mbar_arrive_expect_tx(bar, (uint32_t)((w1 - w0) + (i1 - i0)));
    bulk_load(buf, (const void *)w0, (uint32_t)(w1 - w0), bar);
    bulk_load(buf + part_window(CPT) / 2, (const void *)i0, (uint32_t)(i1 - i0), bar);
    return;
  }
  mbar_arrive_expect_tx(bar, (uint32_t)(w1 - w0));
  bulk_load(buf, (const void *)w0, (uint32_t)(w1 - w0), bar);
}

// Thread 0, after a claim: the item goes to s_item, its range descriptor to
// s_seg (kept while consecutive tiles share a range), and a tile's copy is
// started. A setup item loads its parent's descriptor and copies nothing.
template <int KB, int CPT>
__device__ __forceinline__ void prepare(const SortArgs &a, unsigned long long item, unsigned long long &s_item,
                                        SegDesc &s_seg, unsigned &seg_in_smem, int &s_newtree,
                                        unsigned char *buf, uint64_t *bar) {
  s_item = item;
  s_newtree = 0;
  const unsigned sid = (unsigned)((item >> 32) & 0x7FFFFFFFu);
  if (item & ITEM_SETUP) {
    load_desc(a, item, s_seg);
    seg_in_smem = ~0u;
    return;
  }
  if (sid != seg_in_smem) {
    load_desc(a, item, s_seg);
    seg_in_smem = sid;
    s_newtree = (s_seg.flags & SEG_KWAY) != 0;
  }
  issue_tile<KB, CPT>(a, item, s_seg, buf, bar);
}

// The persistent partition kernel. Per two-way tile: one TMA copy into the
// shared window, a counting pass, one atomic on the range's write cursors
// that reserves this tile's slots on both sides (the GPU form of the
// bidirectional write positions of Sec. 2.1: the order of keys within a side
// is free, so tiles need not wait for one another), and a scatter pass that
// writes every key straight from its ballot rank to global memory (each warp
// store is two contiguous runs). K-way tiles count or scatter by bucket
// (kw_count_tile, kw_scatter_tile); setup items start a child range. A block
// needs only the window and few registers, so several blocks per SM keep
// enough bytes in flight.
template <int KB, int CPT>
__global__ void __launch_bounds__(NT, part_blocks_per_sm(CPT)) k_partition(SortArgs a) {
  using C = typename KT<KB>::Code;
  using M = typename KT<KB>::Mem;
  constexpr int KCPT = kw_cpt(KB, CPT);
  constexpr unsigned TKW = kw_tile_keys(KB, CPT);
  constexpr unsigned RS = kw_sample_r<KB, CPT>();
  static_assert(kw_scratch_bytes<KB, RS>() <= (unsigned)part_window(CPT), "setup sample fits the window");
  static_assert(2 * TKW * kmem(KB) + 32 <= (unsigned)part_window(CPT), "a counting tile fits the window");
  static_assert(NT == KW_MAX, "one thread per bucket");
  constexpr unsigned PIV_BYTES = SAMPLE * sizeof(C) + SAMPLE / (64 / kmem(KB)) * 8;
  constexpr unsigned LOOKUP_BYTES = KW_MAX * sizeof(C) + KW_TABLE * 2;
  constexpr unsigned AUX = PIV_BYTES > LOOKUP_BYTES ? PIV_BYTES : LOOKUP_BYTES;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t s_bar;
  __shared__ SegDesc s_seg, s_fseg;
  __shared__ unsigned long long s_item, s_ticket;
  __shared__ unsigned s_fsid, s_fphase;
  __shared__ int s_go, s_go2, s_fin, s_newtree;
  __shared__ unsigned s_wL[NWARP], s_wV[NWARP], s_bL[NWARP], s_bR[NWARP];
  __shared__ unsigned long long s_cur;
  __shared__ RangeScratch rs;
  // finishers' pivot samples, and the bucket lookup of K-way tiles (reloaded
  // after a finisher ran)
  __shared__ __align__(16) unsigned char s_aux[AUX];
  __shared__ unsigned s_hist[KW_MAX];
  __shared__ unsigned short s_tstart[KW_MAX];
  __shared__ unsigned s_off[KW_MAX];
  __shared__ unsigned long long s_w[NWARP];
  __shared__ unsigned char s_sb[TKW];
  __shared__ unsigned s_shift, s_nsp, s_eqm;
  C *s_split = (C *)s_aux;
  unsigned short *s_table = (unsigned short *)(s_aux + KW_MAX * sizeof(C));
  M *stage = (M *)(smem + part_window(CPT) / 2);

  const unsigned tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (unsigned j = tid; j < KW_MAX; j += NT) {
    s_hist[j] = 0;
    s_off[j] = 0;
  }
  if (blockIdx.x == 0 && tid == 0) a.hdr->part_grid = gridDim.x;
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;
  // Thread 0 state: the range whose descriptor is in s_seg, the next ticket
  // (claimed while the current tile runs) and its queue word, read before the
  // tile's last barrier so that the read overlaps the barrier.
  unsigned seg_in_smem = ~0u;
  bool nclaimed = false;
  unsigned long long nticket = 0, nword = 0;
  // Thread FT state: the last tile's release add on its range's completion
  // count, whose result FT reads at the next claim while thread 0 claims.
  constexpr unsigned FT = NT - 32;
  unsigned pend_sid = ~0u, pend_nt = 0, pend_phase = 0;
  uint32_t pend_prev = 0;

  for (;;) {
    if (tid == 0) {
      const unsigned long long t = nclaimed ? nticket : atomicAdd(&a.hdr->head, 1ull);
      unsigned long long item = 0;
      bool have;
      if (nclaimed && (nword & ITEM_VALID)) {
        item = nword;
        have = true;
      } else {
        have = probe_ticket(a, t, item);
      }
      nclaimed = false;
      if (have) prepare<KB, CPT>(a, item, s_item, s_seg, seg_in_smem, s_newtree, smem, &s_bar);
      s_go = have;
      s_ticket = t;
    }
    if (tid == FT) {
      int fin = 0;
      if (pend_sid != ~0u) {
        fin = pend_prev == pend_nt - 1;
        if (fin) {
          fence_acquire();
          s_fsid = pend_sid;
          s_fphase = pend_phase;
          load_desc(a, (unsigned long long)pend_sid << 32, s_fseg);
        }
        pend_sid = ~0u;
      }
      s_fin = fin;
    }
    __syncthreads();
    // the previous tile finished its range: the rest of Algorithm 1 for it
    if (s_fin) {
      if (!(s_fseg.flags & SEG_KWAY)) finish_range<KB>(a, s_fseg, s_fsid, s_aux, rs);
      else if (!s_fphase) finish_kway_count(a, s_fseg, s_fsid, rs, s_w);
      else finish_kway_scatter(a, s_fseg, s_fsid, s_w);
    }
    if (!s_go) {
      // the claimed item is not published yet (it may come from the range
      // just finished above): wait for it. The outcome goes to s_go2, not
      // s_go: other warps may still be reading s_go for the test above, and
      // a warp that saw it change would skip this block's barrier.
      if (tid == 0) {
        unsigned long long item = 0;
        const int go = wait_ticket(a, s_ticket, item);
        if (go) prepare<KB, CPT>(a, item, s_item, s_seg, seg_in_smem, s_newtree, smem, &s_bar);
        s_go2 = go;
      }
      __syncthreads();
      if (!s_go2) break;
    }

    const unsigned long long item = s_item;
    const SegDesc &sg = s_seg;
    const unsigned sid = (unsigned)((item >> 32) & 0x7FFFFFFFu);
    const unsigned i = (unsigned)(item & ITEM_INDEX);
    if (item & ITEM_SETUP) {
      // no copy was started: the window is free scratch for the sample
      setup_child<KB, RS>(a, sg, sid, i, (item & ITEM_NOKWAY) == 0, smem, rs);
      continue;
    }
    const bool kway = sg.flags & SEG_KWAY;
    if (kway && (s_newtree || s_fin)) {
      const KwayDesc &kw = a.kw[sg.piv_lo];
      for (unsigned j = tid; j < KW_MAX; j += NT)
        s_split[j] = code_of<KB>(__ldcg(&kw.split_lo[j]), kmem(KB) == 16 ? __ldcg(&kw.split_hi[j]) : 0ull);
      for (unsigned j = tid; j < KW_TABLE / 2; j += NT)
        ((unsigned *)s_table)[j] = __ldcg((const unsigned *)kw.table + j);
      if (tid == 0) {
        s_shift = __ldcg(&kw.shift);
        s_nsp = __ldcg(&kw.nsplit);
        s_eqm = __ldcg(&kw.eqmode);
      }
      __syncthreads();
    }
    {
      unsigned it = 0;
      while (!mbar_try_wait(&s_bar, phase)) {
        if (++it > a.spin_limit) {   // a copy that never lands: give up (cannot happen for valid addresses)
          if (tid == 0) raise_error(a, ERR_TIMEOUT);
          break;
        }
      }
      phase ^= 1;
    }
    if (tid == 0) {   // its result is first used at the next claim
      nticket = atomicAdd(&a.hdr->head, 1ull);
      nclaimed = true;
    }

    const bool phase1 = (item & ITEM_PHASE) != 0;
    const unsigned T = kway ? (phase1 ? TKW : 2 * TKW) : a.tile_keys;
    const uint64_t b = sg.begin, e = sg.end;
    const bool par = sg.flags & SEG_PARITY, raw = sg.flags & SEG_RAW;
    const unsigned char *src = (const unsigned char *)(par ? a.alt : a.keys);
    M *dst = (M *)(par ? a.keys : a.alt);
    const uint64_t t0 = b + (uint64_t)i * T;
    const unsigned cnt = (unsigned)min((uint64_t)T, e - t0);
    const uintptr_t g0 = (uintptr_t)(src + t0 * kmem(KB)), g1 = g0 + (uintptr_t)cnt * kmem(KB);
    const uintptr_t w0 = g0 & ~(uintptr_t)15;
    const unsigned nwc = (unsigned)((((g1 + 15) & ~(uintptr_t)15) - w0) / 16);
    const unsigned lo = (unsigned)(g0 - w0), hi = (unsigned)(g1 - w0);
    const uint4 *sw = (const uint4 *)smem;

    if (kway) {
      KwayDesc &kw = a.kw[sg.piv_lo];
      const unsigned K = (unsigned)sg.piv_hi;   // buckets
      KwLookup<C> cl;
      cl.split = s_split;
      cl.table = s_table;
      cl.nsp = s_nsp;
      cl.eqb = s_eqm;
      cl.s1 = s_split[1];
      cl.sk = s_split[s_nsp];
      cl.sh = s_shift;
      if (!phase1) {
        // s_off (free outside a scatter tile) holds the second histogram
        if (raw) kw_count_tile<KB, KCPT, true>(a, sw, nwc, lo, hi, cl, s_hist, s_off, a.kw_ids + t0);
        else kw_count_tile<KB, KCPT, false>(a, sw, nwc, lo, hi, cl, s_hist, s_off, a.kw_ids + t0);
        __syncthreads();
        if (tid < K) {   // each half counts for the stripe of its scatter tile, 2i or 2i + 1
          const unsigned x0 = s_hist[tid], x1 = s_off[tid];
          if (x0) atomicAdd(&kw.cnt[(2 * i) % KW_STRIPES][tid], x0);
          if (x1) atomicAdd(&kw.cnt[(2 * i + 1) % KW_STRIPES][tid], x1);
          s_hist[tid] = 0;
          s_off[tid] = 0;
        }
      } else {
        const unsigned char *s_ids =
            (const unsigned char *)stage + ((uintptr_t)(a.kw_ids + t0) & 15);   // copied with the keys
        if (raw)
          kw_scatter_tile<KB, KCPT, true>(a, sw, nwc, lo, hi, s_ids, K, kw, i % KW_STRIPES, b, dst, stage,
                                          s_sb, s_hist, s_tstart, s_off, s_w);
        else
          kw_scatter_tile<KB, KCPT, false>(a, sw, nwc, lo, hi, s_ids, K, kw, i % KW_STRIPES, b, dst, stage,
                                           s_sb, s_hist, s_tstart, s_off, s_w);
      }
      const unsigned fnt = phase1 ? sg.ntiles : kw_count_items(sg.ntiles);   // s_seg changes after the barrier
      if (tid == 0) nword = nticket < a.cap_q ? ld_acquire(&a.items[nticket]) : 0ull;
      fence_proxy_async_smem();   // the next TMA copy reuses the window
      __syncthreads();
      // a scatter tile leaves its bucket offsets in s_off: clear them for the
      // next counting tile (ordered before it by the barrier after the claim)
      if (phase1) s_off[tid] = 0;
      if (tid == FT) {
        pend_prev = atom_add_release(&a.segs[sid].tiles_done, 1u);
        pend_sid = sid;
        pend_nt = fnt;
        pend_phase = phase1;
      }
      continue;
    }

    const C piv = code_of<KB>(sg.piv_lo, sg.piv_hi);
    // ---- pass 1: per-warp counts of left and valid keys
    unsigned nL = 0, nV = 0;
    int anyLt = 0;
    if (raw) count_tile<KB, CPT, true>(a, sw, nwc, lo, hi, piv, nL, nV, anyLt);
    else count_tile<KB, CPT, false>(a, sw, nwc, lo, hi, piv, nL, nV, anyLt);
    nL = __reduce_add_sync(FULL, nL);
    nV = __reduce_add_sync(FULL, nV);
    if (lane == 0) {
      s_wL[warp] = nL;
      s_wV[warp] = nV;
    }
    anyLt = __syncthreads_or(anyLt);

    // ---- block scan of warp counts, then reserve this tile's output slots
    if (warp == 0) {
      unsigned xL = lane < NWARP ? s_wL[lane] : 0, xV = lane < NWARP ? s_wV[lane] : 0;
      unsigned iL = xL, iV = xV;
#pragma unroll
      for (int o = 1; o < NWARP; o <<= 1) {
        const unsigned yL = __shfl_up_sync(FULL, iL, o), yV = __shfl_up_sync(FULL, iV, o);
        if (lane >= (unsigned)o) { iL += yL; iV += yV; }
      }
      if (lane < NWARP) {
        s_bL[lane] = iL - xL;
        s_bR[lane] = (iV - xV) - (iL - xL);
      }
      if (lane == NWARP - 1) {
        const unsigned long long add = ((unsigned long long)(iV - iL) << 32) | iL;
        unsigned long long cur = atomicAdd(&a.segs[sid].cursor, add);
        if ((cur & 0xFFFFFFFFull) + (cur >> 32) + iV > e - b) {   // guard: slots inside the range
          guard_failed(a, GUARD_BINARY);
          cur = ~0ull;
        }
        s_cur = cur;
        if (anyLt) atomicOr(&a.segs[sid].has_lt, 1u);
      }
    }
    __syncthreads();

    // ---- pass 2: ballot ranks -> direct global stores. Left keys fill the
    // range from its start, right keys from its end.
    if (s_cur != ~0ull) {
      const unsigned long long cur = s_cur;
      const unsigned tileL = s_bL[NWARP - 1] + s_wL[NWARP - 1];
      const unsigned tileR = cnt - tileL;
      M *outL = dst + b + (cur & 0xFFFFFFFFull);
      M *outR = dst + (e - (cur >> 32) - tileR);
      const unsigned runL = s_bL[warp], runR = s_bR[warp];
      if (a.mode == MODE_PARTITION) scatter_tile<KB, CPT, true, true>(a, sw, nwc, lo, hi, piv, outL, outR, runL, runR);
      else if (raw) scatter_tile<KB, CPT, true, false>(a, sw, nwc, lo, hi, piv, outL, outR, runL, runR);
      else scatter_tile<KB, CPT, false, false>(a, sw, nwc, lo, hi, piv, outL, outR, runL, runR);
    }
    const unsigned fnt = sg.ntiles;   // s_seg changes after the barrier
    if (tid == 0) nword = nticket < a.cap_q ? ld_acquire(&a.items[nticket]) : 0ull;
    fence_proxy_async_smem();   // the next TMA copy reuses the window
    __syncthreads();

    // ---- range completion: one release add by thread FT covers the whole
    // block's stores (ordered before it by the barrier above); its result is
    // read at the next claim
    if (tid == FT) {
      pend_prev = atom_add_release(&a.segs[sid].tiles_done, 1u);
      pend_sid = sid;
      pend_nt = fnt;
      pend_phase = 0;
    }
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

template <int KB, int CPT> int partition_grid() {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_partition<KB, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, part_smem(CPT));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_partition<KB, CPT>, NT, part_smem(CPT));
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
  if (a.tile_cpt == 4) {
    k_partition<KB, 4><<<partition_grid<KB, 4>(), NT, part_smem(4), s>>>(a);
  } else if (a.tile_cpt == 16) {
    k_partition<KB, 16><<<partition_grid<KB, 16>(), NT, part_smem(16), s>>>(a);
  } else {
    k_partition<KB, 8><<<partition_grid<KB, 8>(), NT, part_smem(8), s>>>(a);
  }
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
    case KV_KEYONLY: return seed_impl<KV_KEYONLY>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_partition(int kb, const SortArgs &a, cudaStream_t s) {
  switch (kb) {
    case 2: return partition_impl<2>(a, s);
    case 4: return partition_impl<4>(a, s);
    case 8: return partition_impl<8>(a, s);
    case 16: return partition_impl<16>(a, s);
    case KV_KEYONLY: return partition_impl<KV_KEYONLY>(a, s);
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
