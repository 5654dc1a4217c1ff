// Shared device/host definitions of the vqsort CUDA library: key codes,
// the order-preserving codec, memory-model and TMA helpers, and the
// workspace layout that the host driver and the kernels agree on.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vq {

// ---------------------------------------------------------------------------
// Keys in registers ("codes"): every key type is mapped to an unsigned code
// whose unsigned order is the requested sort order (Sec. 2.4 orders; IEEE
// totalOrder for floats). Kernels only ever sort codes ascending.
// ---------------------------------------------------------------------------

struct U128 {
  uint64_t lo, hi;
};

template <int KB> struct KT;
template <> struct KT<2> {   // i16 / u16: 16-bit code held in a 32-bit register
  using Code = uint32_t;
  using Mem = uint16_t;
  static __host__ __device__ Code max_code() { return 0xFFFFu; }
};
template <> struct KT<4> {
  using Code = uint32_t;
  using Mem = uint32_t;
  static __host__ __device__ Code max_code() { return 0xFFFFFFFFu; }
};
template <> struct KT<8> {
  using Code = uint64_t;
  using Mem = uint64_t;
  static __host__ __device__ Code max_code() { return ~0ull; }
};
template <> struct KT<16> {   // u128 and kv64: {lo, hi} words
  using Code = U128;
  using Mem = U128;
  static __host__ __device__ Code max_code() { return U128{~0ull, ~0ull}; }
};

// kv64 pairs ordered by the 64-bit key alone (Sec. 2.4: 64-bit keys with
// 64-bit associated data; Sec. 5: Quicksort is not stable, so pairs with
// equal keys may come out in any order). The code keeps the value in lo and
// the key in hi, and every comparison reads hi only. Kernels instantiate
// this key class as KB = KV_KEYONLY; it occupies 16 bytes of memory.
struct KV {
  uint64_t lo, hi;
};
constexpr int KV_KEYONLY = 17;
template <> struct KT<KV_KEYONLY> {
  using Code = KV;
  using Mem = U128;
  static __host__ __device__ Code max_code() { return KV{~0ull, ~0ull}; }
};

// Bytes a key of class KB occupies in memory.
__host__ __device__ constexpr int kmem(int kb) { return kb == KV_KEYONLY ? 16 : kb; }

__host__ __device__ __forceinline__ bool lt(uint32_t a, uint32_t b) { return a < b; }
__host__ __device__ __forceinline__ bool lt(uint64_t a, uint64_t b) { return a < b; }
// Algorithm 2: the upper word decides unless equal, then the lower word. On
// the device the same order is read from the borrow of the 128-bit
// subtraction a - b (four chained 32-bit subtractions): a < b exactly when it
// borrows.
__host__ __device__ __forceinline__ bool lt(const U128 &a, const U128 &b) {
#ifdef __CUDA_ARCH__
  unsigned borrow;
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "sub.cc.u32 t, %1, %5;\n\t"
      "subc.cc.u32 t, %2, %6;\n\t"
      "subc.cc.u32 t, %3, %7;\n\t"
      "subc.cc.u32 t, %4, %8;\n\t"
      "subc.u32 %0, 0, 0;\n\t"
      "}"
      : "=r"(borrow)
      : "r"((unsigned)a.lo), "r"((unsigned)(a.lo >> 32)), "r"((unsigned)a.hi), "r"((unsigned)(a.hi >> 32)),
        "r"((unsigned)b.lo), "r"((unsigned)(b.lo >> 32)), "r"((unsigned)b.hi), "r"((unsigned)(b.hi >> 32)));
  return borrow != 0;
#else
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
#endif
}
__host__ __device__ __forceinline__ bool lt(const KV &a, const KV &b) { return a.hi < b.hi; }
__host__ __device__ __forceinline__ bool eq(uint32_t a, uint32_t b) { return a == b; }
__host__ __device__ __forceinline__ bool eq(const KV &a, const KV &b) { return a.hi == b.hi; }
__host__ __device__ __forceinline__ bool eq(uint64_t a, uint64_t b) { return a == b; }
__host__ __device__ __forceinline__ bool eq(const U128 &a, const U128 &b) {
  return a.hi == b.hi && a.lo == b.lo;
}

template <class C> __device__ __forceinline__ C cmin(const C &a, const C &b) { return lt(b, a) ? b : a; }
template <class C> __device__ __forceinline__ C cmax(const C &a, const C &b) { return lt(b, a) ? a : b; }
// 32-bit codes use the integer min/max instructions directly (64-bit ones
// are slower than one compare and two selects).
__device__ __forceinline__ uint32_t cmin(const uint32_t &a, const uint32_t &b) { return umin(a, b); }
__device__ __forceinline__ uint32_t cmax(const uint32_t &a, const uint32_t &b) { return umax(a, b); }

// Compare-and-exchange: a <- min, b <- max.
template <class C> __device__ __forceinline__ void cas(C &a, C &b) {
  C lo = cmin(a, b), hi = cmax(a, b);
  a = lo;
  b = hi;
}

__device__ __forceinline__ uint32_t shfl_xor(uint32_t v, int m) { return __shfl_xor_sync(0xFFFFFFFFu, v, m); }
__device__ __forceinline__ uint64_t shfl_xor(uint64_t v, int m) { return __shfl_xor_sync(0xFFFFFFFFu, v, m); }
__device__ __forceinline__ U128 shfl_xor(const U128 &v, int m) {
  return U128{__shfl_xor_sync(0xFFFFFFFFu, v.lo, m), __shfl_xor_sync(0xFFFFFFFFu, v.hi, m)};
}
__device__ __forceinline__ KV shfl_xor(const KV &v, int m) {
  return KV{__shfl_xor_sync(0xFFFFFFFFu, v.lo, m), __shfl_xor_sync(0xFFFFFFFFu, v.hi, m)};
}
__device__ __forceinline__ KV shfl_idx(const KV &v, int l) {
  return KV{__shfl_sync(0xFFFFFFFFu, v.lo, l), __shfl_sync(0xFFFFFFFFu, v.hi, l)};
}
__device__ __forceinline__ uint32_t shfl_idx(uint32_t v, int l) { return __shfl_sync(0xFFFFFFFFu, v, l); }
__device__ __forceinline__ uint64_t shfl_idx(uint64_t v, int l) { return __shfl_sync(0xFFFFFFFFu, v, l); }
__device__ __forceinline__ U128 shfl_idx(const U128 &v, int l) {
  return U128{__shfl_sync(0xFFFFFFFFu, v.lo, l), __shfl_sync(0xFFFFFFFFu, v.hi, l)};
}

// Code one below c (c > 0): used to split "< p" from "== p" after a
// degenerate partition.
__host__ __device__ __forceinline__ uint32_t pred(uint32_t c) { return c - 1; }
__host__ __device__ __forceinline__ uint64_t pred(uint64_t c) { return c - 1; }
__host__ __device__ __forceinline__ U128 pred(const U128 &c) {
  return U128{c.lo - 1, c.lo == 0 ? c.hi - 1 : c.hi};
}
__host__ __device__ __forceinline__ KV pred(const KV &c) { return KV{c.lo, c.hi - 1}; }

// ---------------------------------------------------------------------------
// Codec: raw key bits <-> code. kind: 0 unsigned, 1 signed integer,
// 2 IEEE float, 3 kv64 (word swap so the key is the upper half).
// desc complements the code so descending becomes ascending.
// ---------------------------------------------------------------------------
struct Codec {
  int kind;
  int desc;
};

template <int KB> __host__ __device__ __forceinline__ typename KT<KB>::Code encode(typename KT<KB>::Code x, Codec cd);
template <int KB> __host__ __device__ __forceinline__ typename KT<KB>::Code decode(typename KT<KB>::Code x, Codec cd);

template <> __host__ __device__ __forceinline__ uint32_t encode<2>(uint32_t x, Codec cd) {
  if (cd.kind == 1) x ^= 0x8000u;
  if (cd.desc) x ^= 0xFFFFu;
  return x;
}
template <> __host__ __device__ __forceinline__ uint32_t decode<2>(uint32_t x, Codec cd) {
  if (cd.desc) x ^= 0xFFFFu;
  if (cd.kind == 1) x ^= 0x8000u;
  return x;
}
template <> __host__ __device__ __forceinline__ uint32_t encode<4>(uint32_t x, Codec cd) {
  if (cd.kind == 1) x ^= 0x80000000u;
  // negative floats: flip all bits; others: flip the sign bit
  if (cd.kind == 2) x ^= (uint32_t)((int32_t)x >> 31) | 0x80000000u;
  if (cd.desc) x = ~x;
  return x;
}
template <> __host__ __device__ __forceinline__ uint32_t decode<4>(uint32_t x, Codec cd) {
  if (cd.desc) x = ~x;
  if (cd.kind == 1) x ^= 0x80000000u;
  if (cd.kind == 2) x ^= (uint32_t)((int32_t)~x >> 31) | 0x80000000u;
  return x;
}
template <> __host__ __device__ __forceinline__ uint64_t encode<8>(uint64_t x, Codec cd) {
  if (cd.kind == 1) x ^= 0x8000000000000000ull;
  if (cd.kind == 2) x ^= (uint64_t)((int64_t)x >> 63) | 0x8000000000000000ull;
  if (cd.desc) x = ~x;
  return x;
}
template <> __host__ __device__ __forceinline__ uint64_t decode<8>(uint64_t x, Codec cd) {
  if (cd.desc) x = ~x;
  if (cd.kind == 1) x ^= 0x8000000000000000ull;
  if (cd.kind == 2) x ^= (uint64_t)((int64_t)~x >> 63) | 0x8000000000000000ull;
  return x;
}
template <> __host__ __device__ __forceinline__ U128 encode<16>(U128 x, Codec cd) {
  if (cd.kind == 3) x = U128{x.hi, x.lo};   // memory {key, value}: key becomes hi
  if (cd.desc) x = U128{~x.lo, ~x.hi};
  return x;
}
template <> __host__ __device__ __forceinline__ U128 decode<16>(U128 x, Codec cd) {
  if (cd.desc) x = U128{~x.lo, ~x.hi};
  if (cd.kind == 3) x = U128{x.hi, x.lo};
  return x;
}
// Key-only pairs: memory {key, value} -> code {lo = value, hi = key};
// descending complements the key (the value is complemented too and
// restored by decode).
template <> __host__ __device__ __forceinline__ KV encode<KV_KEYONLY>(KV x, Codec cd) {
  x = KV{x.hi, x.lo};
  if (cd.desc) x = KV{~x.lo, ~x.hi};
  return x;
}
template <> __host__ __device__ __forceinline__ KV decode<KV_KEYONLY>(KV x, Codec cd) {
  if (cd.desc) x = KV{~x.lo, ~x.hi};
  return KV{x.hi, x.lo};
}

// ---------------------------------------------------------------------------
// Global memory access for data written by other thread blocks of the same
// launch: go through L2 (ld.global.cg), never a possibly stale L1 line.
// ---------------------------------------------------------------------------
template <int KB> __device__ __forceinline__ typename KT<KB>::Code load_cg(const void *base, uint64_t i);
template <> __device__ __forceinline__ uint32_t load_cg<2>(const void *b, uint64_t i) {
  return __ldcg((const unsigned short *)b + i);
}
template <> __device__ __forceinline__ uint32_t load_cg<4>(const void *b, uint64_t i) {
  return __ldcg((const unsigned int *)b + i);
}
template <> __device__ __forceinline__ uint64_t load_cg<8>(const void *b, uint64_t i) {
  return __ldcg((const unsigned long long *)b + i);
}
template <> __device__ __forceinline__ U128 load_cg<16>(const void *b, uint64_t i) {
  ulonglong2 v = __ldcg((const ulonglong2 *)b + i);
  return U128{v.x, v.y};
}
template <> __device__ __forceinline__ KV load_cg<KV_KEYONLY>(const void *b, uint64_t i) {
  ulonglong2 v = __ldcg((const ulonglong2 *)b + i);
  return KV{v.x, v.y};
}

template <int KB> __device__ __forceinline__ void store_key(void *base, uint64_t i, typename KT<KB>::Code c);
template <> __device__ __forceinline__ void store_key<2>(void *b, uint64_t i, uint32_t c) { ((uint16_t *)b)[i] = (uint16_t)c; }
template <> __device__ __forceinline__ void store_key<4>(void *b, uint64_t i, uint32_t c) { ((uint32_t *)b)[i] = c; }
template <> __device__ __forceinline__ void store_key<8>(void *b, uint64_t i, uint64_t c) { ((uint64_t *)b)[i] = c; }
template <> __device__ __forceinline__ void store_key<16>(void *b, uint64_t i, U128 c) {
  ((ulonglong2 *)b)[i] = make_ulonglong2(c.lo, c.hi);
}
template <> __device__ __forceinline__ void store_key<KV_KEYONLY>(void *b, uint64_t i, KV c) {
  ((ulonglong2 *)b)[i] = make_ulonglong2(c.lo, c.hi);
}

// ---------------------------------------------------------------------------
// PTX memory-model helpers (gpu scope).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ld_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"((unsigned long long)v) : "memory");
}
__device__ __forceinline__ void st_release(unsigned long long *p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"((unsigned long long)v) : "memory");
}

// Release add (orders this thread's earlier writes, and those it has observed
// through a block barrier, before the add) returning the old value.
__device__ __forceinline__ uint32_t atom_add_release(unsigned int *p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void fence_acquire() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// The same fence used on the release side: followed by relaxed stores it
// publishes everything ordered before it (one fence for many stores).
__device__ __forceinline__ void fence_release() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------------------
// TMA bulk copy (cp.async.bulk) global -> shared with an mbarrier that
// counts the transferred bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_load(void *smem_dst, const void *gsrc, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Orders this thread's generic-proxy accesses before later async-proxy (TMA)
// accesses: of shared memory (a buffer read by threads, then refilled by a
// TMA copy) and of global memory (data written by other blocks, then read
// by a TMA copy).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Workspace layout (device memory, owned by the caller or by the library).
// ---------------------------------------------------------------------------

// Counters and status shared by every kernel of one sort call.
struct Header {
  unsigned long long head;        // next work-queue ticket to claim
  unsigned long long tail;        // next free work-queue slot
  unsigned long long remaining;   // keys still owned by live partition ranges
  unsigned long long nseg;        // segment descriptors allocated
  unsigned long long n_leaf_warp, n_leaf_block, n_fb;
  unsigned long long cur_leaf_warp, cur_leaf_block;
  unsigned long long bar_count, bar_gen;   // grid barrier of the merge fallback
  unsigned long long abort;       // set with the first error: every wait gives up
  unsigned long long error;       // first vq_status raised on the device
  // statistics
  unsigned long long keys_partitioned, tiles, segments;
  unsigned long long leaves_warp, leaves_block, leaf_keys;
  unsigned long long equal_ranges, equal_keys, degenerate;
  unsigned long long fallback_ranges, fallback_keys, max_depth;
  unsigned long long nkw;          // K-way range records allocated
  unsigned long long keys_counted; // keys read by K-way counting passes (statistics)
  unsigned long long kway_ranges;  // ranges split K ways (statistics)
  unsigned long long guard;        // first failed bounds guard (GUARD_*), 0 if none
  unsigned long long part_grid;    // blocks of the partition kernel (statistics)
  unsigned long long n_leaf_mid, cur_leaf_mid;   // mid-size leaf list
  unsigned long long leaves_mid;   // (statistics)
  unsigned long long leaf_ce;      // key comparisons of the leaf sorts (statistics)
  unsigned long long leaf_keys_warp, leaf_keys_mid, leaf_keys_block;   // keys per leaf list (statistics)
  unsigned long long pad[3];
};
static_assert(sizeof(Header) % 64 == 0, "header size");

// One range being partitioned (a node of the Quicksort recursion).
struct SegDesc {
  unsigned long long begin, end;    // key indices [begin, end)
  unsigned long long piv_lo, piv_hi;// pivot code (piv_hi only for 16-byte keys)
  unsigned long long cursor;        // write cursors (atomic): left keys written in bits
                                    // 0..31, right keys written in bits 32..63
  unsigned int depth;               // partition levels above this range
  unsigned int flags;               // SEG_* bits
  unsigned int ntiles;
  unsigned int tiles_done;          // tiles finished (atomic)
  unsigned int has_lt;              // some key < pivot was seen (atomic)
  unsigned int depth_limit;         // bound of its root range
};
static_assert(sizeof(SegDesc) == 64, "segment descriptor size");

enum : unsigned int {
  SEG_PARITY = 1u,   // keys live in the alternate buffer (else the user buffer)
  SEG_RAW = 2u,      // keys are still in input form (root ranges)
  SEG_EXCL = 4u,     // pivot is one below a repeated maximum: right side all equal
  SEG_KWAY = 16u,    // split into piv_hi buckets by the splitters of K-way record piv_lo
  SEG_NOKWAY = 32u,  // a K-way split made no progress here: split in two
};

// A range handed to the leaf or fallback kernels.
struct LeafEntry {
  unsigned long long begin;
  unsigned int len;
  unsigned int flags;   // SEG_PARITY, SEG_RAW, LEAF_COPY
};
enum : unsigned int { LEAF_COPY = 8u };   // all keys equal: decode and copy only

// Work-queue item: bit 63 valid, bits 32..62 segment id, bit 31 phase (K-way
// ranges: 0 = counting pass, 1 = scatter pass), bit 30 setup (start child
// `index` of the segment: sample it and publish its tiles), bit 29 (setup
// items) the child is split in two, bits 0..28 the tile or child index.
constexpr unsigned long long ITEM_VALID = 1ull << 63;
constexpr unsigned long long ITEM_PHASE = 1ull << 31;
constexpr unsigned long long ITEM_SETUP = 1ull << 30;
constexpr unsigned long long ITEM_NOKWAY = 1ull << 29;
constexpr unsigned long long ITEM_INDEX = (1ull << 29) - 1;

// K-way levels (multi-pivot partition of large ranges): 2^4 .. 2^8 buckets.
constexpr unsigned KW_MIN_BITS = 4;
constexpr unsigned KW_MAX_BITS = 8;
constexpr unsigned KW_MAX = 1u << KW_MAX_BITS;
// Tile i of a K-way range updates counter stripe i % KW_STRIPES, so the
// atomics of one large range spread over KW_STRIPES x 8 cache lines.
constexpr unsigned KW_STRIPES = 16;

// Buckets are looked up by KW_TABLE_BITS key bits after the prefix that the
// first and last splitter share.
constexpr unsigned KW_TABLE_BITS = 10;
constexpr unsigned KW_TABLE = 1u << KW_TABLE_BITS;

// Splitters and per-bucket counters of one K-way range (the bucket count is
// kept in the range descriptor's piv_hi).
struct KwayDesc {
  // counting pass: keys of stripe s in bucket b (atomic); then, for the
  // scatter pass, the next free slot of stripe s in bucket b, relative to the
  // range start (atomic). Ranges are shorter than 2^32 keys.
  unsigned int cnt[KW_STRIPES][KW_MAX];
  unsigned long long start[KW_MAX + 1];  // bucket bounds (key indices), set between the passes
  unsigned long long split_lo[KW_MAX];   // splitters 1..K-1, ascending
  unsigned long long split_hi[KW_MAX];   // (high words: 16-byte keys only)
  // per value p of the table bits: (number of splitters whose table bits
  // are below p) | (number equal to p) << 8
  unsigned short table[KW_TABLE];
  unsigned int shift;                    // leading bits shared by the first and last splitter
  unsigned int nsplit;                   // splitters (K - 1, or the distinct values in
                                         // equality mode)
  unsigned int eqmode;                   // equality mode: 2 * nsplit + 1 buckets, the odd
                                         // ones holding the keys equal to one splitter
  unsigned int pad;
};

// Warp leaves handle ranges up to this many keys (32 lanes x 16 keys).
constexpr unsigned WARP_LEAF_MAX = 512;
// Keys in the pivot sample (Sec. 2.2: 64-byte chunks; here 256 keys).
constexpr unsigned SAMPLE = 256;

enum : unsigned int {
  MODE_SORT = 0,
  MODE_PARTITION = 1,   // one partition only: input raw, output decoded
};

// Everything a kernel needs, passed by value.
struct SortArgs {
  void *keys;                 // user buffer (parity 0)
  void *alt;                  // alternate buffer (parity 1)
  void *out;                  // where leaves and the fallback write the sorted keys: the user
                              // buffer, or a device-accessible host buffer of the same keys
  Header *hdr;
  SegDesc *segs;
  unsigned long long *items;
  LeafEntry *leaf_warp, *leaf_mid, *leaf_block, *fb;
  KwayDesc *kw;                        // K-way range records (null: K-way levels off)
  unsigned char *kw_ids;               // bucket of each key, written by K-way counting passes
  const unsigned long long *offsets;   // CSR offsets or null (one segment)
  unsigned long long n_total;
  unsigned long long num_segments;
  unsigned long long *out_left;        // MODE_PARTITION result
  unsigned long long seed;
  unsigned int cap_q, cap_segs, cap_leaf_warp, cap_leaf_mid, cap_leaf_block, cap_fb, cap_kw;
  unsigned int mid_max;                // leaves of (WARP_LEAF_MAX, mid_max] keys go to the mid list
  unsigned int tile_keys;              // keys per partition tile
  unsigned int kw_tile_keys;           // keys per K-way tile
  unsigned int kw_min_keys;            // smallest range split K ways
  unsigned int kw_target;              // aimed-for keys per K-way bucket
  unsigned int tile_cpt;               // 16-byte chunks per thread of the partition tile window
  unsigned int leaf_threads;           // threads of a block-leaf CTA (0: 16 keys per thread)
  unsigned int leaf_cutoff;            // ranges <= this go to the leaf kernels
  int depth_override;                  // < 0: 2*floor(log2 m)+4
  unsigned int spin_limit;
  unsigned int mode;
  unsigned int test_stall;
  Codec codec;
  U128 pivot;                          // MODE_PARTITION pivot code
};

__host__ __device__ __forceinline__ unsigned floor_log2_u64(unsigned long long x) {
  unsigned r = 0;
  while (x > 1) { x >>= 1; ++r; }
  return r;
}

// Per-range seed of the SFC64 sampling stream: SplitMix64 finaliser of the
// sort seed, the range start and the depth.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}
__host__ __device__ __forceinline__ uint64_t range_seed(uint64_t seed, uint64_t begin, uint32_t depth) {
  return mix64(seed ^ mix64(begin * 0x9E3779B97F4A7C15ull + depth));
}

// Raises a device-side error (first one wins) and tells every wait to stop.
__device__ __forceinline__ void raise_error(const SortArgs &a, unsigned code) {
  atomicCAS(&a.hdr->error, 0ull, (unsigned long long)code);
  st_release(&a.hdr->abort, 1);
}

// Bounds guards: a failed guard skips the access it protects, latches
// VQ_ERR_INTERNAL and records which guard failed first.
enum : unsigned {
  GUARD_TILE = 1,       // a tile index past its range
  GUARD_BINARY = 2,     // a two-way tile's reserved slots overflow its range
  GUARD_BUCKET = 3,     // a K-way tile's reserved slots overflow a bucket
  GUARD_BOUNDS = 4,     // K-way bucket bounds outside their range
  GUARD_LEAF = 5,       // a leaf or fallback entry outside the array
};
__device__ __forceinline__ void guard_failed(const SortArgs &a, unsigned which) {
  atomicCAS(&a.hdr->guard, 0ull, (unsigned long long)which);
  raise_error(a, 6);
}

__device__ __forceinline__ bool aborted(const SortArgs &a) { return ld_relaxed(&a.hdr->abort) != 0; }

}  // namespace vq
