/*
 * CPU oracle for the vqsort hot path ("Vectorized and performance-portable
 * Quicksort", Blacher, Giesen, Sanders, Wassenberg).
 *
 * TEST INFRASTRUCTURE. This file is the plain, slow, scalar statement of what
 * the GPU library computes. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table
 * or helper with the CUDA library; the only thing both sides see is the
 * seeded input data the tests feed them.
 *
 * Passages followed (paper sections):
 *   - Sec. 2.4: ascending and descending order, 128-bit keys as two 64-bit
 *     words with the upper word compared first (Algorithm 2), 64-bit keys
 *     with 64-bit associated data.
 *   - Algorithm 1 / Sec. 2: Partition (keys <= pivot move left), the
 *     degenerate-partition rule (right side empty -> scan min/max; all equal
 *     -> done, else recurse with the first key in sort order as pivot), the
 *     base case for small ranges.
 *   - Sec. 2.2: the recursion limit 2*log2(n)+4, past which Heapsort runs;
 *     the median-of-3 network (0,2)(0,1)(1,2); SFC64 random draws and the
 *     division-free multiply-high bounded offset; 64-byte sample chunks.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - floats sort by IEEE 754 totalOrder on bit patterns:
 *     -NaN < -inf < ... < -0.0 < +0.0 < ... < +inf < +NaN, NaNs by payload.
 *   - kv64 sorts each (key, value) pair as one 128-bit number whose upper
 *     word is the key, so ties on the key order by value and the output is
 *     unique. Descending reverses the whole 128-bit order.
 *   - the recursion limit uses floor(log2 n) of the root range length and
 *     counts partition steps on the path from the root.
 *   - the base case of this scalar oracle is insertion sort on <= 16 keys
 *     (the vector base case is a sorting network; the result is the same).
 *
 * Parity: every function here is pinned by the CPU test suite against
 * brute force, library routines (numpy sort, numpy's SFC64), a totalOrder
 * comparator written from the IEEE definition, and invariants.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* Key types. The numbering is this file's own; callers map names to it. */
enum {
  OR_I16 = 0, OR_U16 = 1, OR_I32 = 2, OR_U32 = 3, OR_F32 = 4,
  OR_I64 = 5, OR_U64 = 6, OR_F64 = 7, OR_U128 = 8, OR_KV64 = 9
};

static int key_bytes(int dt) {
  switch (dt) {
    case OR_I16: case OR_U16: return 2;
    case OR_I32: case OR_U32: case OR_F32: return 4;
    case OR_I64: case OR_U64: case OR_F64: return 8;
    case OR_U128: case OR_KV64: return 16;
    default: return 0;
  }
}

/* ------------------------------------------------------------------------ */
/* Order-preserving map from a key's bit pattern to an unsigned integer.     */
/* (Sec. 2.4 orders; IEEE totalOrder reading for floats.)                   */
/* ------------------------------------------------------------------------ */

static uint64_t enc_narrow(int dt, uint64_t bits, int ascending) {
  uint64_t u;
  switch (dt) {
    case OR_U16: u = bits & 0xFFFFu; break;
    case OR_I16: u = (bits ^ 0x8000u) & 0xFFFFu; break;
    case OR_U32: u = bits & 0xFFFFFFFFu; break;
    case OR_I32: u = (bits ^ 0x80000000u) & 0xFFFFFFFFu; break;
    case OR_F32:
      bits &= 0xFFFFFFFFu;
      /* negative floats: larger magnitude is smaller, so flip every bit;
         non-negative floats: set the sign bit so they sort above negatives */
      u = (bits & 0x80000000u) ? (~bits & 0xFFFFFFFFu) : (bits | 0x80000000u);
      break;
    case OR_U64: u = bits; break;
    case OR_I64: u = bits ^ 0x8000000000000000ull; break;
    case OR_F64:
      u = (bits & 0x8000000000000000ull) ? ~bits : (bits | 0x8000000000000000ull);
      break;
    default: u = 0;
  }
  if (!ascending) {
    /* descending order = ascending order of the complemented code */
    int w = 8 * key_bytes(dt);
    uint64_t mask = (w == 64) ? ~0ull : ((1ull << w) - 1);
    u = ~u & mask;
  }
  return u;
}

static uint64_t dec_narrow(int dt, uint64_t u, int ascending) {
  int w = 8 * key_bytes(dt);
  uint64_t mask = (w == 64) ? ~0ull : ((1ull << w) - 1);
  if (!ascending) u = ~u & mask;
  switch (dt) {
    case OR_U16: case OR_U32: case OR_U64: return u;
    case OR_I16: return u ^ 0x8000u;
    case OR_I32: return u ^ 0x80000000u;
    case OR_I64: return u ^ 0x8000000000000000ull;
    case OR_F32: return (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : (~u & 0xFFFFFFFFu);
    case OR_F64: return (u & 0x8000000000000000ull) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
    default: return 0;
  }
}

static uint64_t load_bits(int dt, const void *p, size_t i) {
  switch (key_bytes(dt)) {
    case 2: { uint16_t v; memcpy(&v, (const char *)p + 2 * i, 2); return v; }
    case 4: { uint32_t v; memcpy(&v, (const char *)p + 4 * i, 4); return v; }
    case 8: { uint64_t v; memcpy(&v, (const char *)p + 8 * i, 8); return v; }
    default: return 0;
  }
}

static void store_bits(int dt, void *p, size_t i, uint64_t v) {
  switch (key_bytes(dt)) {
    case 2: { uint16_t w = (uint16_t)v; memcpy((char *)p + 2 * i, &w, 2); break; }
    case 4: { uint32_t w = (uint32_t)v; memcpy((char *)p + 4 * i, &w, 4); break; }
    case 8: { memcpy((char *)p + 8 * i, &v, 8); break; }
    default: break;
  }
}

/* 128-bit keys: memory holds two 64-bit words per key. For u128 word 0 is
   the low half and word 1 the high half (little-endian integer). For kv64
   word 0 is the key and word 1 the value, and the key is the upper half of
   the compared number. */
static u128 enc_wide(int dt, const uint64_t w[2], int ascending) {
  uint64_t hi, lo;
  if (dt == OR_KV64) { hi = w[0]; lo = w[1]; } else { lo = w[0]; hi = w[1]; }
  u128 u = ((u128)hi << 64) | lo;
  return ascending ? u : ~u;
}

static void dec_wide(int dt, u128 u, int ascending, uint64_t w[2]) {
  if (!ascending) u = ~u;
  uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
  if (dt == OR_KV64) { w[0] = hi; w[1] = lo; } else { w[0] = lo; w[1] = hi; }
}

/* ------------------------------------------------------------------------ */
/* Scalar Quicksort on encoded keys (Algorithm 1 structure).                 */
/* ------------------------------------------------------------------------ */

struct oracle_stats {
  uint64_t heapsort_calls;  /* ranges finished by the Heapsort fallback */
  uint64_t max_depth;       /* deepest partition count on any path */
  uint64_t partitions;      /* number of Partition calls */
  uint64_t degenerate;      /* right side empty after Partition */
};

enum { BASE_CASE_MAX = 16 };

template <class K> static void swap_keys(K *a, K *b) { K t = *a; *a = *b; *b = t; }

/* Base case: insertion sort of a[0, n). */
template <class K> static void insertion_sort(K *a, size_t n) {
  for (size_t i = 1; i < n; ++i) {
    K v = a[i];
    size_t j = i;
    while (j > 0 && v < a[j - 1]) { a[j] = a[j - 1]; --j; }
    a[j] = v;
  }
}

/* Heapsort fallback (Sec. 2.2): textbook binary max-heap. */
template <class K> static void sift_down(K *a, size_t root, size_t n) {
  for (;;) {
    size_t child = 2 * root + 1;
    if (child >= n) return;
    if (child + 1 < n && a[child] < a[child + 1]) ++child;
    if (!(a[root] < a[child])) return;
    swap_keys(&a[root], &a[child]);
    root = child;
  }
}

template <class K> static void heap_sort(K *a, size_t n) {
  if (n < 2) return;
  for (size_t i = n / 2; i-- > 0;) sift_down(a, i, n);
  for (size_t end = n - 1; end > 0; --end) {
    swap_keys(&a[0], &a[end]);
    sift_down(a, 0, end);
  }
}

/* Median of three by the network (0,2)(0,1)(1,2) of Sec. 2.2: after (0,2)
   element 0 is the minimum and element 2 the maximum; (0,1) leaves the
   larger of elements 0 and 1 in slot 1; (1,2) leaves the smaller of slots 1
   and 2 in slot 1, which is then the median. */
template <class K> static K median_of_3(K x0, K x1, K x2) {
  if (x2 < x0) swap_keys(&x0, &x2);    /* (0,2) */
  if (x1 < x0) x1 = x0;                /* (0,1): only slot 1 is needed */
  if (x2 < x1) x1 = x2;                /* (1,2): only slot 1 is needed */
  return x1;
}

/* Partition: moves keys <= pivot before the others and returns the index
   of the first key of the right side (Sec. 2.1 definition). Two-pointer
   scan: the left pointer skips keys that belong left, the right pointer
   skips keys that belong right, and a misplaced pair is swapped. */
template <class K> static size_t partition_le(K *a, size_t begin, size_t end, K pivot) {
  size_t i = begin, j = end;  /* unexamined keys are [i, j) */
  for (;;) {
    while (i < j && !(pivot < a[i])) ++i;
    while (i < j && pivot < a[j - 1]) --j;
    if (i + 1 >= j) break;
    swap_keys(&a[i], &a[j - 1]);
    ++i; --j;
  }
  return i;
}

template <class K> struct Sorter {
  K *a;
  uint64_t depth_limit;
  oracle_stats *st;

  K choose_pivot(size_t begin, size_t end) {
    return median_of_3(a[begin], a[begin + (end - begin) / 2], a[end - 1]);
  }

  /* One range whose size exceeds the base case, at the given depth. The
     smaller child recurses, the larger one continues in the loop (the tail
     call of Algorithm 1). `depth` counts Partition calls on the path. */
  void recurse(size_t begin, size_t end, K pivot, uint64_t depth) {
    for (;;) {
      if (depth >= depth_limit) {
        st->heapsort_calls++;
        heap_sort(a + begin, end - begin);
        return;
      }
      depth++;
      if (depth > st->max_depth) st->max_depth = depth;
      st->partitions++;
      size_t bound = partition_le(a, begin, end, pivot);
      if (bound == end) {
        /* degenerate partition: every key <= pivot */
        st->degenerate++;
        K lo = a[begin], hi = a[begin];
        for (size_t k = begin + 1; k < end; ++k) {
          if (a[k] < lo) lo = a[k];
          if (hi < a[k]) hi = a[k];
        }
        if (!(lo < hi)) return;       /* all keys equal: sorted */
        pivot = lo;                   /* first key in sort order */
        continue;                     /* Recurse(keys, begin, end, first) */
      }
      size_t nl = bound - begin, nr = end - bound;
      /* children that fit the base case are finished right away */
      bool left_small = nl <= BASE_CASE_MAX, right_small = nr <= BASE_CASE_MAX;
      if (left_small) insertion_sort(a + begin, nl);
      if (right_small) insertion_sort(a + bound, nr);
      if (left_small && right_small) return;
      if (left_small) { pivot = choose_pivot(bound, end); begin = bound; continue; }
      if (right_small) { pivot = choose_pivot(begin, bound); end = bound; continue; }
      if (nl <= nr) {
        recurse(begin, bound, choose_pivot(begin, bound), depth);
        pivot = choose_pivot(bound, end); begin = bound;
      } else {
        recurse(bound, end, choose_pivot(bound, end), depth);
        pivot = choose_pivot(begin, bound); end = bound;
      }
    }
  }
};

static uint64_t floor_log2(uint64_t n) {
  uint64_t r = 0;
  while (n > 1) { n >>= 1; ++r; }
  return r;
}

template <class K>
static void sort_encoded(K *a, size_t n, int64_t depth_limit_override, oracle_stats *st) {
  if (n <= BASE_CASE_MAX) { insertion_sort(a, n); return; }
  Sorter<K> s;
  s.a = a;
  s.st = st;
  /* Sec. 2.2: at most 2*log2(n)+4 recursions */
  s.depth_limit = depth_limit_override >= 0 ? (uint64_t)depth_limit_override
                                             : 2 * floor_log2(n) + 4;
  s.recurse(0, n, s.choose_pivot(0, n), 0);
}

/* ------------------------------------------------------------------------ */
/* SFC64 (Doty-Humphrey's "small fast chaotic" generator, 64-bit) and the   */
/* multiply-high bounded offset used by pivot sampling (Sec. 2.2).          */
/* ------------------------------------------------------------------------ */

struct sfc64 { uint64_t a, b, c, counter; };

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t sfc64_next(sfc64 *s) {
  uint64_t out = s->a + s->b + s->counter++;
  s->a = s->b ^ (s->b >> 11);
  s->b = s->c + (s->c << 3);
  s->c = rotl64(s->c, 24) + out;
  return out;
}

/* Published seeding: all three state words take the seed, the counter
   starts at 1, and the first 12 outputs are discarded. */
static void sfc64_seed(sfc64 *s, uint64_t seed) {
  s->a = s->b = s->c = seed;
  s->counter = 1;
  for (int i = 0; i < 12; ++i) sfc64_next(s);
}

/* Division-free map of a 64-bit draw onto [0, range): the upper 64 bits of
   the 128-bit product (Lemire). */
static uint64_t bounded(uint64_t draw, uint64_t range) {
  return (uint64_t)(((u128)draw * range) >> 64);
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (C ABI, host pointers only).                        */
/* Return 0 on success, -1 on a bad argument.                                */
/* ------------------------------------------------------------------------ */

extern "C" {

int oracle_key_bytes(int dt) { return key_bytes(dt); }

/* Encoded keys: 2/4/8-byte keys become uint64 codes in out[n]; 16-byte
   keys become two uint64 words per key, {low, high} of the 128-bit code. */
int oracle_encode(int dt, const void *in, uint64_t *out, size_t n, int ascending) {
  int kb = key_bytes(dt);
  if (!kb) return -1;
  for (size_t i = 0; i < n; ++i) {
    if (kb == 16) {
      uint64_t w[2];
      memcpy(w, (const char *)in + 16 * i, 16);
      u128 u = enc_wide(dt, w, ascending);
      out[2 * i] = (uint64_t)u;
      out[2 * i + 1] = (uint64_t)(u >> 64);
    } else {
      out[i] = enc_narrow(dt, load_bits(dt, in, i), ascending);
    }
  }
  return 0;
}

int oracle_decode(int dt, const uint64_t *in, void *out, size_t n, int ascending) {
  int kb = key_bytes(dt);
  if (!kb) return -1;
  for (size_t i = 0; i < n; ++i) {
    if (kb == 16) {
      u128 u = ((u128)in[2 * i + 1] << 64) | in[2 * i];
      uint64_t w[2];
      dec_wide(dt, u, ascending, w);
      memcpy((char *)out + 16 * i, w, 16);
    } else {
      store_bits(dt, out, i, dec_narrow(dt, in[i], ascending));
    }
  }
  return 0;
}

/* Sorts keys[n] in place. depth_limit < 0 selects the paper's bound
   2*floor(log2 n)+4; a value >= 0 overrides it (0 = Heapsort only). */
int oracle_sort(int dt, void *keys, size_t n, int ascending, int64_t depth_limit,
                oracle_stats *stats) {
  int kb = key_bytes(dt);
  if (!kb) return -1;
  oracle_stats local;
  memset(&local, 0, sizeof local);
  if (!stats) stats = &local;
  if (n == 0) return 0;
  if (kb == 16) {
    u128 *e = (u128 *)malloc(n * sizeof(u128));
    if (!e) return -1;
    for (size_t i = 0; i < n; ++i) {
      uint64_t w[2];
      memcpy(w, (const char *)keys + 16 * i, 16);
      e[i] = enc_wide(dt, w, ascending);
    }
    sort_encoded(e, n, depth_limit, stats);
    for (size_t i = 0; i < n; ++i) {
      uint64_t w[2];
      dec_wide(dt, e[i], ascending, w);
      memcpy((char *)keys + 16 * i, w, 16);
    }
    free(e);
  } else {
    uint64_t *e = (uint64_t *)malloc(n * sizeof(uint64_t));
    if (!e) return -1;
    for (size_t i = 0; i < n; ++i) e[i] = enc_narrow(dt, load_bits(dt, keys, i), ascending);
    sort_encoded(e, n, depth_limit, stats);
    for (size_t i = 0; i < n; ++i) store_bits(dt, keys, i, dec_narrow(dt, e[i], ascending));
    free(e);
  }
  return 0;
}

/* Sorts each segment [offsets[s], offsets[s+1]) of keys independently. */
int oracle_sort_segmented(int dt, void *keys, const uint64_t *offsets, size_t num_segments,
                          int ascending) {
  int kb = key_bytes(dt);
  if (!kb) return -1;
  for (size_t s = 0; s < num_segments; ++s) {
    if (offsets[s + 1] < offsets[s]) return -1;
    int r = oracle_sort(dt, (char *)keys + (size_t)kb * offsets[s], offsets[s + 1] - offsets[s],
                        ascending, -1, NULL);
    if (r) return r;
  }
  return 0;
}

/* The Partition operation by its definition (Sec. 2.1): out[0, L) holds
   the keys whose code is <= the pivot's code, out[L, n) the others, each
   side in input order. *left_count receives L. */
int oracle_partition(int dt, const void *in, size_t n, const void *pivot, int ascending,
                     void *out, uint64_t *left_count) {
  int kb = key_bytes(dt);
  if (!kb) return -1;
  size_t l = 0;
  if (kb == 16) {
    uint64_t pw[2];
    memcpy(pw, pivot, 16);
    u128 p = enc_wide(dt, pw, ascending);
    for (size_t pass = 0; pass < 2; ++pass) {
      for (size_t i = 0; i < n; ++i) {
        uint64_t w[2];
        memcpy(w, (const char *)in + 16 * i, 16);
        bool goes_left = !(p < enc_wide(dt, w, ascending));
        if (goes_left == (pass == 0)) { memcpy((char *)out + 16 * l, w, 16); ++l; }
      }
      if (pass == 0) *left_count = l;
    }
  } else {
    uint64_t p = enc_narrow(dt, load_bits(dt, pivot, 0), ascending);
    for (size_t pass = 0; pass < 2; ++pass) {
      for (size_t i = 0; i < n; ++i) {
        uint64_t b = load_bits(dt, in, i);
        bool goes_left = !(p < enc_narrow(dt, b, ascending));
        if (goes_left == (pass == 0)) store_bits(dt, out, l++, b);
      }
      if (pass == 0) *left_count = l;
    }
  }
  return 0;
}

/* SFC64 stream after the published seeding: out[i] = i-th output. */
void oracle_sfc64(uint64_t seed, uint64_t *out, size_t count) {
  sfc64 s;
  sfc64_seed(&s, seed);
  for (size_t i = 0; i < count; ++i) out[i] = sfc64_next(&s);
}

uint64_t oracle_bounded(uint64_t draw, uint64_t range) { return bounded(draw, range); }

uint64_t oracle_median3(uint64_t a, uint64_t b, uint64_t c) { return median_of_3(a, b, c); }

/* Pivot sampling rule of the GPU library, a reading of Sec. 2.2:
     - a chunk is 64 bytes, kc = 64 / key_bytes keys, aligned to 64 bytes in
       memory; `addr_mod64` is the byte address of keys[0] modulo 64, so the
       first whole chunk starts at key off = ((64 - addr_mod64) % 64) / kb;
     - nc = (n - off) / kc whole chunks lie inside the range;
     - 256 / kc chunks are drawn: draw j is the j-th SFC64 output after
       seeding with `seed`, and chunk ci = bounded(draw, nc) covers keys
       [off + ci*kc, off + (ci+1)*kc);
     - the 256 sampled codes are sorted and the pivot is the code at rank
       127 (the lower median), returned as a key in its input form.
   Requires n >= 1024. */
int oracle_choose_pivot(int dt, const void *keys, size_t n, uint64_t addr_mod64, uint64_t seed,
                        int ascending, void *pivot_out) {
  int kb = key_bytes(dt);
  if (!kb || n < 1024 || addr_mod64 >= 64 || addr_mod64 % kb) return -1;
  const size_t S = 256;
  size_t kc = 64 / kb;
  size_t off = ((64 - addr_mod64) % 64) / kb;
  size_t nc = (n - off) / kc;
  sfc64 rng;
  sfc64_seed(&rng, seed);
  if (kb == 16) {
    u128 sample[256];
    size_t k = 0;
    for (size_t j = 0; j < S / kc; ++j) {
      size_t first = off + bounded(sfc64_next(&rng), nc) * kc;
      for (size_t t = 0; t < kc; ++t) {
        uint64_t w[2];
        memcpy(w, (const char *)keys + 16 * (first + t), 16);
        sample[k++] = enc_wide(dt, w, ascending);
      }
    }
    insertion_sort(sample, S);
    uint64_t w[2];
    dec_wide(dt, sample[S / 2 - 1], ascending, w);
    memcpy(pivot_out, w, 16);
  } else {
    uint64_t sample[256];
    size_t k = 0;
    for (size_t j = 0; j < S / kc; ++j) {
      size_t first = off + bounded(sfc64_next(&rng), nc) * kc;
      for (size_t t = 0; t < kc; ++t)
        sample[k++] = enc_narrow(dt, load_bits(dt, keys, first + t), ascending);
    }
    insertion_sort(sample, S);
    store_bits(dt, pivot_out, 0, dec_narrow(dt, sample[S / 2 - 1], ascending));
  }
  return 0;
}

}  /* extern "C" */
