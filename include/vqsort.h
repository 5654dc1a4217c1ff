/*
 * vqsort for GB300 (sm_103a): C ABI of libvqsort.so.
 *
 * A GPU implementation of the vectorised Quicksort of "Vectorized and
 * performance-portable Quicksort" (Blacher, Giesen, Sanders, Wassenberg):
 * pivot-sampled Quicksort whose levels are data-parallel partitions (every
 * key compared with the pivot and compacted to the left or right side) and
 * whose small ranges are finished by transpose-free sorting networks.
 *
 * Conventions for every entry point below:
 *   - Pointers named d_* are CUDA device pointers (global memory of the
 *     current device); h_* are host pointers. The caller owns all of them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Work is enqueued asynchronously on it; the call returns after
 *     the host-side argument checks and launches. Device-side failures (a
 *     bounded wait that ran out, a capacity overflow) are latched in the
 *     workspace and read by vqsort_last_device_status().
 *   - Keys are sorted in place, by the order of Sec. 2.4 of the paper:
 *     integers by value, floats by IEEE 754 totalOrder on their bit patterns
 *     (-NaN < -inf < ... < -0.0 < +0.0 < ... < +inf < +NaN, NaNs by
 *     payload), u128 as unsigned 128-bit numbers, kv64 pairs as the 128-bit
 *     number (key, value) with the key as the upper word. `ascending` = 0
 *     gives the exact reverse order. The sorted output is therefore unique:
 *     any correct sort yields the same bytes.
 *   - d_keys must be aligned to the key size (16 bytes for u128 and kv64).
 *     n = 0 or 1 is a no-op that returns VQ_OK.
 *   - Calls that share a workspace must not overlap on the device; calls
 *     without an explicit workspace use one the library keeps per (device,
 *     stream), so concurrent calls must use different streams.
 */
#ifndef VQSORT_H
#define VQSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Key types (Sec. 1 contributions and Sec. 2.4: 16/32/64-bit integers,
   32/64-bit floats, 128-bit keys, 64-bit keys with 64-bit data). Memory
   layout: u128 = two little-endian uint64 words {low, high}; kv64 =
   struct { uint64_t key; uint64_t value; }. */
typedef enum vq_dtype {
  VQ_I16 = 0, VQ_U16 = 1, VQ_I32 = 2, VQ_U32 = 3, VQ_F32 = 4,
  VQ_I64 = 5, VQ_U64 = 6, VQ_F64 = 7, VQ_U128 = 8, VQ_KV64 = 9
} vq_dtype;

typedef enum vq_status {
  VQ_OK = 0,
  VQ_ERR_INVALID = 1,      /* bad argument (null pointer, misalignment, bad dtype) */
  VQ_ERR_UNSUPPORTED = 2,  /* device is not compute capability 10.3 */
  VQ_ERR_NOMEM = 3,        /* workspace too small or allocation failed */
  VQ_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  VQ_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out; output undefined */
  VQ_ERR_INTERNAL = 6      /* device-side capacity overflow; output undefined */
} vq_status;

/* ---------------------------------------------------------------------- */
/* Sorting (Algorithm 1 and Secs. 2.1-2.3 of the paper).                   */
/* ---------------------------------------------------------------------- */

/* Sorts n keys of type dt at d_keys in place on `stream`, using a
   workspace the library allocates and keeps for this (device, stream).
   The recursion runs on the device: a persistent kernel pulls partition
   tiles from an on-device work queue (Sec. 2.1 partition, Sec. 2.2 pivot
   sampling, Algorithm 1 degenerate rule; large ranges are split into up to
   256 buckets per level, Sec. 4.2), small ranges are finished by
   sorting networks (Sec. 2.3, Sec. 3), and ranges deeper than
   2*floor(log2 n)+4 partition levels go to a device merge sort (the
   paper's Heapsort fallback of Sec. 2.2, replaced). */
vq_status vqsort_sort(vq_dtype dt, void *d_keys, size_t n, int ascending, void *stream);

/* 64-bit keys with 64-bit values (Sec. 2.4): d_pairs holds n structs
   {uint64_t key; uint64_t value;}. Pairs are ordered by key, ties by value,
   so every pair stays intact and the output is unique. Same as
   vqsort_sort(VQ_KV64, ...). */
vq_status vqsort_sort_kv(void *d_pairs, size_t n, int ascending, void *stream);

/* Key-only order of the same pairs (Sec. 2.4, 64-bit keys with 64-bit
   data; Sec. 5, Quicksort is not stable): d_pairs holds n structs
   {uint64_t key; uint64_t value;}; afterwards the keys are non-decreasing
   (ascending = 0: non-increasing) and the pairs are the input's pairs, each
   value still beside its key. Only the 64-bit key is compared, so pairs
   with equal keys come out in an unspecified order (it may differ from
   vqsort_sort_kv's). A leaf range holding the key 0 or 2^64 - 1 is finished
   in the (key, value) order, one of the valid orders. In place on
   `stream`, library-owned workspace per (device, stream); the _ws form
   takes a caller-owned workspace of vqsort_workspace_bytes(VQ_KV64, n, 1)
   bytes (256-byte aligned) and allocates nothing. Argument checks and
   status as vqsort_sort. */
vq_status vqsort_sort_kv_by_key(void *d_pairs, size_t n, int ascending, void *stream);
vq_status vqsort_sort_kv_by_key_ws(void *d_pairs, size_t n, int ascending, void *d_ws, size_t ws_bytes,
                                   void *stream);

/* Stable sort (Sec. 5: appending a unique row identifier below the key makes
   Quicksort stable). Sorts the n keys at d_keys in place, in the same order
   as vqsort_sort, and writes to d_rows (device, n uint64_t, 8-byte aligned)
   the input position of each output key; keys that compare equal (same bit
   pattern after encoding) keep their input order, in both sort orders.
   2-, 4- and 8-byte key types; 16-byte types return VQ_ERR_UNSUPPORTED.
   Each key's code is packed with its row (keys of up to 4 bytes into a
   64-bit code, 8-byte keys into a 128-bit one), the packed codes are sorted
   and unpacked; the library's workspace for this stream grows to hold them. */
vq_status vqsort_sort_stable(vq_dtype dt, void *d_keys, size_t n, int ascending, uint64_t *d_rows,
                             void *stream);

/* Sorts num_segments independent arrays in one set of launches: segment s
   is keys [d_offsets[s], d_offsets[s+1]) of d_keys (CSR, uint64, device
   memory, num_segments + 1 entries, non-decreasing, last entry == n_total).
   Each segment gets its own recursion with its own depth bound. Keys
   outside [d_offsets[0], n_total) are not touched. A malformed offsets
   array is detected on the device and reported as VQ_ERR_INVALID by
   vqsort_last_device_status(). */
vq_status vqsort_sort_segmented(vq_dtype dt, void *d_keys, size_t n_total,
                                const uint64_t *d_offsets, size_t num_segments,
                                int ascending, void *stream);

/* Bytes of device workspace that vqsort_sort_ws / _segmented_ws need for
   n_total keys in num_segments segments (1 for a plain sort): the
   out-of-place partition buffer (n_total keys) plus the work queue, tile
   status words, segment descriptors and leaf lists. */
size_t vqsort_workspace_bytes(vq_dtype dt, size_t n_total, size_t num_segments);

/* As vqsort_sort / vqsort_sort_segmented, with a caller-owned workspace
   of ws_bytes >= vqsort_workspace_bytes() at d_ws (256-byte aligned). The
   workspace needs no initialisation. These calls allocate nothing, so they
   can be captured into a CUDA graph. */
vq_status vqsort_sort_ws(vq_dtype dt, void *d_keys, size_t n, int ascending,
                         void *d_ws, size_t ws_bytes, void *stream);
vq_status vqsort_sort_segmented_ws(vq_dtype dt, void *d_keys, size_t n_total,
                                   const uint64_t *d_offsets, size_t num_segments,
                                   int ascending, void *d_ws, size_t ws_bytes, void *stream);

/* End-to-end sort of a HOST array: copies h_keys to the device, sorts, and
   waits. Uses a library-owned stream and device buffer on the current
   device. The sorted keys are copied back by a copy engine after the sort;
   with VQ_OPT_HOST_DIRECT = 1 the leaf kernels write them straight into a
   pinned (page-locked, mapped) array instead. Pageable memory is always
   copied back. */
vq_status vqsort_sort_host(vq_dtype dt, void *h_keys, size_t n, int ascending);

/* The same end-to-end sort of a HOST array, enqueued on `stream` without
   waiting: the upload, the sort and the download (or the leaves' direct
   writes into a pinned array) follow one another on that stream, and h_keys
   must stay untouched until the stream has passed them. The device copy and
   the workspace belong to the library, one per (device, stream), so arrays
   on different streams overlap: one uploads while another sorts and writes
   back. Completion: synchronize the stream; the status is then read with
   vqsort_last_device_status(NULL, stream). */
vq_status vqsort_sort_host_async(vq_dtype dt, void *h_keys, size_t n, int ascending, void *stream);

/* ---------------------------------------------------------------------- */
/* The two per-level kernels on their own.                                 */
/* ---------------------------------------------------------------------- */

/* One Partition (Sec. 2.1): reads n keys from d_in and writes them to
   d_out (a different buffer) so that d_out[0, L) holds every key that is
   <= *h_pivot in the chosen order and d_out[L, n) every other key, in an
   unspecified order within each side; L is written to *d_left_count
   (device uint64). h_pivot points to one key (host memory) of type dt. */
vq_status vqsort_partition(vq_dtype dt, const void *d_in, void *d_out, size_t n,
                           const void *h_pivot, int ascending, uint64_t *d_left_count,
                           void *stream);

/* Pivot sampling (Sec. 2.2) as the sorter does it: 256 / (64 / key bytes)
   chunks of 64 bytes, aligned to 64 bytes in memory, are drawn from the n
   keys at d_keys with the SFC64 generator seeded by `seed` (a = b = c =
   seed, counter = 1, 12 outputs discarded) and the multiply-high map of
   each draw onto the number of whole chunks; the 256 sampled keys are
   sorted in the chosen order and the key at rank 127 is written to
   d_pivot_out (device, one key). Requires n >= 1024. */
vq_status vqsort_choose_pivot(vq_dtype dt, const void *d_keys, size_t n, uint64_t seed,
                              int ascending, void *d_pivot_out, void *stream);

/* One Partition, as vqsort_partition, that allocates nothing. The paper has
   no counterpart: this entry point exists for callers that must not call
   cudaMalloc while they work, because cudaMalloc can synchronize the device
   and can fail once a fixed memory budget is used up (a latency-bound
   serving loop, code running inside another allocator's hooks).
   Its scratch (counters, the range descriptor and the tile queue) is a
   fixed array of about 517 KiB in device memory that belongs to the loaded
   library: every GPU that loads libvqsort.so holds it until the process
   exits. Limit: n <= 65536 * ((32768 - 16) / key bytes) keys (about 1.07e9
   2-byte, 5.4e8 4-byte, 2.7e8 8-byte, 1.3e8 16-byte keys); larger n returns
   VQ_ERR_INVALID before anything is launched.
   The first call on a device looks up the array's device address
   (cudaGetSymbolAddress) with that device current; make that first call
   before any stream capture. Every call clears the counters and queue it
   needs, so a call never depends on the previous one, but all calls share
   the one array: calls that overlap on the GPU (different streams, or
   different host threads) race and give wrong results. Device-side
   timeouts are not reported by this entry point. */
vq_status vqsort_partition_noalloc(vq_dtype dt, const void *d_in, void *d_out, size_t n,
                                   const void *h_pivot, int ascending, uint64_t *d_left_count,
                                   void *stream);

/* ---------------------------------------------------------------------- */
/* Status, statistics, options, profiling.                                 */
/* ---------------------------------------------------------------------- */

/* Waits for `stream` and returns the device-side status latched by the
   last sort that used the workspace d_ws (NULL = the library's workspace
   for this device and stream; VQ_OK, and zero statistics below, while no
   sort has used that one). */
vq_status vqsort_last_device_status(const void *d_ws, void *stream);

/* Enqueues on `stream` a copy of the device-side status word of the
   caller-owned workspace d_ws into *h_status (8 bytes of host memory; page-
   locked memory keeps the call asynchronous). Once the stream has passed
   this point, *h_status holds the vq_status latched by the sorts enqueued
   before it on that workspace (VQ_OK = 0). For serving loops that must not
   wait for a stream to learn whether a sort succeeded. VQ_ERR_INVALID for
   null pointers. */
vq_status vqsort_device_status_async(const void *d_ws, uint64_t *h_status, void *stream);

/* Library resource management (the paper has no counterpart). Waits for
   `stream`, then frees what the library holds for it on the current device:
   the workspace it allocated for sorts given none (vqsort_sort and the
   other forms without a workspace argument), and the two side streams and
   three events on which a sort runs its leaf kernels concurrently. The next
   sort on the stream creates them again. For callers that create and
   destroy streams, e.g. one per request. No sort may be enqueued on the
   stream while this runs. VQ_ERR_CUDA if the wait fails (nothing is freed
   then); VQ_OK when nothing was held. */
vq_status vqsort_release_stream(void *stream);

/* Counters of the last sort on a workspace (waits for `stream`). */
typedef struct vq_stats {
  uint64_t keys_partitioned;     /* sum over partition levels (two-way and K-way) of keys
                                    read once and written once */
  uint64_t tiles;                /* partition tiles processed */
  uint64_t segments;             /* ranges partitioned */
  uint64_t leaves_warp;          /* ranges of <= 512 keys sorted by one warp */
  uint64_t leaves_block;         /* ranges sorted by one thread block */
  uint64_t leaf_keys;            /* keys in those ranges */
  uint64_t equal_ranges;         /* ranges found all-equal (copied, not sorted) */
  uint64_t equal_keys;
  uint64_t degenerate;           /* partitions whose right side was empty */
  uint64_t fallback_ranges;      /* ranges past the depth bound (merge sort) */
  uint64_t fallback_keys;
  uint64_t max_depth;            /* deepest partition level reached */
  uint64_t device_status;        /* vq_status latched on the device */
  uint64_t keys_counted;         /* keys read by K-way counting passes */
  uint64_t kway_ranges;          /* ranges split K ways (16..256 buckets) */
  uint64_t guard;                /* first failed device bounds guard (0: none); a failed guard
                                    skips the access and latches VQ_ERR_INTERNAL */
  uint64_t partition_blocks;     /* thread blocks of the persistent partition kernel */
  uint64_t leaves_mid;           /* ranges of 513..2048 keys (16-byte keys: ..1024) sorted by
                                    128-thread blocks */
  uint64_t leaf_ce;              /* key comparisons of the leaf sorts: compare-exchanges of
                                    the register networks plus the comparisons of the
                                    shared-memory merges (padding slots included) */
  uint64_t leaf_keys_warp;       /* keys of the ranges sorted by one warp */
  uint64_t leaf_keys_mid;        /* keys of the ranges sorted by 128-thread blocks */
  uint64_t leaf_keys_block;      /* keys of the ranges sorted by the block leaves (all-equal
                                    ranges, copied by the same kernel, are in equal_keys) */
} vq_stats;
vq_status vqsort_get_stats(const void *d_ws, void *stream, vq_stats *out);

const char *vqsort_status_string(vq_status s);

/* Process-wide options read by later calls. */
typedef enum vq_option {
  VQ_OPT_DEPTH_LIMIT = 0,   /* -1: 2*floor(log2 n)+4 per root range (default);
                               k >= 0: at most k partition levels (test hook for the
                               merge-sort fallback) */
  VQ_OPT_LEAF_CUTOFF = 1,   /* 0 (default): by key size and array length: one array of
                               at most 2^21 keys (keys of 4 bytes or fewer: 2^22) 16384,
                               below 2^26 keys (2^25) 8192, else, and for segmented
                               batches and 16-byte keys, 4096; else largest range (keys,
                               a power of two in [1024, 16384] that fits 128 KiB of shared
                               memory) finished by the block network */
  VQ_OPT_SEED = 2,          /* seed of the per-range pivot sampling streams */
  VQ_OPT_SPIN_LIMIT = 3,    /* iterations of each bounded device wait (default 2^22,
                               about a second) */
  VQ_OPT_TEST_STALL = 4,    /* 1: the root range never publishes its children, so every
                               block's bounded wait for work runs out and the sort reports
                               VQ_ERR_TIMEOUT (test of the bounded-wait path; never hangs) */
  VQ_OPT_TILE_BYTES = 5,    /* partition tile window: 16384, 32768 or 65536 bytes; 0 (default):
                               16 KiB for a sort of one array of 4- or 8-byte keys short
                               enough for the 16384-key leaf cutoff, else 64 KiB for 8- and
                               16-byte keys and 32 KiB for narrower keys */
  VQ_OPT_LEAF_THREADS = 6,  /* 0: block leaves use cutoff/16 threads (16 keys per thread);
                               256, 512 or 1024: that many threads when they hold a
                               cutoff-size leaf at 16 keys each (else cutoff/16); 16-byte
                               keys: 256 or (otherwise) 512 threads */
  VQ_OPT_KWAY = 7,          /* 1 (default): ranges of at least 4x the leaf cutoff are split
                               into 16..256 buckets per level (sampled splitters, a counting
                               pass and a scatter pass; the K > 2 partition of Sec. 4.2),
                               with equality buckets when the splitters repeat; 0: every
                               level is the paper's two-way Partition. The output is the
                               same. */
  VQ_OPT_HOST_DIRECT = 8    /* host-array sorts of pinned memory: 0 (default): a copy
                               engine copies the result back after the sort; 1: the leaf
                               kernels store it straight into the pinned array, so the
                               download overlaps the leaves (about 8 % faster for one sort
                               alone, but several times slower while another stream's sort
                               or upload runs, as the leaves' host stores then contend with
                               the other work). The output is the same. */
} vq_option;
vq_status vqsort_set_option(vq_option opt, int64_t value);
int64_t vqsort_get_option(vq_option opt);

/* Comparator schedule of the bitonic merge that joins two sorted runs of
   run_len keys (Sec. 3, Fig. "Bitonic Merge"), as the networks execute it
   with keys_per_thread keys in each thread's registers (a power of two
   <= run_len): writes the (i, j) index pairs, i < j, step by step and in
   increasing i within a step, as 2*k unsigned ints into pairs_out (at most
   max_pairs pairs; pairs_out may be NULL to count) and k to *n_pairs.
   Indices are logical positions t * keys_per_thread + r in a block of
   2 * run_len keys. */
vq_status vqsort_merge_schedule(unsigned run_len, unsigned keys_per_thread, unsigned *pairs_out,
                                size_t max_pairs, size_t *n_pairs);

/* Per-kernel timing with CUDA events recorded on the launching stream
   around every launch the library makes while enabled. */
vq_status vqsort_profile_enable(int enable);
vq_status vqsort_profile_reset(void);
/* Fills up to `max` entries: kernel names, summed milliseconds and launch
   counts (waits for all recorded events). *count gets the entry count. */
vq_status vqsort_profile_read(const char **names, double *ms, uint64_t *launches, size_t max,
                              size_t *count);

/* Integer throughput probe, a measurement helper (the paper has no
   counterpart): launches `blocks` blocks of 256 threads on `stream`; each
   thread updates eight independent registers `iters` times with
   kind 0: a 32-bit min and an xor (2 lane operations per register and
   iteration), kind 1: a 64-bit compare, two selects and an xor of both
   words (6 lane operations), and writes one 32-bit word to d_sink (device
   memory of blocks * 256 words, caller-owned). *ops_per_thread gets the
   lane operations per thread. Timed with CUDA events on `stream`, it gives
   the integer lane-operation rate the leaf networks are measured against.
   Returns VQ_ERR_INVALID for another kind, zero blocks or null pointers. */
vq_status vqsort_probe_int_throughput(int kind, unsigned blocks, unsigned iters, void *d_sink,
                                      uint64_t *ops_per_thread, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VQSORT_H */
