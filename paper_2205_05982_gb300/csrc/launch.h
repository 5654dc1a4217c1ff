// Launch interface between the host driver (vqsort.cu) and the kernel
// translation units. Every function enqueues on `stream` and returns the
// CUDA error of the launch.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace vq {

// Partition kernel geometry: 256 threads, CPT chunks of 16 bytes per thread
// (CPT = 8: 32 KiB tile windows, the default; CPT = 4: 16 KiB windows;
// CPT = 16: 64 KiB windows).
constexpr int PART_NT = 256;
constexpr int PART_CPT = 8;                            // default
// blocks per SM the kernel is built for (shared memory allows this many)
__host__ __device__ constexpr int part_blocks_per_sm(int cpt) { return cpt >= 16 ? 3 : 5; }
__host__ __device__ constexpr int part_window(int cpt) { return PART_NT * cpt * 16; }
__host__ __device__ constexpr int part_smem(int cpt) { return part_window(cpt); }
// Tile keys: the tile plus its 16-byte misalignment fits the window.
__host__ __device__ constexpr unsigned part_tile_keys(int kb, int cpt = PART_CPT) {
  return (unsigned)((part_window(cpt) - 16) / kmem(kb));
}

// K-way tiles: keys in the first half of the window, the second half stages
// them in bucket order; at most 16 keys per thread.
__host__ __device__ constexpr int kw_cpt(int kb, int cpt) { return cpt / 2 < kmem(kb) ? cpt / 2 : kmem(kb); }
__host__ __device__ constexpr unsigned kw_tile_keys(int kb, int cpt = PART_CPT) {
  return (unsigned)((PART_NT * kw_cpt(kb, cpt) * 16 - 16) / kmem(kb));
}

// Mid-size leaves (more than a warp leaf, at most MID_NT * 16 keys; 16-byte
// keys: MID_NT * 8) are sorted by MID_NT threads holding 8 or 16 keys each:
// many small blocks per SM, and every thread's merge-path search shared by
// as many keys as its registers hold.
constexpr int MID_NT = 128;
__host__ __device__ constexpr unsigned mid_max_keys(int kb) { return kmem(kb) == 16 ? MID_NT * 8u : MID_NT * 16u; }
__host__ __device__ constexpr unsigned mid_leaf_limit(int kb) { return mid_max_keys(kb); }

constexpr int LEAF_NT = 1024;       // threads of the block leaf kernel
constexpr int FB_NT = 256;          // threads of the merge fallback kernel
constexpr int FB_R = 8;             // keys per thread in its chunk sort
constexpr int FB_CHUNK = FB_NT * FB_R;

// Threads of a block-leaf CTA: 16 keys per thread at the cutoff, or the
// thread count set by option when that many threads hold a cutoff-size leaf
// at up to 16 keys each.
__host__ constexpr int leaf_nt_default(unsigned cutoff) {
  return cutoff >= 16384 ? 1024 : cutoff >= 8192 ? 512 : 256;
}
__host__ constexpr int leaf_nt_for(unsigned cutoff, int threads) {
  return threads && (unsigned)threads * 16u >= cutoff ? threads : leaf_nt_default(cutoff);
}

// Default and largest block-leaf cutoff (keys) per key size. The default
// also sets the K-way bucket target (a quarter of it); measured on 1e8-key
// sorts, 4096 is best for every key size (u32 3.01 -> 2.37 ms against
// 16384; u64 3.38 -> 3.24 ms against 8192: block leaves then run on 256
// threads with 16 keys each, one code path).
__host__ constexpr unsigned default_leaf_cutoff(int kb) {
  return kb == 2 ? 4096u : kb == 4 ? 4096u : kb == 8 ? 4096u : 4096u;
}
// Default cutoff of a one-array sort of n keys: a larger cutoff saves a
// partition level where n is small enough that the leaves stay few, which
// matters most for short sorts, whose levels are latency-bound. Measured on
// uniform keys with L2 flushed (u64: 1e6 keys 210 -> 169 us at 16384, 3.2e7
// keys 1.20 -> 1.13 ms at 8192; 1e8 keys stay fastest at 4096). Segmented
// batches and 16-byte keys keep the per-key-size default.
constexpr uint64_t LEAF_N_SMALL_WIDE = 1ull << 21, LEAF_N_SMALL_NARROW = 1ull << 22;   // up to here: 16384
constexpr uint64_t LEAF_N_MID_WIDE = 1ull << 26, LEAF_N_MID_NARROW = 1ull << 25;       // below here: 8192
__host__ constexpr unsigned size_leaf_cutoff(int kb, uint64_t n, uint64_t segments) {
  return segments != 1 || kmem(kb) == 16 ? default_leaf_cutoff(kb)
         : n <= (kb == 8 ? LEAF_N_SMALL_WIDE : LEAF_N_SMALL_NARROW) ? 16384u
         : n < (kb == 8 ? LEAF_N_MID_WIDE : LEAF_N_MID_NARROW)     ? 8192u
                                                                    : default_leaf_cutoff(kb);
}
__host__ __device__ constexpr unsigned max_leaf_cutoff(int kb) {
  return kb <= 8 ? 16384u : 4096u;   // 16-byte keys: at most 4 per thread in registers
}
__host__ constexpr unsigned code_bytes(int kb) { return kb == 2 ? 4u : (unsigned)kmem(kb); }

// Keys per thread for a leaf of len keys on nt threads: the fewest of 4, 8
// and 16 (at most rmax) that hold it, so that as many threads as possible
// share the work.
__host__ __device__ constexpr int leaf_r_for(unsigned len, int nt, int rmax) {
  return len <= 4u * (unsigned)nt || rmax <= 4 ? 4 : len <= 8u * (unsigned)nt || rmax <= 8 ? 8 : 16;
}
// Most keys per thread of a block leaf on nt threads: 16, or fewer when the
// largest cutoff of the key size needs fewer (16-byte keys: 4096 / nt).
__host__ __device__ constexpr int leaf_rmax(int kb, int nt) {
  return (int)max_leaf_cutoff(kb) / nt < 16 ? (int)max_leaf_cutoff(kb) / nt : 16;
}
// Shared memory of a block leaf on nt threads for leaves of up to `cutoff`
// keys: R keys per thread plus one spare slot per thread (bank spread).
__host__ constexpr size_t leaf_block_smem(int kb, unsigned cutoff, int nt) {
  return (size_t)nt * (leaf_r_for(cutoff, nt, leaf_rmax(kb, nt)) + 1) * code_bytes(kb);
}

cudaError_t launch_prep(const SortArgs &a, cudaStream_t s);
cudaError_t launch_seed(int kb, const SortArgs &a, cudaStream_t s);
cudaError_t launch_partition(int kb, const SortArgs &a, cudaStream_t s);
cudaError_t launch_choose_pivot(int kb, const SortArgs &a, const void *keys, unsigned long long n,
                                unsigned long long seed, void *out, cudaStream_t s);
cudaError_t launch_leaf_warp(int kb, const SortArgs &a, cudaStream_t s);
cudaError_t launch_leaf_mid(int kb, const SortArgs &a, cudaStream_t s);
cudaError_t launch_leaf_block(int kb, const SortArgs &a, cudaStream_t s);
cudaError_t launch_fallback(int kb, const SortArgs &a, cudaStream_t s);
cudaError_t launch_stable_pack(int kb, const void *keys, void *packed, uint64_t n, Codec cd, cudaStream_t s);
cudaError_t launch_stable_unpack(int kb, const void *packed, void *keys, uint64_t *rows, uint64_t n, Codec cd,
                                 cudaStream_t s);

}  // namespace vq
