/*
 * Column-sort networks of the base case (Sec. 3 of the paper: each column of
 * the key matrix is sorted by a network with few compare-and-exchange
 * modules, the same module applied to all columns at once). On the GPU a
 * column is the R keys one thread holds in registers.
 *
 * Written as X-macros: CE(a, b) is one module that leaves the smaller key in
 * slot a and the larger in slot b. The header is plain C/C++ so the CPU test
 * suite compiles these exact tables and checks them by the 0-1 principle.
 *
 *   R = 2:  1 module.
 *   R = 4:  5 modules, odd-even merge sort (the size the paper's 4x4
 *           showcase uses; 5 is the lower bound for 4 inputs).
 *   R = 8:  19 modules, depth 6 (the best known size for 8 inputs).
 *   R = 16: 60 modules, depth 10 (the smallest known size for 16 inputs,
 *           the count of Green's network that the paper cites).
 */
#ifndef VQ_NETWORKS_H
#define VQ_NETWORKS_H

#define VQ_NET2(CE) CE(0, 1)

#define VQ_NET4(CE) CE(0, 1) CE(2, 3) CE(0, 2) CE(1, 3) CE(1, 2)

#define VQ_NET8(CE)                                 \
  CE(0, 2) CE(1, 3) CE(4, 6) CE(5, 7)               \
  CE(0, 4) CE(1, 5) CE(2, 6) CE(3, 7)               \
  CE(0, 1) CE(2, 3) CE(4, 5) CE(6, 7)               \
  CE(2, 4) CE(3, 5)                                 \
  CE(1, 4) CE(3, 6)                                 \
  CE(1, 2) CE(3, 4) CE(5, 6)

#define VQ_NET16(CE)                                                                   \
  CE(0, 13) CE(1, 12) CE(2, 15) CE(3, 14) CE(4, 8) CE(5, 6) CE(7, 11) CE(9, 10)         \
  CE(0, 5) CE(1, 7) CE(2, 9) CE(3, 4) CE(6, 13) CE(8, 14) CE(10, 15) CE(11, 12)         \
  CE(0, 1) CE(2, 3) CE(4, 5) CE(6, 8) CE(7, 9) CE(10, 11) CE(12, 13) CE(14, 15)         \
  CE(0, 2) CE(1, 3) CE(4, 10) CE(5, 11) CE(6, 7) CE(8, 9) CE(12, 14) CE(13, 15)         \
  CE(1, 2) CE(3, 12) CE(4, 6) CE(5, 7) CE(8, 10) CE(9, 11) CE(13, 14)                   \
  CE(1, 4) CE(2, 6) CE(5, 8) CE(7, 10) CE(9, 13) CE(11, 14)                             \
  CE(2, 4) CE(3, 6) CE(9, 12) CE(11, 13)                                                \
  CE(3, 5) CE(6, 8) CE(7, 9) CE(10, 12)                                                 \
  CE(3, 4) CE(5, 6) CE(7, 8) CE(9, 10) CE(11, 12)                                       \
  CE(6, 7) CE(8, 9)

/*
 * Bitonic merge of two sorted runs of L keys each (Sec. 3, Fig. "Bitonic
 * Merge"), on keys laid out as logical index i = thread * R + register.
 * Step 0 compares i with 2L-1-i inside each block of 2L keys; step s >= 1
 * compares i with i + L/2^s. Expressed per (thread, register) so no
 * transpose is ever needed:
 *   lane_xor != 0: partner thread = thread ^ lane_xor, partner register =
 *                  reverse ? R-1-r : r;
 *   lane_xor == 0: partner is register r ^ reg_xor of the same thread.
 * The thread whose index has the bit `lower_bit` clear keeps the minimum.
 */
struct VqMergeStep {
  unsigned lane_xor;
  unsigned reg_xor;
  unsigned lower_bit;
  int reverse;
};

#ifdef __CUDACC__
#define VQ_HD __host__ __device__ __forceinline__
#else
#define VQ_HD static inline
#endif

/* Steps of one merge: 1 + log2(L). */
VQ_HD unsigned vq_merge_steps(unsigned L) {
  unsigned s = 1;
  while ((1u << (s - 1)) < L) ++s;
  return s;
}

VQ_HD struct VqMergeStep vq_merge_step(unsigned L, unsigned R, unsigned step) {
  struct VqMergeStep m;
  if (step == 0) {
    /* needs L >= R: a block of 2L keys spans 2L/R threads */
    m.lane_xor = (2 * L) / R - 1;
    m.reg_xor = 0;
    m.lower_bit = L / R;
    m.reverse = 1;
    return m;
  }
  unsigned d = L >> step;
  if (d >= R) {
    m.lane_xor = d / R;
    m.reg_xor = 0;
    m.lower_bit = d / R;
  } else {
    m.lane_xor = 0;
    m.reg_xor = d;
    m.lower_bit = 0;
  }
  m.reverse = 0;
  return m;
}

#endif /* VQ_NETWORKS_H */
