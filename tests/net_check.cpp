// Checks the column-sort networks of the CUDA library (networks.h, compiled
// here by the host compiler) by the 0-1 principle: a comparator network
// sorts every input iff it sorts every 0/1 input. Also checks that one
// bitonic merge, as the kernels schedule it for each keys-per-thread value,
// merges every pair of sorted 0/1 runs. Prints "ok" on success.
#include <cstdio>
#include <vector>
#include "networks.h"

static int fail = 0;

template <int N> static void check_net(const std::vector<std::pair<int, int>> &net, const char *name) {
  for (unsigned x = 0; x < (1u << N); ++x) {
    int v[N];
    for (int i = 0; i < N; ++i) v[i] = (x >> i) & 1;
    for (auto &c : net)
      if (v[c.first] > v[c.second]) { int t = v[c.first]; v[c.first] = v[c.second]; v[c.second] = t; }
    for (int i = 1; i < N; ++i)
      if (v[i - 1] > v[i]) { std::printf("%s fails on %u\n", name, x); fail = 1; return; }
  }
}

static void check_merge(unsigned L, unsigned R) {
  // all (a, b): run 1 has a ones at its end, run 2 has b ones at its end
  for (unsigned a = 0; a <= L; ++a)
    for (unsigned b = 0; b <= L; ++b) {
      std::vector<int> v(2 * L);
      for (unsigned i = 0; i < L; ++i) { v[i] = i >= L - a; v[L + i] = i >= L - b; }
      for (unsigned s = 0; s < vq_merge_steps(L); ++s) {
        VqMergeStep m = vq_merge_step(L, R, s);
        for (unsigned t = 0; t < 2 * L / R; ++t)
          for (unsigned r = 0; r < R; ++r) {
            unsigned pt = m.lane_xor ? (t ^ m.lane_xor) : t;
            unsigned pr = m.lane_xor ? (m.reverse ? R - 1 - r : r) : (r ^ m.reg_xor);
            unsigned i = t * R + r, j = pt * R + pr;
            if (i < j && v[i] > v[j]) { int tmp = v[i]; v[i] = v[j]; v[j] = tmp; }
          }
      }
      for (unsigned i = 1; i < 2 * L; ++i)
        if (v[i - 1] > v[i]) { std::printf("merge L=%u R=%u fails (%u,%u)\n", L, R, a, b); fail = 1; return; }
    }
}

int main() {
  std::vector<std::pair<int, int>> n2, n4, n8, n16;
#define CE2(a, b) n2.push_back({a, b});
#define CE4(a, b) n4.push_back({a, b});
#define CE8(a, b) n8.push_back({a, b});
#define CE16(a, b) n16.push_back({a, b});
  VQ_NET2(CE2) VQ_NET4(CE4) VQ_NET8(CE8) VQ_NET16(CE16)
  check_net<2>(n2, "net2");
  check_net<4>(n4, "net4");
  check_net<8>(n8, "net8");
  check_net<16>(n16, "net16");
  std::printf("sizes %zu %zu %zu %zu\n", n2.size(), n4.size(), n8.size(), n16.size());
  for (unsigned L = 1; L <= 256; L *= 2)
    for (unsigned R = 1; R <= 16 && R <= L; R *= 2) check_merge(L, R);
  std::printf(fail ? "FAIL\n" : "ok\n");
  return fail;
}
