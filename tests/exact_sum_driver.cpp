// Host driver for the exact fixed-point sums of the cluster form
// (paper_2608_09647_gb300/csrc/cg_exact.cuh), run by tests/test_exact_sum.py.
// Reads commands on stdin, one per line, numbers in hex:
//   conv <T as 32 hex digits, two's complement> <E>   -> bits of to_fp64(T, E)
//   convi <T> <E>                                      -> bits of to_fp64_int(T, E) (integer path only)
//   sum <w> <g> <n> <bits_1> ... <bits_n>             -> bits of the three-level sum:
//        groups of w terms at their own scale (a warp), groups of g of those
//        moved to their largest scale and added (a CTA), then all of those (the
//        cluster), each level's sums packed and unpacked, rounded once at the end
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../paper_2608_09647_gb300/csrc/cg_exact.cuh"

using namespace cg_exact;

int main() {
  char cmd[16];
  while (std::scanf("%15s", cmd) == 1) {
    if (!std::strcmp(cmd, "conv") || !std::strcmp(cmd, "convi")) {
      char hex[40];
      int E;
      if (std::scanf("%39s %d", hex, &E) != 2) return 1;
      u128 t = 0;
      for (const char* c = hex; *c; ++c) t = (t << 4) | (u128)std::stoul(std::string(1, *c), nullptr, 16);
      const double r = cmd[4] == 'i' ? to_fp64_int((i128)t, E, false) : to_fp64((i128)t, E, false);
      std::printf("%016llx\n", bits_of(r));
    } else if (!std::strcmp(cmd, "sum")) {
      int w, g, n;
      if (std::scanf("%d %d %d", &w, &g, &n) != 3) return 1;
      std::vector<double> v((size_t)n);
      for (int i = 0; i < n; ++i) {
        unsigned long long b;
        if (std::scanf("%llx", &b) != 1) return 1;
        v[(size_t)i] = double_of(b);
      }
      // level 1: groups of w terms at their own scale (a warp)
      std::vector<unsigned long long> lo, hi;
      for (int a = 0; a < n; a += w) {
        const int z = a + w < n ? a + w : n;
        int E = 1;
        bool bad = false;
        for (int i = a; i < z; ++i) {
          const Parts p = parts(v[(size_t)i]);
          E = p.e > E ? p.e : E;
          bad = bad || p.bad;
        }
        i128 S = 0;
        for (int i = a; i < z; ++i) S += (i128)to_fixed(parts(v[(size_t)i]), E);
        unsigned long long l, h;
        pack(S, E, bad, &l, &h);
        lo.push_back(l);
        hi.push_back(h);
      }
      // levels 2 and 3: groups of g entries (a CTA), then all entries (the cluster)
      for (int level = 0; level < 2; ++level) {
        const size_t m = lo.size(), gs = level == 0 ? (size_t)g : m;
        std::vector<unsigned long long> lo2, hi2;
        for (size_t a = 0; a < m; a += gs) {
          const size_t z = a + gs < m ? a + gs : m;
          int Em = 1;
          bool bad = false;
          std::vector<i128> S(z - a);
          std::vector<int> E(z - a);
          for (size_t k = a; k < z; ++k) {
            bool b;
            S[k - a] = unpack(lo[k], hi[k], &E[k - a], &b);
            bad = bad || b;
            Em = E[k - a] > Em ? E[k - a] : Em;
          }
          i128 acc = 0;
          for (size_t k = a; k < z; ++k) acc += shift_down(S[k - a], Em - E[k - a]);
          unsigned long long l, h;
          pack(acc, Em, bad, &l, &h);
          lo2.push_back(l);
          hi2.push_back(h);
        }
        lo.swap(lo2);
        hi.swap(hi2);
      }
      int E;
      bool bad;
      const i128 T = unpack(lo[0], hi[0], &E, &bad);
      std::printf("%016llx\n", bits_of(to_fp64(T, E, bad)));
    } else {
      return 1;
    }
  }
  return 0;
}
