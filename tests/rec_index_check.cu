// Host-side check of the CommFlux record layout (rec_index, rec_elems in internal.h):
// for padded shapes of several sizes, the entries (axis, side, quantity, sub-cycle,
// transverse position) map one to one onto [0, rec_elems).  Prints "OK <entries>" and
// exits 0, or "FAIL ..." and exits 1.
#include <cstdio>
#include <vector>

#include "internal.h"

using namespace dfn;

int main() {
  const int shapes[][3] = {{24, 24, 24}, {40, 40, 40}, {16, 24, 40}, {80, 28, 144}, {9, 13, 7}};
  long long total = 0;
  for (const auto& s : shapes) {
    const long long n = rec_elems(s);
    std::vector<unsigned char> seen((size_t)n, 0);
    for (int d = 0; d < 3; ++d) {
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      for (int side = 0; side < 2; ++side)
        for (int q = 0; q < 3; ++q)
          for (int sub = 0; sub < 2; ++sub)
            for (int c2 = 0; c2 < s[t2]; ++c2)
              for (int c1 = 0; c1 < s[t1]; ++c1) {
                const int i = rec_index(s, d, side, q, sub, c1, c2);
                if (i < 0 || i >= n || seen[(size_t)i]) {
                  std::printf("FAIL s=%d,%d,%d d=%d index %d of %lld\n", s[0], s[1], s[2], d, i,
                              n);
                  return 1;
                }
                seen[(size_t)i] = 1;
                ++total;
              }
    }
    for (long long i = 0; i < n; ++i)
      if (!seen[(size_t)i]) {
        std::printf("FAIL s=%d,%d,%d: entry %lld unused\n", s[0], s[1], s[2], i);
        return 1;
      }
  }
  std::printf("OK %lld\n", total);
  return 0;
}
