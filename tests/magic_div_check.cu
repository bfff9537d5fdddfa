// Host-side check of the box decode's division by multiply-shift (Box::magic in
// internal.h): for divisors up to 4096 and sampled plane sizes up to 2^20 + 2^19,
// (t m) >> s equals t / d at every quotient boundary (t = k d - 1, k d, k d + 1) of a
// sample of k with t < 2^31, and at pseudo-random t.  Prints "OK <checks>" and exits
// 0, or "FAIL d t" and exits 1.
#include <cstdint>
#include <cstdio>

#include "internal.h"

using namespace dfn;

static uint64_t rng = 0x9e3779b97f4a7c15ull;
static uint32_t next31() {  // xorshift64*, top 31 bits
  rng ^= rng >> 12;
  rng ^= rng << 25;
  rng ^= rng >> 27;
  return (uint32_t)((rng * 0x2545f4914f6cdd1dull) >> 33);
}

static bool check(unsigned d, long long& n) {
  unsigned long long m;
  int s;
  Box::magic(d, m, s);
  auto ok = [&](unsigned long long t) {
    if (t >= (1ull << 31)) return true;
    ++n;
    return ((t * m) >> s) == t / d;
  };
  const unsigned long long kmax = ((1ull << 31) - 1) / d;
  for (unsigned long long j = 0; j < 200; ++j) {
    const unsigned long long k = j < 100 ? j + 1 : kmax - (j - 100);
    for (long long e = -1; e <= 1; ++e) {
      const long long t = (long long)(k * d) + e;
      if (t >= 0 && !ok((unsigned long long)t)) {
        std::printf("FAIL %u %lld\n", d, t);
        return false;
      }
    }
  }
  for (int i = 0; i < 2000; ++i) {
    const unsigned long long t = next31();
    if (!ok(t)) {
      std::printf("FAIL %u %llu\n", d, t);
      return false;
    }
  }
  return true;
}

int main() {
  long long n = 0;
  for (unsigned d = 1; d <= 4096; ++d)
    if (!check(d, n)) return 1;
  for (int i = 0; i < 4000; ++i) {
    const unsigned d = 4097 + next31() % ((1u << 20) + (1u << 19));
    if (!check(d, n)) return 1;
  }
  const unsigned edge[] = {(1u << 20) - 1, 1u << 20, (1u << 20) + 1, 1040u * 1040u, 65535u, 65536u};
  for (unsigned d : edge)
    if (!check(d, n)) return 1;
  std::printf("OK %lld\n", n);
  return 0;
}
