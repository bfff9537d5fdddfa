// Host-side check of the double-float arithmetic (df64.h) against FP64: for operands
// spread over 40 decades and both signs, each operation's result, converted back to
// double, lies within its stated bound of the FP64 result of the same (exactly
// represented) operands:
//   conversion   |x - to_double(to_df64(x))| <= 2^-45 |x|
//   a + b, a - b <= 2^-46 (|a| + |b|)
//   a * b        <= 2^-46 |a b| + 2^-120
//   a / b        <= 2^-42 |a / b| + 2^-120  (the device's reciprocal estimate is
//                                    checked on the GPU; here it is IEEE division)
//   mul_u, div_u (unnormalised): the same bounds as *, /; |lo| <= 2^-21 |hi|; the sign
//   of hi is the sign of the value; as operands of +, * and / they keep the bounds of
//   the two operations added
// The absolute floor 2^-120: below about 2^-102 the low float of a result leaves the
// normal range of float, so its relative precision falls (on the device, where
// subnormals flush to zero, the loss is below 2^-126 absolutely); the stencils' fields
// are compared with an absolute tolerance far above it.
// Prints "OK <checks>" and exits 0, or the first failure and exits 1.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "df64.h"

using namespace dfn;

static uint64_t rng = 0x2545f4914f6cdd1dull;
static double uniform() {  // xorshift64*, [0, 1)
  rng ^= rng >> 12;
  rng ^= rng << 25;
  rng ^= rng >> 27;
  return (double)((rng * 0x2545f4914f6cdd1dull) >> 11) * 0x1.0p-53;
}
static double operand() {
  const double mag = std::pow(10.0, -20.0 + 22.0 * uniform());
  return (uniform() < 0.5 ? -1.0 : 1.0) * mag * (1.0 + uniform());
}

int main() {
  long long n = 0;
  for (int k = 0; k < 2000000; ++k) {
    const double x = operand(), y = operand();
    const df64 a = to_df64(x), b = to_df64(y);
    const double A = to_double(a), B = to_double(b);
    ++n;
    if (std::fabs(A - x) > 0x1.0p-45 * std::fabs(x)) {
      std::printf("FAIL conversion %.17g -> %.17g\n", x, A);
      return 1;
    }
    const double s = to_double(a + b), d = to_double(a - b);
    const double m = to_double(a * b), q = to_double(a / b);
    const double sb = 0x1.0p-46 * (std::fabs(A) + std::fabs(B));
    if (std::fabs(s - (A + B)) > sb || std::fabs(d - (A - B)) > sb) {
      std::printf("FAIL add %.17g %.17g: %.17g %.17g\n", A, B, s, d);
      return 1;
    }
    if (std::fabs(m - A * B) > 0x1.0p-46 * std::fabs(A * B) + 0x1.0p-120) {
      std::printf("FAIL mul %.17g %.17g: %.17g\n", A, B, m);
      return 1;
    }
    if (std::fabs(q - A / B) > 0x1.0p-42 * std::fabs(A / B) + 0x1.0p-120) {
      std::printf("FAIL div %.17g %.17g: %.17g\n", A, B, q);
      return 1;
    }
    // sign tests follow the value's sign
    if (gt0(a) != (A > 0) || lt0(a) != (A < 0)) {
      std::printf("FAIL sign %.17g\n", A);
      return 1;
    }
    // unnormalised product and quotient, alone and as operands (value of a pair:
    // hi + lo in double, exact to 2^-53)
    const double C3 = to_double(to_df64(operand()));
    const df64 c = to_df64(C3);
    const df64 mu = mul_u(a, b), qu = div_u(a, b);
    const double MU = (double)mu.hi + (double)mu.lo, QU = (double)qu.hi + (double)qu.lo;
    const double AB = A * B, QB = A / B;
    if (std::fabs(MU - AB) > 0x1.0p-46 * std::fabs(AB) + 0x1.0p-120 ||
        std::fabs(QU - QB) > 0x1.0p-42 * std::fabs(QB) + 0x1.0p-120 ||
        std::fabs(mu.lo) > 0x1.0p-21 * std::fabs(mu.hi) ||
        std::fabs(qu.lo) > 0x1.0p-21 * std::fabs(qu.hi) || gt0(mu) != (AB > 0) ||
        lt0(mu) != (AB < 0) || gt0(qu) != (QB > 0)) {
      std::printf("FAIL mul_u/div_u %.17g %.17g: %.17g %.17g\n", A, B, MU, QU);
      return 1;
    }
    // (as operands: where the unnormalised pair's low float is itself normal, |value|
    // >= 2^-100; below, its absolute error, within the floor, is what a quotient scales)
    const double s2 = to_double(mu + c), m2 = to_double(mu * c), q2 = to_double(mu / c);
    const double m3 = to_double(mul_u(qu, c) + c);
    if (std::fabs(AB) >= 0x1.0p-100 && std::fabs(QB) >= 0x1.0p-100 &&
        (std::fabs(s2 - (AB + C3)) > 0x1.0p-45 * (std::fabs(AB) + std::fabs(C3)) + 0x1.0p-120 ||
        std::fabs(m2 - AB * C3) > 0x1.0p-45 * std::fabs(AB * C3) + 0x1.0p-120 ||
        std::fabs(q2 - AB / C3) > 0x1.0p-41 * std::fabs(AB / C3) + 0x1.0p-120 ||
        std::fabs(m3 - (QB * C3 + C3)) >
            0x1.0p-41 * (std::fabs(QB * C3) + std::fabs(C3)) + 0x1.0p-120)) {
      std::printf("FAIL unnormalised operands %.17g %.17g %.17g\n", A, B, C3);
      return 1;
    }
  }
  // the conversions against the compiler's: to_double of a normalised pair is the
  // correctly rounded sum to within one unit in the last place, and a float converts
  // exactly both ways
  for (int k = 0; k < 2000000; ++k) {
    const double x = operand();
    const float h = (float)x, l = (float)(x - (double)h);
    const double ref = (double)h + (double)l;
    const double got = to_double(df64(h, l));
    if (std::fabs(got - ref) > 0x1.0p-52 * std::fabs(ref)) {
      std::printf("FAIL to_double %.17g %.9g %.9g: %.17g\n", ref, h, l, got);
      return 1;
    }
    const df64 f = to_df64((double)h);
    if (f.hi != h || f.lo != 0.f || to_double(df64(h)) != (double)h) {
      std::printf("FAIL float round trip %.9g\n", h);
      return 1;
    }
    ++n;
  }
  // the stored form of the FP64 state (canonical): its value is a double, the cut
  // moves it by less than 2^-45 of itself, it is its own canonical form, and it
  // survives the trip through double bit for bit (results of sums, products and
  // quotients, whose low parts take every size, and values down to 1e-30, below the
  // 2^-80 where lo becomes 0 and hi alone stands for the value, as in to_df64)
  for (int k = 0; k < 2000000; ++k) {
    const double x = operand() * (k % 7 == 0 ? 1e-10 : 1.0), y = operand();
    const df64 a = to_df64(x), b = to_df64(y);
    const df64 r = k % 3 == 0 ? a + b : (k % 3 == 1 ? a * b : a / b);
    const df64 c = canonical(r);
    const double v = to_double(c), vr = to_double(r);
    const double cut = std::fabs(vr) < 0x1.0p-79 ? 0x1.0p-23 : 0x1.0p-45;  // hi alone below
    if (v != (double)c.hi + (double)c.lo || std::fabs(v - vr) > cut * std::fabs(vr)) {
      std::printf("FAIL canonical value %.17g %.17g\n", vr, v);
      return 1;
    }
    const df64 cc = canonical(c), back = to_df64(v);
    // (bit for bit but for the sign of a zero lo: to_df64 gives -0 beside a negative hi
    // where the cut leaves +0; the pairs' values are the same double)
    if (f2u(cc.hi) != f2u(c.hi) || f2u(cc.lo) != f2u(c.lo) || f2u(back.hi) != f2u(c.hi) ||
        (f2u(back.lo) != f2u(c.lo) && !(back.lo == 0.f && c.lo == 0.f))) {
      std::printf("FAIL canonical round trip %.17g: (%a, %a) -> (%a, %a)\n", v, c.hi, c.lo,
                  back.hi, back.lo);
      return 1;
    }
    ++n;
  }
  // signed zeros, infinities and NaN survive both conversions
  if (to_double(to_df64(-0.0)) != 0.0 || !std::signbit(to_double(to_df64(-0.0))) ||
      !std::isinf(to_double(to_df64(1e300))) || !std::isnan(to_double(to_df64(NAN)))) {
    std::printf("FAIL special values\n");
    return 1;
  }
  // exact cases: zero stays zero, x - x = 0, 1 * x = x
  const df64 z = df64(0.f);
  if (to_double(z + z) != 0.0 || to_double(to_df64(0.3) - to_df64(0.3)) != 0.0 ||
      to_double(df64(1.f) * to_df64(0.3)) != to_double(to_df64(0.3))) {
    std::printf("FAIL exact cases\n");
    return 1;
  }
  std::printf("OK %lld\n", n);
  return 0;
}
