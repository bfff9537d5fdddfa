// df64.h -- double-float arithmetic for the FP64 stencils.
//
// A df64 holds a value as the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2: a 48-bit significand (relative rounding 2^-48, about 3.6e-15)
// computed entirely on the FP32 pipe.  GB300 executes FP64 at 1/64 of its FP32 rate,
// so the FP64 state's stencils (bound by that pipe) run their arithmetic in this
// type; the state itself stays FP64 in memory.
//
// Published error-free transformations:
//   two_sum       Knuth, The Art of Computer Programming vol. 2 (1969), 4.2.2:
//                 s = fl(a + b) and the exact error e, a + b = s + e, for any a, b;
//   fast_two_sum  Dekker, Numer. Math. 18 (1971): the same in 3 operations when
//                 |a| >= |b| (or a = 0);
//   two_prod      the exact error of a product from one fused multiply-add:
//                 a b = p + fma(a, b, -p) (no overflow or underflow);
// and the double-length operations built on them (Dekker 1971, the same algorithms
// as the double-double library of Hida, Li & Bailey, ARITH 15, 2001, with float in
// place of double).  Each operation below rounds its result to about 2^-48 of the
// operands' magnitude; the sums are the "sloppy" variant, whose error is bounded
// absolutely by 2^-47 (|a| + |b|) rather than relatively to a + b, which is the
// bound the state's absolute tolerance needs.
//
// These functions must be compiled without reassociation of float additions (nvcc's
// default): the error terms rely on IEEE rounding of every operation.
#pragma once

#include <math.h>

namespace dfn {

struct __align__(8) df64 {  // 8-byte aligned: one 64-bit load or store per value
  float hi, lo;
  df64() = default;  // trivial, so it may live in shared memory; {} gives zeros
  __host__ __device__ constexpr df64(float h) : hi(h), lo(0.f) {}
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
};

__host__ __device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df64(s, (a - (s - bb)) + (b - bb));
}

__host__ __device__ __forceinline__ df64 fast_two_sum(float a, float b) {
  const float s = a + b;
  return df64(s, b - (s - a));
}

__host__ __device__ __forceinline__ df64 two_prod(float a, float b) {
  const float p = a * b;
  return df64(p, fmaf(a, b, -p));
}

__host__ __device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

__host__ __device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  df64 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__host__ __device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__host__ __device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  df64 p = two_prod(a.hi, b.hi);
  float e = fmaf(a.hi, b.lo, p.lo);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p.hi, e);
}

// reciprocal estimate of a float: the hardware approximation on the device (its
// error is removed by the correction step of the division), IEEE division on the host
__host__ __device__ __forceinline__ float rcp_est(float b) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
  return r;
#else
  return 1.0f / b;
#endif
}

// a / b: q1 from the reciprocal estimate, the remainder a - b q1, then one correction
// q2 = remainder * r (the long division of Dekker 1971).  The remainder is about
// 2^-22 |a|, so it needs no double-float sum: one fused multiply-add gives
// a.hi - b.hi q1 rounded once (2^-24 of the remainder, about 2^-46 |a|), a second
// takes away b.lo q1 and adds a.lo.  The quotient's relative error is about the
// square of q1's (2^-22 each, so about 2^-44, 6e-14) plus those roundings.
// For the normal, non-zero divisors of the stencils (densities, 1 + a, sums of two
// same-signed slopes).
__host__ __device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  const float r = rcp_est(b.hi);
  const float q1 = a.hi * r;
  const float rem = fmaf(-b.lo, q1, fmaf(-b.hi, q1, a.hi) + a.lo);
  return fast_two_sum(q1, rem * r);
}

// a times a power of two (exact, both parts scaled; no overflow or underflow)
// A product and a quotient without the final renormalisation: the pair (p, e) of the
// operators above before their fast_two_sum, which is exact, so the value and its error
// are the same; e may reach about 2^-22 |p| instead of half an ulp of p.  Such a pair is
// an operand of +, -, * and / (their error bounds hold with |lo| <= 2^-21 |hi|) and of
// the sign tests (p carries the sign), never of canonical(), to_double() or an ordered
// comparison.  Three instructions fewer each, where the result feeds more arithmetic.
__host__ __device__ __forceinline__ df64 mul_u(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  return df64(p, fmaf(a.lo, b.hi, e));
}
__host__ __device__ __forceinline__ df64 div_u(df64 a, df64 b) {
  const float r = rcp_est(b.hi);
  const float q1 = a.hi * r;
  const float rem = fmaf(-b.lo, q1, fmaf(-b.hi, q1, a.hi) + a.lo);
  return df64(q1, rem * r);
}

__host__ __device__ __forceinline__ df64 scale(df64 a, float p2) {
  return df64(a.hi * p2, a.lo * p2);
}

__host__ __device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__host__ __device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }

// sign tests: the sign of hi is the sign of the value (hi = fl(hi + lo))
__host__ __device__ __forceinline__ bool gt0(df64 v) { return v.hi > 0.f; }
__host__ __device__ __forceinline__ bool le0(df64 v) { return !(v.hi > 0.f); }
__host__ __device__ __forceinline__ bool lt0(df64 v) { return v.hi < 0.f; }

// ---- conversions between double and double-float, in integer arithmetic.
// GB300 converts between double and float on its FP64 pipe (measured: about 2
// conversions per SM per cycle, the rate of an FP64 add, against 113 FP32 multiply-
// adds), so (float)x and (double)f would cost the stencils as much as the FP64
// arithmetic they replace.  These work on the bit patterns instead (integer and FP32
// instructions only).  Values below 2^-126 in magnitude become 0 (the stencils'
// tolerance is absolute and far above that), infinities and NaNs are kept.

__host__ __device__ __forceinline__ unsigned f2u(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  __builtin_memcpy(&u, &f, 4);
  return u;
#endif
}
__host__ __device__ __forceinline__ float u2f(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  __builtin_memcpy(&f, &u, 4);
  return f;
#endif
}
__host__ __device__ __forceinline__ unsigned long long d2u(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long u;
  __builtin_memcpy(&u, &d, 8);
  return u;
#endif
}
__host__ __device__ __forceinline__ double u2d(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  __builtin_memcpy(&d, &u, 8);
  return d;
#endif
}

// x = hi + lo: x cut to 24 significant bits (the double's bit pattern shifted and its
// exponent re-biased) plus the next 23 bits of the remainder as a float (the 2^23
// magic-number conversion, scaled by a power of two built with the remainder's sign),
// then normalised; error below 2^-45 |x|.  |x| below 2^-80 keeps hi alone; |x| below
// 2^-126 becomes 0.
__host__ __device__ __forceinline__ df64 to_df64(double x) {
  const unsigned long long b = d2u(x);
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  const unsigned sign = bh & 0x80000000u;
  const unsigned e = (bh >> 20) & 0x7FFu;  // biased exponent of x
  if (e - 897u >= 254u) {                   // outside float's normal range
    if (e < 897u) return df64(u2f(sign), 0.f);
    const bool nan = e == 0x7FFu && (((bh & 0xFFFFFu) | bl) != 0u);
    return df64(u2f(nan ? 0x7FC00000u : (sign | 0x7F800000u)), 0.f);
  }
  // sign | exponent | top 23 fraction bits, exponent re-biased from 1023 to 127
  const unsigned hb = (unsigned)(((b >> 29) & 0x3FFFFFFFFull) - (896ull << 23));
  const float hi = u2f(sign | hb);
  // the remainder's next 23 bits, times 2^(e - 1069) carrying x's sign
  const float r = u2f(0x4B000000u | ((bl >> 6) & 0x7FFFFFu)) - 8388608.0f;
  const float p2 = e >= 943u ? u2f(sign | ((e - 942u) << 23)) : 0.f;
  return fast_two_sum(hi, r * p2);
}

// hi + lo rounded to double: hi's significand and lo's, aligned in a 64-bit integer
// (|lo| < ulp(hi), so the sum stays within one binade step of hi)
__host__ __device__ __forceinline__ double to_double(df64 v) {
  const unsigned sh = f2u(v.hi), sl = f2u(v.lo);
  const int eh = (int)((sh >> 23) & 0xFFu), el = (int)((sl >> 23) & 0xFFu);
  const unsigned long long sign = (unsigned long long)(sh & 0x80000000u) << 32;
  if (eh == 0) return u2d(sign);  // zero (subnormal hi: flushed)
  if (eh == 255)                  // infinity or NaN
    return u2d(sign | 0x7FF0000000000000ull |
               ((unsigned long long)(sh & 0x7FFFFFu) << 29));
  unsigned long long S = (unsigned long long)((sh & 0x7FFFFFu) | 0x800000u) << 29;
  if (el != 0) {
    const unsigned long long ml = (sl & 0x7FFFFFu) | 0x800000u;
    const int shift = el - eh + 29;  // lo in units of 2^-52 of hi's binade
    unsigned long long L = 0;
    if (shift >= 0)
      L = ml << shift;
    else if (shift > -25)
      L = ml >> (-shift);
    if ((sl ^ sh) & 0x80000000u)
      S -= L;
    else
      S += L;
  }
  int ex = eh - 127 + 1023;
  if (S < (1ull << 52)) {  // fell below hi's binade: renormalise
    S <<= 1;
    ex -= 1;
  }
  return u2d(sign | ((unsigned long long)ex << 52) | (S & 0xFFFFFFFFFFFFFull));
}

// ---- the FP64 state as stored.  A double-float pair whose value is a double: lo is
// cut (toward zero) to a multiple of 2^-23 ulp(hi), so hi + lo has at most 47
// significant bits and no bit below 2^-46 of hi's binade.  to_double of such a pair is
// exact and to_df64 of that double gives the same pair back (hi = the 24-bit value
// nearest to hi + lo, as the error-free transformations leave it), so the state
// converts to and from FP64 without loss while the stencils load and store the pairs
// directly.  Where |hi| < 2^-80 (to_df64 keeps hi alone there) lo becomes 0, and a
// subnormal hi becomes a zero of its sign (both conversions flush it).
struct __align__(8) dstate {
  float hi, lo;
};

__host__ __device__ __forceinline__ df64 canonical(df64 v) {
  const unsigned uh = f2u(v.hi), ul = f2u(v.lo);
  const int eh = (int)((uh >> 23) & 0xFFu), el = (int)((ul >> 23) & 0xFFu);
  const int k = eh - el - 23;  // bits of lo's significand below the grid
  unsigned lo = 0u;
  if (eh >= 47 && k < 24) lo = k > 0 ? ul & (0xFFFFFFFFu << k) : ul;
  return df64(eh == 0 ? u2f(uh & 0x80000000u) : v.hi, u2f(lo));
}

}  // namespace dfn
