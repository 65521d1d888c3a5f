// Double-float ("ff") arithmetic for the complex128 kernels.
//
// A double is carried as the unevaluated sum hi + lo of two floats (about 47
// significant bits), so the bulk arithmetic of complex128 kernels runs on the
// FP32 pipe, whose rate on GB300 is ~70x the FP64 rate (FP32 FMA 37 Top/s,
// FP64 0.5 Top/s measured).  The state in memory stays IEEE double; values
// are split on load and joined on store with integer bit manipulation, so
// a kernel issues no FP64 instruction at all.
//
// Error-free transformations: two-sum (Knuth, TAOCP vol. 2) and the
// fma-based two-product; products and sums are renormalised so that
// |lo| <= ulp(hi)/2 after every operation.  Relative error per operation is
// about 2^-46; the engine's tolerance on complex128 results is 1e-12
// absolute.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define FF_HD __host__ __device__ __forceinline__
#else
#define FF_HD inline
#endif

namespace qc {

struct ff {
  float hi, lo;
};
struct ffc {
  ff re, im;
};

FF_HD uint64_t ff_dbits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  memcpy(&b, &d, 8);
  return b;
#endif
}
FF_HD double ff_bitsd(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}
FF_HD uint32_t ff_fbits(float f) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
#endif
}
FF_HD float ff_bitsf(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
FF_HD float ff_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return __builtin_fmaf(a, b, c);
#endif
}
FF_HD int ff_rint(float x) {
#ifdef __CUDA_ARCH__
  return __float2int_rn(x);
#else
  return (int)__builtin_rintf(x);
#endif
}
// plain float operations that must not be fused or reassociated
FF_HD float ff_add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
FF_HD float ff_sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
FF_HD float ff_mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

// Float with 24-bit significand -> its double bit pattern (normal floats;
// zero and subnormal floats map to signed zero: |x| < 2^-126 is dropped).
FF_HD uint64_t ff_f2dbits(float x) {
  const uint32_t b = ff_fbits(x);
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  if (e == 0) return sign;
  return sign | ((uint64_t)(e - 127 + 1023) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29);
}

// double -> (hi, lo): hi = d truncated to 24 significant bits, lo = the
// remaining (up to 29) bits rounded to a float.  |d - (hi + lo)| <= 2^-47 |d|
// for 2^-74 <= |d| < 2^128; smaller magnitudes lose only absolute 2^-98.
FF_HD ff ff_from_d(double d) {
  const uint64_t b = ff_dbits(d);
  const uint32_t E = (uint32_t)((b >> 52) & 0x7FFu);
  ff r;
  if (E < 897u) {  // |d| < 2^-126: below float's normal range, negligible here
    r.hi = 0.f;
    r.lo = 0.f;
    return r;
  }
  // hi: sign, exponent re-biased, top 23 mantissa bits
  const uint32_t hb = (uint32_t)(b >> 63) << 31 | (E - 1023u + 127u) << 23 | (uint32_t)((b >> 29) & 0x7FFFFFu);
  r.hi = ff_bitsf(hb);
  const uint32_t low = (uint32_t)(b & 0x1FFFFFFFull);
  float lo = 0.f;
  if (E >= 949u && low) {  // 2^(E-1075) is a normal float
    lo = ff_mul_rn((float)low, ff_bitsf((E - 948u) << 23));
    if (b >> 63) lo = -lo;
  }
  r.lo = lo;
  return r;
}

// (hi, lo) with |lo| <= ulp(hi) -> the double nearest hi + lo (within one
// unit in the last place), by adding lo, in units of ulp_53(hi), to hi's
// bit pattern.
FF_HD double ff_to_d(ff x) {
  uint64_t hb = ff_f2dbits(x.hi);
  if ((hb << 1) == 0) return ff_bitsd(ff_f2dbits(x.lo));  // hi = 0
  const int E = (int)((hb >> 52) & 0x7FF);
  const int sc = 1075 - E + 127;  // float exponent field of 2^(1075 - E)
  if (sc <= 0 || sc >= 255) return ff_bitsd(hb);
  const float t = ff_mul_rn(x.lo, ff_bitsf((uint32_t)sc << 23));  // exact power-of-two scaling
  long long m = (long long)ff_rint(t);
  if (hb >> 63) m = -m;  // magnitude units
  // a power of two whose magnitude decreases lands in the binade below,
  // where one unit of the pattern is half as large
  if ((hb & 0x000FFFFFFFFFFFFFull) == 0 && m < 0) m *= 2;
  return ff_bitsd(hb + (uint64_t)m);
}

// Integer-lean conversions for the arithmetic-bound kernels (the general
// one-qubit operator, the QFT passes' conversions): about half the integer
// operations of ff_from_d / ff_to_d and no int-to-float conversion.  The
// streaming kernels (Hadamard, real operators, the Grover pass) keep the
// forms above, which measured faster there.
//
// double -> (hi, lo): hi = d truncated to 24 significant bits; lo = the
// remaining 29 bits rounded (half up) to a multiple of 2^6 of d's last unit,
// formed without an int-to-float conversion: the float 2^(E-1046)(1 + k/2^23)
// minus 2^(E-1046) is exactly k 2^(E-1069) (E = d's biased exponent; k <= 2^23,
// where the carry into the exponent gives the same difference).
// |d - (hi + lo)| <= 2^-47 |d| and |lo| <= ulp(hi) for 2^-103 <= |d| < 2^128;
// smaller magnitudes map to zero (an absolute error below 1e-31).
FF_HD ff ff_from_d_fast(double d) {
  const uint64_t b = ff_dbits(d);
  const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
  ff r;
  if ((bh & 0x7FF00000u) < (920u << 20)) {
    r.hi = 0.f;
    r.lo = 0.f;
    return r;
  }
  // sign, exponent re-biased from 1023 to 127 (subtracting 896 from the
  // field), mantissa bits 51..29
  const uint32_t hb = (bh & 0x80000000u) | (((uint32_t)(b >> 29) - (896u << 23)) & 0x7FFFFFFFu);
  const uint32_t eb = (hb & 0xFF800000u) - (23u << 23);  // sign | exponent field of 2^(E-1046)
  const uint32_t k = ((bl & 0x1FFFFFFFu) + 32u) >> 6;
  r.hi = ff_bitsf(hb);
  r.lo = ff_sub_rn(ff_bitsf(eb + k), ff_bitsf(eb));
  return r;
}

// (hi, lo) with |lo| <= ulp(hi) -> the double nearest hi + lo (within one
// unit in the last place): hi's binary64 pattern (exponent field + 896,
// mantissa << 29) plus lo in units of ulp_53(hi).  |hi| below 2^-75 (where
// that unit leaves float's range), zero included: the larger part alone.
FF_HD double ff_to_d_fast(ff x) {
  const uint32_t hb = ff_fbits(x.hi);
  const uint32_t ef = hb & 0x7F800000u;
  if (ef < (52u << 23)) return ff_bitsd(ff_f2dbits(ef ? x.hi : x.lo));
  const uint32_t dh = (hb & 0x80000000u) | (((hb & 0x7FFFFFFFu) >> 3) + (896u << 20));
  const uint32_t dl = hb << 29;
  const float t = ff_mul_rn(x.lo, ff_bitsf((306u << 23) - ef));  // lo / 2^(e_hi - 52), exact
  int m = ff_rint(t);
  if (hb >> 31) m = -m;  // magnitude units
  // a power of two whose magnitude decreases lands in the binade below,
  // where one unit of the pattern is half as large
  if ((hb & 0x7FFFFFu) == 0 && m < 0) m *= 2;
  return ff_bitsd((((uint64_t)dh << 32) | dl) + (uint64_t)(int64_t)m);
}

// Knuth two-sum: s + e == a + b exactly.
FF_HD void two_sum(float a, float b, float& s, float& e) {
  s = ff_add_rn(a, b);
  const float v = ff_sub_rn(s, a);
  e = ff_add_rn(ff_sub_rn(a, ff_sub_rn(s, v)), ff_sub_rn(b, v));
}

// Dekker fast two-sum: s + e == a + b exactly when |a| >= |b| (or a == 0).
// Used for the final renormalisation of a result whose high part dominates;
// where cancellation leaves it smaller, the error stays at the level of the
// low part (about 2^-48 of the operands), which absolute amplitude errors
// tolerate.
FF_HD void fast_two_sum(float a, float b, float& s, float& e) {
  s = ff_add_rn(a, b);
  e = ff_sub_rn(b, ff_sub_rn(s, a));
}

FF_HD ff ff_make(float hi, float lo) {
  ff r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

FF_HD ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = ff_add_rn(e, ff_add_rn(a.lo, b.lo));
  float h, l;
  fast_two_sum(s, e, h, l);
  return ff_make(h, l);
}
FF_HD ff ff_neg(ff a) { return ff_make(-a.hi, -a.lo); }
FF_HD ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
// a + b without the final renormalisation: hi = fl(a.hi + b.hi), lo = its
// exact rounding error plus the low parts, so hi + lo holds the sum to the
// same accuracy; only for a value that goes straight into another ff_add
// (whose two-sum of the high parts is exact for any inputs).
FF_HD ff ff_add_u(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return ff_make(s, ff_add_rn(e, ff_add_rn(a.lo, b.lo)));
}
FF_HD ff ff_sub_u(ff a, ff b) { return ff_add_u(a, ff_neg(b)); }

FF_HD ff ff_mul(ff a, ff b) {
  const float p = ff_mul_rn(a.hi, b.hi);
  float e = ff_fma(a.hi, b.hi, -p);
  e = ff_fma(a.hi, b.lo, e);
  e = ff_fma(a.lo, b.hi, e);
  float h, l;
  fast_two_sum(p, e, h, l);  // |e| <= ulp(p): exact
  return ff_make(h, l);
}

// a*b - c*d  (the real part of a complex product) with one renormalisation
FF_HD ff ff_dot2m(ff a, ff b, ff c, ff d) {
  const float p1 = ff_mul_rn(a.hi, b.hi);
  const float e1 = ff_fma(a.hi, b.hi, -p1);
  const float p2 = ff_mul_rn(c.hi, d.hi);
  const float e2 = ff_fma(c.hi, d.hi, -p2);
  float s, t;
  two_sum(p1, -p2, s, t);
  t = ff_add_rn(t, ff_sub_rn(e1, e2));
  t = ff_fma(a.hi, b.lo, t);
  t = ff_fma(a.lo, b.hi, t);
  t = ff_fma(-c.hi, d.lo, t);
  t = ff_fma(-c.lo, d.hi, t);
  float h, l;
  fast_two_sum(s, t, h, l);
  return ff_make(h, l);
}
// a*b + c*d
FF_HD ff ff_dot2p(ff a, ff b, ff c, ff d) { return ff_dot2m(a, b, ff_neg(c), d); }

// a*b + c*d + e*f + g*h with one closing renormalisation: the high
// products' rounding errors are exact (fma), their sum is carried by
// two-sums, and the low-part cross terms and the errors are summed in the
// low word.
FF_HD ff ff_dot4(ff a, ff b, ff c, ff d, ff e, ff f, ff g, ff h) {
  const float p1 = ff_mul_rn(a.hi, b.hi), p2 = ff_mul_rn(c.hi, d.hi);
  const float p3 = ff_mul_rn(e.hi, f.hi), p4 = ff_mul_rn(g.hi, h.hi);
  float t = ff_fma(a.hi, b.hi, -p1);
  t = ff_add_rn(t, ff_fma(c.hi, d.hi, -p2));
  t = ff_add_rn(t, ff_fma(e.hi, f.hi, -p3));
  t = ff_add_rn(t, ff_fma(g.hi, h.hi, -p4));
  float s, e1, e2, e3;
  two_sum(p1, p2, s, e1);
  two_sum(s, p3, s, e2);
  two_sum(s, p4, s, e3);
  t = ff_add_rn(t, ff_add_rn(e1, ff_add_rn(e2, e3)));
  t = ff_fma(a.hi, b.lo, t);
  t = ff_fma(a.lo, b.hi, t);
  t = ff_fma(c.hi, d.lo, t);
  t = ff_fma(c.lo, d.hi, t);
  t = ff_fma(e.hi, f.lo, t);
  t = ff_fma(e.lo, f.hi, t);
  t = ff_fma(g.hi, h.lo, t);
  t = ff_fma(g.lo, h.hi, t);
  float hh, ll;
  fast_two_sum(s, t, hh, ll);
  return ff_make(hh, ll);
}

// A running dot product sum a_i b_i of double-float operands with one
// closing renormalisation: the high products' sum s is carried by two-sums,
// and their rounding errors (fma), the cross terms a.hi b.lo + a.lo b.hi and
// the two-sums' errors accumulate in t.  About 13 FP32 operations per term
// with a renormalisation after every fourth.
struct ffacc {
  float s, t;
};
FF_HD ffacc ffacc_first(ff a, ff b) {
  ffacc A;
  A.s = ff_mul_rn(a.hi, b.hi);
  float t = ff_fma(a.hi, b.hi, -A.s);
  t = ff_fma(a.hi, b.lo, t);
  A.t = ff_fma(a.lo, b.hi, t);
  return A;
}
FF_HD void ffacc_add(ffacc& A, ff a, ff b) {
  const float p = ff_mul_rn(a.hi, b.hi);
  float t = ff_fma(a.hi, b.hi, -p);
  t = ff_fma(a.hi, b.lo, t);
  t = ff_fma(a.lo, b.hi, t);
  float s, e;
  two_sum(A.s, p, s, e);
  A.s = s;
  A.t = ff_add_rn(A.t, ff_add_rn(t, e));
}
// moves t into s (fast two-sum; |t| stays far below |s| between calls), so
// that t's own roundings stay at 2^-24 of a few units of s.  Called after
// every fourth term, the error of up to 64 terms stays below 2^-44 of
// sum |a_i b_i| (mostly the operands' own splitting error); without it the
// low word's roundings grow with the square of the number of terms.
FF_HD void ffacc_norm(ffacc& A) {
  float h, l;
  fast_two_sum(A.s, A.t, h, l);
  A.s = h;
  A.t = l;
}
FF_HD ff ffacc_result(const ffacc& A) {
  float h, l;
  fast_two_sum(A.s, A.t, h, l);
  return ff_make(h, l);
}

FF_HD ffc ffc_make(ff re, ff im) {
  ffc z;
  z.re = re;
  z.im = im;
  return z;
}
FF_HD ffc ffc_add(ffc a, ffc b) { return ffc_make(ff_add(a.re, b.re), ff_add(a.im, b.im)); }
FF_HD ffc ffc_sub(ffc a, ffc b) { return ffc_make(ff_sub(a.re, b.re), ff_sub(a.im, b.im)); }
FF_HD ffc ffc_add_u(ffc a, ffc b) { return ffc_make(ff_add_u(a.re, b.re), ff_add_u(a.im, b.im)); }
FF_HD ffc ffc_sub_u(ffc a, ffc b) { return ffc_make(ff_sub_u(a.re, b.re), ff_sub_u(a.im, b.im)); }
FF_HD ffc ffc_mul(ffc a, ffc b) {
  return ffc_make(ff_dot2m(a.re, b.re, a.im, b.im), ff_dot2p(a.re, b.im, a.im, b.re));
}
// a*b + c*d for complex values
FF_HD ffc ffc_mul2(ffc a, ffc b, ffc c, ffc d) { return ffc_add(ffc_mul(a, b), ffc_mul(c, d)); }
// complex times a real ff
FF_HD ffc ffc_scale(ffc a, ff r) { return ffc_make(ff_mul(a.re, r), ff_mul(a.im, r)); }

FF_HD ffc ffc_from_d(double re, double im) { return ffc_make(ff_from_d(re), ff_from_d(im)); }

}  // namespace qc
