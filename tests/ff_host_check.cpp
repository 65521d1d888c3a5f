// Host-side check of the double-float layer the complex128 kernels use
// (paper_0902_0699_gb300/csrc/ff.cuh compiled as plain C++): conversions
// double <-> (hi, lo) (both conversion pairs) and the ff arithmetic against
// long double references.
// Prints "ok" and exits 0, or prints the first failure and exits 1.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>

#include "../paper_0902_0699_gb300/csrc/ff.cuh"

using namespace qc;

static long double val(ff x) { return (long double)x.hi + (long double)x.lo; }

static int fail(const char* what, double a, double b, long double err) {
  printf("FAIL %s: a=%.17g b=%.17g err=%Lg\n", what, a, b, err);
  return 1;
}

// The conversions' stated bounds: |d - (hi + lo)| <= 2^-47 |d| and
// |lo| <= ulp(hi) for 2^-103 <= |d| < 2^128 (2^-74 for the general form;
// the lean form maps smaller magnitudes to zero), including low words that round up into the next
// power of two; and the join of any (hi, lo) with |lo| <= ulp(hi) within one
// unit of hi + lo.
template <typename FROM, typename TO>
static int conversion_bounds(FROM from_d, TO to_d, bool zero_below, std::mt19937_64& rng) {
  std::uniform_int_distribution<uint64_t> M(0, (1ull << 52) - 1);
  std::uniform_int_distribution<int> EX(-103, 127);
  for (int i = 0; i < 3000000; ++i) {
    uint64_t mant = M(rng);
    if (i % 4 == 1) mant |= (1ull << 29) - 1 - (i & 31);  // low word at the top of its range
    if (i % 4 == 2) mant &= ~((1ull << 29) - 1);          // low word zero
    const double d = std::ldexp(1.0 + std::ldexp((double)mant, -52), EX(rng)) * ((i & 8) ? -1.0 : 1.0);
    const ff f = from_d(d);
    const long double err = std::fabs(val(f) - (long double)d);
    // the general form keeps the relative bound from 2^-74 up (below it the
    // low word is dropped: an absolute error under 2^-98)
    const long double fb = (zero_below || std::fabs(d) >= std::ldexp(1.0, -74)) ? std::ldexp(std::fabs((long double)d), -47)
                                                                                 : std::ldexp((long double)1, -98);
    if (err > fb) return fail("from_d 2^-47", d, 0, err);
    const float uh = std::ldexp(1.0f, std::ilogb(f.hi) - 23);
    if (std::fabs(f.lo) > uh) return fail("from_d |lo| <= ulp(hi)", d, 0, f.lo);
    if ((f.hi < 0) != (d < 0) || (f.lo != 0 && (f.lo < 0) != (d < 0))) return fail("from_d sign", d, 0, 0);
    // the join keeps the low word for |hi| >= 2^-75 (below: hi alone, an
    // absolute error under 2^-98; the general split keeps it from 2^-74)
    const double back = to_d(f);
    const double rt = std::fabs(d) >= std::ldexp(1.0, -74) ? std::ldexp(std::fabs(d), -47) : std::ldexp(1.0, -98);
    if (std::fabs(back - d) > rt) return fail("round trip 2^-47", d, back, back - d);
  }
  if (zero_below)
    for (double d : {std::ldexp(1.0, -104), -std::ldexp(1.7, -110), 1e-300}) {
      const ff f = from_d(d);
      if (f.hi != 0.f || f.lo != 0.f) return fail("below 2^-103", d, 0, f.hi);
    }
  std::uniform_real_distribution<float> UF(-1.0f, 1.0f);
  for (int i = 0; i < 3000000; ++i) {
    const float hi = std::ldexp(1.0f + std::fabs(UF(rng)), EX(rng) / 2) * ((i & 1) ? -1.f : 1.f);
    const float lo = UF(rng) * std::ldexp(1.0f, std::ilogb(hi) - 23);
    const long double want = (long double)hi + (long double)lo;
    const double got = to_d(ff_make(hi, lo));
    const long double ulp = std::ldexp((long double)1, std::ilogb((double)want) - 52);
    if (std::fabs((long double)got - want) > ulp) return fail("join", (double)want, got, got - want);
  }
  // exact edges and the binade below a power of two
  for (double d : {0.0, -0.0, 1.0, -1.0, 0.5, 0.7071067811865476, -0.7071067811865476, 1e-30}) {
    const double b = to_d(from_d(d));
    if (std::fabs(b - d) > std::fmax(std::ldexp(std::fabs(d), -46), std::ldexp(1.0, -97))) return fail("edge", d, b, b - d);
  }
  for (int e = -40; e <= 4; ++e)
    for (int k = 1; k < 1000; ++k) {
      const float hi = std::ldexp(1.0f, e), lo = -std::ldexp((float)k, e - 34);
      const double want = (double)hi + (double)lo;
      if (std::fabs(to_d(ff_make(hi, lo)) - want) > std::ldexp(1.0, e - 52)) return fail("binade", want, 0, 0);
      if (std::fabs(to_d(ff_make(-hi, -lo)) + want) > std::ldexp(1.0, e - 52)) return fail("binade neg", -want, 0, 0);
    }
  return 0;
}

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::uniform_int_distribution<int> X(-70, 8);
  // 1. round trips and representation error
  for (int i = 0; i < 2000000; ++i) {
    const double d = std::ldexp(U(rng), X(rng));
    const ff f = ff_from_d(d);
    // relative 2^-46, with an absolute floor of 2^-97 below |d| = 2^-74
    const double tol = std::fmax(std::ldexp(std::fabs(d), -46), std::ldexp(1.0, -97));
    if (std::fabs((double)(val(f) - (long double)d)) > tol) return fail("from_d", d, 0, val(f) - d);
    if (std::fabs(f.lo) > std::fabs(f.hi) * std::ldexp(1.0, -23)) return fail("from_d norm", d, 0, f.lo);
    const double back = ff_to_d(f);
    if (std::fabs(back - d) > tol) return fail("round trip", d, back, back - d);
  }
  // 2. exact edge cases
  const double edge[] = {0.0, -0.0, 1.0, -1.0, 0.5, 0.7071067811865476, -0.7071067811865476, 1e-30, 3e-39, 1e-300};
  for (double d : edge) {
    const double back = ff_to_d(ff_from_d(d));
    const double tol = std::fmax(std::ldexp(std::fabs(d), -46), std::ldexp(1.0, -97));
    if (std::fabs(back - d) > tol) return fail("edge", d, back, back - d);
  }
  // 3. join at a power of two with a lo of opposite sign (binade below)
  for (int e = -40; e <= 4; ++e) {
    for (int k = 1; k < 1000; ++k) {
      const float hi = std::ldexp(1.0f, e);
      const float lo = -std::ldexp((float)k, e - 34);  // |lo| < ulp(hi)/2
      const double want = (double)hi + (double)lo;
      const double got = ff_to_d(ff_make(hi, lo));
      if (std::fabs(got - want) > std::ldexp(1.0, e - 52)) return fail("binade", want, got, got - want);
      const double got2 = ff_to_d(ff_make(-hi, -lo));
      if (std::fabs(got2 + want) > std::ldexp(1.0, e - 52)) return fail("binade neg", -want, got2, got2 + want);
    }
  }
  // 4. arithmetic: relative (to operand size) error bounds
  for (int i = 0; i < 1000000; ++i) {
    const double a = std::ldexp(U(rng), X(rng) / 4), b = std::ldexp(U(rng), X(rng) / 4);
    const double c = std::ldexp(U(rng), X(rng) / 4), d = std::ldexp(U(rng), X(rng) / 4);
    const ff A = ff_from_d(a), B = ff_from_d(b), C = ff_from_d(c), D = ff_from_d(d);
    const long double sc = std::fabs(a) + std::fabs(b);
    long double err = std::fabs(val(ff_add(A, B)) - ((long double)a + b));
    if (err > std::ldexp(sc, -45)) return fail("add", a, b, err);
    err = std::fabs(val(ff_sub(A, B)) - ((long double)a - b));
    if (err > std::ldexp(sc, -45)) return fail("sub", a, b, err);
    err = std::fabs(val(ff_mul(A, B)) - (long double)a * b);
    if (err > std::ldexp(std::fabs(a * b), -44)) return fail("mul", a, b, err);
    const long double ref = (long double)a * b - (long double)c * d;
    err = std::fabs(val(ff_dot2m(A, B, C, D)) - ref);
    if (err > std::ldexp(std::fabs(a * b) + std::fabs(c * d), -44)) return fail("dot2m", a, c, err);
    // joins of arithmetic results stay within the same bound
    const double j = ff_to_d(ff_add(A, B));
    if (std::fabs(j - ((long double)a + b)) > std::ldexp(sc, -44)) return fail("join add", a, b, j - (a + b));
    // unnormalised first-level sums (radix-4 butterflies) carry the value, and
    // a normalising second level over them keeps the bound
    err = std::fabs(val(ff_add_u(A, B)) - ((long double)a + b));
    if (err > std::ldexp(sc, -45)) return fail("add_u", a, b, err);
    err = std::fabs(val(ff_sub_u(A, B)) - ((long double)a - b));
    if (err > std::ldexp(sc, -45)) return fail("sub_u", a, b, err);
    const long double sc4 = sc + std::fabs(c) + std::fabs(d);
    const ff S0 = ff_add_u(A, B), S1 = ff_add_u(C, D), D0 = ff_sub_u(A, B), D1 = ff_sub_u(C, D);
    err = std::fabs(val(ff_add(S0, S1)) - (((long double)a + b) + ((long double)c + d)));
    if (err > std::ldexp(sc4, -44)) return fail("radix4 t0", a, c, err);
    err = std::fabs(val(ff_sub(D0, D1)) - (((long double)a - b) - ((long double)c - d)));
    if (err > std::ldexp(sc4, -44)) return fail("radix4 u1", a, c, err);
    const ff T = ff_add(S0, S1);
    if (std::fabs(T.lo) > std::fabs(T.hi) * std::ldexp(1.0, -23)) return fail("radix4 norm", a, c, T.lo);
    // a product over an unnormalised sum (the twiddle after a radix-4 step)
    const long double pm = (long double)c * ((long double)a - b);
    err = std::fabs(val(ff_mul(C, D0)) - pm);
    if (err > std::ldexp(std::fabs(c) * sc, -43)) return fail("mul over sub_u", a, c, err);
    err = std::fabs(val(ff_dot2m(C, D0, D, S0)) - (pm - (long double)d * ((long double)a + b)));
    if (err > std::ldexp((std::fabs(c) + std::fabs(d)) * sc, -43)) return fail("dot2m over add_u", a, c, err);
    // the four-term dot of the general one-qubit operator (one renormalisation)
    const long double r4 = (long double)a * b + (long double)c * d + (long double)b * c - (long double)a * d;
    err = std::fabs(val(ff_dot4(A, B, C, D, B, C, ff_neg(A), D)) - r4);
    const long double s4 = std::fabs(a * b) + std::fabs(c * d) + std::fabs(b * c) + std::fabs(a * d);
    if (err > std::ldexp(s4, -43)) return fail("dot4", a, c, err);  // four products, ~12 low-word roundings
    const ff R4 = ff_dot4(A, B, C, D, B, C, ff_neg(A), D);
    if (std::fabs(R4.lo) > std::fabs(R4.hi) * std::ldexp(1.0, -23) + std::ldexp(s4, -70))
      return fail("dot4 norm", a, c, R4.lo);
  }
  // 5. running dots of up to 64 terms, renormalised after every fourth (the
  // dense blocks' accumulation): within 2^-43 of sum |a_i b_i|
  for (int i = 0; i < 200000; ++i) {
    const int nt = 1 + (i % 64);
    double a[64], b[64];
    long double ref = 0, mag = 0;
    ffacc A{};
    for (int j = 0; j < nt; ++j) {
      a[j] = std::ldexp(U(rng), X(rng) / 8);
      b[j] = std::ldexp(U(rng), X(rng) / 8);
      ref += (long double)a[j] * b[j];
      mag += std::fabs((long double)a[j] * b[j]);
      if (j == 0) A = ffacc_first(ff_from_d(a[j]), ff_from_d(b[j]));
      else ffacc_add(A, ff_from_d(a[j]), ff_from_d(b[j]));
      if ((j & 3) == 3) ffacc_norm(A);
    }
    const ff r = ffacc_result(A);
    const long double err = std::fabs(val(r) - ref);
    if (err > std::ldexp(mag, -43)) return fail("dot acc", a[0], (double)nt, err);
    if (std::fabs(r.lo) > std::fabs(r.hi) * std::ldexp(1.0, -23) + std::ldexp(mag, -70)) return fail("dot acc norm", a[0], nt, r.lo);
  }
  // 6. the stated conversion bounds, for both conversion pairs
  if (conversion_bounds(ff_from_d, ff_to_d, false, rng)) return 1;
  if (conversion_bounds(ff_from_d_fast, ff_to_d_fast, true, rng)) return 1;
  printf("ok\n");
  return 0;
}
