// Host-side check of the double-float layer the complex128 kernels use
// (paper_0902_0699_gb300/csrc/ff.cuh compiled as plain C++): conversions
// double <-> (hi, lo) and the ff arithmetic against long double references.
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
  printf("ok\n");
  return 0;
}
