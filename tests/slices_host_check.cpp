// Host-side check of the bf16 digit slices that the tensor-core dense block
// uses (paper_0902_0699_gb300/csrc/slices.cuh compiled as plain C++):
//  1. the digits of a row: a0, a1 small integers, exact in bf16; |a2| <= 1/2;
//     the row rebuilt from (a0, a1, bf16(a2)) within 2^-18 of a unit of the
//     scaled row (2^-25 of its largest magnitude), with no bias;
//  2. the block's product formula (acc0 = sum a0 b0, acc1 = sum a0 b1 +
//     a1 b0, acc2 = sum a0 b2 + a2 b0 + a1 (2^-8 b1) + a1 (2^-8 b2) +
//     a2 (2^-8 b1), y = (acc0 + 2^-8 (acc1 + acc2)) * scales) in exact host
//     arithmetic against the long-double product of the unsliced values:
//     FP32-class accuracy against the output's scale, and a plausible slip
//     (a dropped cross term, a wrong scale) fails it;
//  3. acc0 and acc1 are integers below 2^24 (exact in FP32).
// Prints "ok" and exits 0, or prints the first failure and exits 1.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "../paper_0902_0699_gb300/csrc/slices.cuh"

using namespace qc;

static int fail(const char* what, double a, double b) {
  printf("FAIL %s: %.17g %.17g\n", what, a, b);
  return 1;
}

struct Digits {
  std::vector<float> d0, d1, d2;  // d2 already rounded to bf16
  uint32_t E;
};

static Digits slice_row(const std::vector<float>& x) {
  uint32_t mx = 0;
  for (float v : x) mx = std::max(mx, ff_fbits(v) & 0x7FFFFFFFu);
  Digits D;
  D.E = slice_exp(mx);
  const float sc = slice_scale(D.E);
  for (float v : x) {
    float a0, a1, a2;
    slice_digits(v, sc, a0, a1, a2);
    D.d0.push_back(bf16_value(bf16_bits_rn(a0)));
    D.d1.push_back(bf16_value(bf16_bits_rn(a1)));
    D.d2.push_back(bf16_value(bf16_bits_rn(a2)));
    if (D.d0.back() != a0 || D.d1.back() != a1) {
      printf("FAIL digit not exact in bf16: %.9g %.9g\n", a0, a1);
      exit(1);
    }
    if (a0 != std::nearbyint(a0) || a1 != std::nearbyint(a1) || std::fabs(a0) > 256.f || std::fabs(a1) > 128.f ||
        std::fabs(a2) > 0.5f) {
      printf("FAIL digit range: %.9g %.9g %.9g\n", a0, a1, a2);
      exit(1);
    }
  }
  return D;
}

int main() {
  std::mt19937_64 rng(2026);
  std::normal_distribution<float> N01(0.f, 1.f);
  std::uniform_int_distribution<int> X(-60, 2);
  // 1. digits of rows
  long double bias = 0.0L, bias2 = 0.0L;
  long count = 0;
  for (int it = 0; it < 20000; ++it) {
    std::vector<float> x(64);
    const int e = X(rng);
    for (auto& v : x) v = std::ldexp(N01(rng), e) * ((it % 7 == 0) ? std::ldexp(1.f, -(int)(rng() % 20)) : 1.f);
    if (it % 11 == 0) x[rng() % 64] = 0.f;
    const Digits D = slice_row(x);
    const double unit = std::ldexp(1.0, (int)D.E - 134);  // the scaled row's unit
    for (int i = 0; i < 64; ++i) {
      const long double rec = ((long double)D.d0[i] + ((long double)D.d1[i] + (long double)D.d2[i]) / 256.0L) * unit;
      const long double err = rec - (long double)x[i];
      if (std::fabs((double)err) > std::ldexp(unit, -18)) return fail("rebuilt row", x[i], (double)rec);
      bias += err / std::ldexp(unit, -18);
      bias2 += (err / std::ldexp(unit, -18)) * (err / std::ldexp(unit, -18));
      ++count;
    }
  }
  // the rounding of a2 to nearest: mean error within 4 standard errors of 0
  const double mean = (double)(bias / count), sd = std::sqrt((double)(bias2 / count));
  if (std::fabs(mean) > 4.0 * sd / std::sqrt((double)count)) return fail("digit rounding bias", mean, sd);
  // 2. + 3. the product formula on random rows against random operator rows
  double worst = 0.0, msq = 0.0;
  for (int it = 0; it < 2000; ++it) {
    // W: a row of K = 64 operator reals (entries of magnitude <= 1), x: a row
    std::vector<float> w(64), x(64);
    for (auto& v : w) v = std::tanh(N01(rng)) * 0.9f;
    const int e = X(rng);
    for (auto& v : x) v = std::ldexp(N01(rng), e);
    const Digits A = slice_row(x);
    const Digits Bw = slice_row(w);
    long double acc0 = 0, acc1 = 0, acc2 = 0, exact = 0, sum2 = 0;
    for (int k = 0; k < 64; ++k) {
      const long double a0 = A.d0[k], a1 = A.d1[k], a2 = A.d2[k];
      const long double b0 = Bw.d0[k], b1 = Bw.d1[k], b2 = Bw.d2[k];
      const long double b1s = bf16_value(bf16_bits_rn(Bw.d1[k] * 0.00390625f));
      const long double b2s = bf16_value(bf16_bits_rn(Bw.d2[k] * 0.00390625f));
      if (b1s != b1 / 256.0L || b2s != b2 / 256.0L) return fail("2^-8 digit not exact", (double)b1s, (double)b2s);
      acc0 += a0 * b0;
      acc1 += a0 * b1 + a1 * b0;
      acc2 += a0 * b2 + a2 * b0 + a1 * b1s + a1 * b2s + a2 * b1s;
      const long double t = (long double)x[k] * (long double)w[k];
      exact += t;
      sum2 += t * t;
    }
    if (std::fabs((double)acc0) >= 16777216.0 || std::fabs((double)acc1) >= 16777216.0 ||
        acc0 != std::nearbyint((double)acc0) || acc1 != std::nearbyint((double)acc1))
      return fail("acc0, acc1 exact integers below 2^24", (double)acc0, (double)acc1);
    const long double ys =
        (acc0 + (acc1 + acc2) / 256.0L) * std::ldexp(1.0L, (int)A.E - 134) * std::ldexp(1.0L, (int)Bw.E - 134);
    // FP32 class against the output's natural scale sqrt(sum of squared
    // terms): the digits keep about 25 bits of each row, so the error is a
    // few 2^-25 of that scale (rms over the draws below 2^-24.75, no draw
    // above 2^-22); dropping a 2^-16 cross term (a1 b2 or a2 b1) costs about
    // 2^-23 to 2^-22 on every draw and fails the rms bound
    const double ratio = std::fabs((double)(ys - exact)) / std::sqrt((double)sum2);
    worst = std::max(worst, ratio);
    msq += ratio * ratio;
    if (ratio > std::ldexp(1.0, -22)) return fail("product formula", (double)ys, (double)exact);
  }
  const double rms = std::sqrt(msq / 2000.0);
  if (std::getenv("SLICE_VERBOSE"))
    printf("error / rms scale: worst %.3g (2^%.2f), rms %.3g (2^%.2f)\n", worst, std::log2(worst), rms, std::log2(rms));
  if (rms > std::pow(2.0, -24.75)) return fail("product formula rms", rms, 0);
  printf("ok\n");
  return 0;
}
