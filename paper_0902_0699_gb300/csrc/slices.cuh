// Fixed-point bf16 digit slices for the tensor-core dense block (host and
// device).
//
// A row of reals (one group of 32 complex64 amplitudes) is scaled by a power
// of two taken from its largest magnitude, so that every scaled value y lies
// in (-256, 256), and written as three bf16 "digits"
//   y = a0 + 2^-8 (a1 + a2),   a0, a1 integers, |a0| <= 256, |a1| <= 128,
//   |a2| <= 1/2 (a2 rounded to bf16, 8 significant bits).
// a0 and a1 are small integers, exact in bf16, so products a0 * b0 of two
// such digits are integers below 2^16 and a sum of 64 of them is an exact
// integer below 2^22: the tensor cores' FP32 accumulation, which truncates
// what does not fit, has nothing to truncate there.  This is the splitting
// of Ozaki, Ogita, Oishi and Rump ("Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012) with bf16 digits.  The same
// digits serve the operator (per matrix instead of per row).
#pragma once

#include <stdint.h>

#include "ff.cuh"

namespace qc {

// 1.5 * 2^23: adding it to a float of magnitude below 2^22 rounds that float
// to an integer (round to nearest even), subtracting it again is exact.
#define QC_RINT_MAGIC 12582912.0f

// Scale 2^(134 - E) for a row whose largest magnitude has biased float
// exponent E (clamped to [8, 254] so that the scale is a normal float):
// |x| < 2^(E - 126) gives |x * scale| < 2^8.
FF_HD uint32_t slice_exp(uint32_t max_abs_bits) {
  uint32_t E = (max_abs_bits >> 23) & 0xFFu;
  if (E < 8u) E = 8u;
  if (E > 254u) E = 254u;
  return E;
}
FF_HD float slice_scale(uint32_t E) { return ff_bitsf((261u - E) << 23); }   // 2^(134 - E)
FF_HD float slice_unscale(uint32_t E) { return ff_bitsf((E - 7u) << 23); }  // 2^(E - 134)

// The three digits of y = x * scale.  Every step but the last rounding is
// exact: y + M rounds y to the integer a0, y - a0 and its product by 256 are
// exact, and so is r - a1.
FF_HD void slice_digits(float x, float scale, float& a0, float& a1, float& a2) {
  const float y = ff_mul_rn(x, scale);
  a0 = ff_sub_rn(ff_add_rn(y, QC_RINT_MAGIC), QC_RINT_MAGIC);
  const float r = ff_mul_rn(ff_sub_rn(y, a0), 256.f);
  a1 = ff_sub_rn(ff_add_rn(r, QC_RINT_MAGIC), QC_RINT_MAGIC);
  a2 = ff_sub_rn(r, a1);
}

// bf16 bit pattern of a finite float, rounded to nearest even (the device
// uses the hardware conversion, which rounds the same way).
FF_HD uint16_t bf16_bits_rn(float x) {
  const uint32_t b = ff_fbits(x);
  return (uint16_t)((b + 0x7FFFu + ((b >> 16) & 1u)) >> 16);
}
FF_HD float bf16_value(uint16_t h) { return ff_bitsf((uint32_t)h << 16); }

}  // namespace qc
