// Reductions with FP64 accumulation: the amplitude sum (for Grover's mean),
// the norm sum |C|^2 (sec. 2), Born-rule probabilities, Pauli expectation
// values, and the seeded integer-CDF measurement sampler.
//
// Partial sums go to per-block slots in the state's scratch and are added
// in block order by one final block, so every result is deterministic for a
// given launch shape.  complex64 squares and products are formed exactly
// with the FP32 two-product (x*y = p + e, e = fma(x, y, -p)) and summed as
// float pairs (two-sum) over runs of 32 amplitudes before they are added in
// FP64: GB300 issues FP64 at about 1/70 of its FP32 rate, which would
// otherwise bound these passes well below memory bandwidth.
#include <algorithm>
#include <cmath>

#include <atomic>

#include "common.cuh"

namespace qc {

#define RED_T 256
#define RED_MAXB (QC_PARTIALS / 2)

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of two doubles; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      x += sa[i];
      y += sb[i];
    }
    a = x;
    b = y;
  }
  __syncthreads();
}

// Sum of the partial pairs written by `nb` blocks, in block order.
__global__ void k_final2(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

// float-float accumulator: (s, c) += (p, e) via two-sum.
__device__ __forceinline__ void ff_acc(float& s, float& c, float p, float e) {
  const float t = s + p;
  const float bp = t - s;
  const float err = (s - (t - bp)) + (p - bp);
  s = t;
  c += err + e;
}

// ------------------------------------------------ Born probabilities ----
// p_i = re*re + im*im, each product and the sum rounded on its own (the
// same operations as the FP64 reference; complex64 inputs are widened
// first, which makes the products exact).
//
// GB300 issues FP64 at about 1.6 operations per SM and clock.  For
// complex64 the exact square of a float (at most 48 significant bits) is
// assembled as a binary64 from the IEEE-754 fields with integer operations,
// so one FP64 add per amplitude remains; infinities and NaNs take the FP64
// formula.  complex128 squares need a rounded 106-bit product, which costs
// more in integer operations than the FP64 pipe takes for it.
template <typename R>
__device__ __forceinline__ double prob_fp64(typename CT<R>::V2 v) {
  const double re = (double)v.x, im = (double)v.y;
  return __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
}

// x*x as an exact binary64 for a finite float x: x = m 2^(f - 150) with the
// integer significand m < 2^24 (f = 1 for subnormals), x^2 = m^2 2^(2f - 300)
// with 1 <= L <= 48 significant bits; the biased exponent stays in
// [725, 1278], always normal.
__device__ __forceinline__ double sq_exact_f32(uint32_t b) {
  int f = (int)(b >> 23);
  uint32_t m = b & 0x7fffffu;
  if (f) m |= 0x800000u;
  else if (!m) return 0.0;
  else f = 1;
  const uint64_t q = (uint64_t)m * m;  // 32 x 32 -> 64 (a 64-bit multiply runs far slower)
  const int L = 64 - __clzll((long long)q);
  const uint64_t sig = q << (53 - L);
  const uint64_t E = (uint64_t)(2 * f - 300 - (53 - L) + 1075);
  return __longlong_as_double((long long)((E << 52) | (sig & 0xFFFFFFFFFFFFFull)));
}

template <typename R>
__device__ __forceinline__ double prob_of(typename CT<R>::V2 v);

template <>
__device__ __forceinline__ double prob_of<double>(double2 v) {
  return prob_fp64<double>(v);
}

// a call, so that the compiler cannot if-convert the FP64 formula into the
// common path (every amplitude would then pay for it)
__device__ __noinline__ double prob_nonfinite_f32(float2 v) { return prob_fp64<float>(v); }

template <>
__device__ __forceinline__ double prob_of<float>(float2 v) {
  const uint32_t a = __float_as_uint(v.x) & 0x7fffffffu, b = __float_as_uint(v.y) & 0x7fffffffu;
  if (a >= 0x7f800000u || b >= 0x7f800000u) return prob_nonfinite_f32(v);  // inf or NaN
  return __dadd_rn(sq_exact_f32(a), sq_exact_f32(b));
}

// ---------------------------------------------------------------- sum ----
__global__ void __launch_bounds__(RED_T) k_sum_c128(const double2* __restrict__ s, uint64_t N,
                                                    double* __restrict__ part) {
  double a = 0.0, b = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) {
    const double2 v = s[i];
    a += v.x;
    b += v.y;
  }
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// complex64: float-pair runs of RUN vectors (2 RUN amplitudes, every
// rounding error kept by the two-sum), FP64 across runs; the FP64 pipe sees
// four operations per run instead of four per amplitude.
#define RUN 16
__global__ void __launch_bounds__(RED_T) k_sum_c64(const float4* __restrict__ s, uint64_t N2,
                                                   double* __restrict__ part) {
  double a = 0.0, b = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  while (i < N2) {
    float as = 0.f, ac = 0.f, bs = 0.f, bc = 0.f;
#pragma unroll 4
    for (int r = 0; r < RUN; ++r, i += G) {
      if (i < N2) {
        const float4 v = s[i];
        ff_acc(as, ac, v.x, 0.f);
        ff_acc(as, ac, v.z, 0.f);
        ff_acc(bs, bc, v.y, 0.f);
        ff_acc(bs, bc, v.w, 0.f);
      }
    }
    a += (double)as + (double)ac;
    b += (double)bs + (double)bc;
  }
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

qc_status launch_sum(qc_state* s) {
  const uint64_t N = 1ull << s->n;
  double* part = s->scratch + QC_SCR_PARTIALS;
  unsigned nb;
  if (s->dt == QC_C128) {
    nb = std::min<unsigned>(grid_for(N, RED_T * 4, 8), RED_MAXB);
    k_sum_c128<<<nb, RED_T, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), N, part);
  } else {  // n >= 1: N / 2 >= 1 vectors of two amplitudes
    nb = std::min<unsigned>(grid_for(N / 2, RED_T * 4, 8), RED_MAXB);
    k_sum_c64<<<nb, RED_T, 0, s->stream>>>(reinterpret_cast<const float4*>(s->data), N / 2, part);
  }
  k_final2<<<1, RED_T, 0, s->stream>>>(part, nb, s->scratch + QC_SCR_SUM);
  qc_status st = check_launch("amplitude sum", 2);
  if (!st) s->sum_valid = true;
  return st;
}

// --------------------------------------------------------------- norm ----
__global__ void __launch_bounds__(RED_T) k_norm_c128(const double2* __restrict__ s, uint64_t N,
                                                     double* __restrict__ part) {
  double a = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) {
    const double2 v = s[i];
    a = fma(v.x, v.x, a);
    a = fma(v.y, v.y, a);
  }
  double b = 0.0;
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

// complex64: exact FP32 squares, float-pair runs of RUN vectors, FP64
// across runs.
__global__ void __launch_bounds__(RED_T) k_norm_c64(const float4* __restrict__ s, uint64_t N2,
                                                    double* __restrict__ part) {
  double acc = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  while (i < N2) {
    float hs = 0.f, hc = 0.f;
#pragma unroll 4
    for (int r = 0; r < RUN; ++r, i += G) {
      if (i < N2) {
        const float4 v = s[i];
        const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float p = x[k] * x[k];
          ff_acc(hs, hc, p, fmaf(x[k], x[k], -p));
        }
      }
    }
    acc += (double)hs + (double)hc;
  }
  double b = 0.0;
  block_sum2(acc, b);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = acc;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

qc_status reduce_norm(const qc_state* s, double* out_host) {
  const uint64_t N = 1ull << s->n;
  double* part = s->scratch + QC_SCR_PARTIALS;
  unsigned nb;
  if (s->dt == QC_C128) {
    nb = std::min<unsigned>(grid_for(N, RED_T * 4, 8), RED_MAXB);
    k_norm_c128<<<nb, RED_T, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), N, part);
  } else {  // n >= 1, so N / 2 >= 1 vectors of two amplitudes
    nb = std::min<unsigned>(grid_for(N / 2, RED_T * 4, 8), RED_MAXB);
    k_norm_c64<<<nb, RED_T, 0, s->stream>>>(reinterpret_cast<const float4*>(s->data), N / 2, part);
  }
  k_final2<<<1, RED_T, 0, s->stream>>>(part, nb, s->scratch + QC_SCR_MISC);
  qc_status st = check_launch("norm", 2);
  if (st) return st;
  double h[2];
  cudaError_t e = cudaMemcpyAsync(h, s->scratch + QC_SCR_MISC, sizeof h, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "norm readback");
  *out_host = h[0];
  return QC_OK;
}

// -------------------------------------------------------------- probs ----
template <typename R>
__global__ void __launch_bounds__(RED_T) k_probs(const typename CT<R>::V2* __restrict__ s, uint64_t N,
                                                 double* __restrict__ p) {
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) p[i] = prob_of<R>(s[i]);
}

qc_status launch_probs(const qc_state* s, double* out) {
  const uint64_t N = 1ull << s->n;
  if (s->dt == QC_C128)
    k_probs<double><<<grid_for(N, RED_T, 8), RED_T, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), N, out);
  else
    k_probs<float><<<grid_for(N, RED_T, 8), RED_T, 0, s->stream>>>(reinterpret_cast<const float2*>(s->data), N, out);
  return check_launch("probs");
}

// ------------------------------------------------------------- expect ----
// <psi|P|psi> = i^{|x&z|} h,  h = sum_j conj(C[j^x]) (-1)^{|j&z|} C[j].
//
// x = 0: h = sum_j (-1)^{|j&z|} |C_j|^2 (real).  x != 0: with b the lowest
// set bit of x, the terms of j0 (bit b clear) and j1 = j0 ^ x add up to
// (-1)^{|j0&z|} (u + sigma conj(u)), u = conj(C[j1]) C[j0], sigma =
// (-1)^{|x&z|}: 2 Re u when sigma = 1, 2i Im u when sigma = -1.  So every
// amplitude is read once and a pair costs two real products.

// sign bit of (-1)^{|j&z|} as a 64-bit mask
__device__ __forceinline__ uint64_t parity_sign(uint64_t j, uint64_t z) {
  return (uint64_t)(__popcll(j & z) & 1) << 63;
}

__device__ __forceinline__ double flip(double v, uint64_t sg) {
  return __longlong_as_double((long long)((uint64_t)__double_as_longlong(v) ^ sg));
}

__device__ __forceinline__ float flipf(float v, uint64_t sg) {
  return __uint_as_float(__float_as_uint(v) ^ (uint32_t)(sg >> 32));
}

// complex128, x = 0: signed |C_j|^2
__global__ void __launch_bounds__(RED_T) k_expect_diag_c128(const double2* __restrict__ s, uint64_t N, uint64_t z,
                                                            double* __restrict__ part) {
  double a = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += G) {
    const double2 v = s[j];
    const uint64_t sg = parity_sign(j, z);
    a = fma(flip(v.x, sg), v.x, a);
    a = fma(flip(v.y, sg), v.y, a);
  }
  double b = 0.0;
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

// complex64, x = 0: exact FP32 squares, signed, float-pair runs
__global__ void __launch_bounds__(RED_T) k_expect_diag_c64(const float4* __restrict__ s, uint64_t N2, uint64_t z,
                                                           double* __restrict__ part) {
  double acc = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t z0 = (z & 1ull) << 63;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  while (i < N2) {
    float hs = 0.f, hc = 0.f;
#pragma unroll 4
    for (int r = 0; r < RUN; ++r, i += G) {
      if (i < N2) {
        const float4 v = s[i];
        const uint64_t s0 = parity_sign(2 * i, z), s1 = s0 ^ z0;
        const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t sg = k < 2 ? s0 : s1;
          const float p = x[k] * x[k];
          ff_acc(hs, hc, flipf(p, sg), flipf(fmaf(x[k], x[k], -p), sg));
        }
      }
    }
    acc += (double)hs + (double)hc;
  }
  double b = 0.0;
  block_sum2(acc, b);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = acc;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

// complex128, x != 0: sum over pairs of (-1)^{|j0&z|} Re u (IM = false) or
// Im u (IM = true), u = conj(w) v, v = C[j0], w = C[j0 ^ x]
template <bool IM>
__global__ void __launch_bounds__(RED_T) k_expect_pair_c128(const double2* __restrict__ s, uint64_t NP, int b,
                                                            uint64_t x, uint64_t z, double* __restrict__ part) {
  double a = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
#pragma unroll 4
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += G) {
    const uint64_t j0 = insert0(p, b);
    const double2 v = s[j0], w = s[j0 ^ x];
    const uint64_t sg = parity_sign(j0, z);
    // Re u = wr vr + wi vi;  Im u = wr vi - wi vr
    const double c0 = flip(w.x, sg), c1 = flip(IM ? -w.y : w.y, sg);
    a = fma(c0, IM ? v.y : v.x, a);
    a = fma(c1, IM ? v.x : v.y, a);
  }
  double b2 = 0.0;
  block_sum2(a, b2);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

// complex64, x != 0: the two products exactly as float pairs
// (two-product), float-pair runs, FP64 across runs
template <bool IM>
__global__ void __launch_bounds__(RED_T) k_expect_pair_c64(const float2* __restrict__ s, uint64_t NP, int b,
                                                           uint64_t x, uint64_t z, double* __restrict__ part) {
  double acc = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  while (p < NP) {
    float hs = 0.f, hc = 0.f;
#pragma unroll 4
    for (int r = 0; r < 2 * RUN; ++r, p += G) {
      if (p < NP) {
        const uint64_t j0 = insert0(p, b);
        const float2 v = s[j0], w = s[j0 ^ x];
        const uint64_t sg = parity_sign(j0, z);
        const float c0 = flipf(w.x, sg), c1 = flipf(IM ? -w.y : w.y, sg);
        const float d0 = IM ? v.y : v.x, d1 = IM ? v.x : v.y;
        float q = c0 * d0;
        ff_acc(hs, hc, q, fmaf(c0, d0, -q));
        q = c1 * d1;
        ff_acc(hs, hc, q, fmaf(c1, d1, -q));
      }
    }
    acc += (double)hs + (double)hc;
  }
  double b2 = 0.0;
  block_sum2(acc, b2);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = acc;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

qc_status reduce_expect(const qc_state* s, uint64_t x, uint64_t z, double* out_host) {
  const uint64_t N = 1ull << s->n;
  double* part = s->scratch + QC_SCR_PARTIALS;
  const bool c128 = (s->dt == QC_C128);
  const bool im = x && (__builtin_popcountll(x & z) & 1);  // sigma = -1
  unsigned nb;
  if (!x) {
    if (c128) {
      nb = std::min<unsigned>(grid_for(N, RED_T * 4, 8), RED_MAXB);
      k_expect_diag_c128<<<nb, RED_T, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), N, z, part);
    } else {  // n >= 1: N / 2 >= 1 vectors of two amplitudes
      nb = std::min<unsigned>(grid_for(N / 2, RED_T * 4, 8), RED_MAXB);
      k_expect_diag_c64<<<nb, RED_T, 0, s->stream>>>(reinterpret_cast<const float4*>(s->data), N / 2, z, part);
    }
  } else {
    const int b = __builtin_ctzll(x);
    nb = std::min<unsigned>(grid_for(N / 2, RED_T * 4, 8), RED_MAXB);
    const double2* d2 = reinterpret_cast<const double2*>(s->data);
    const float2* f2 = reinterpret_cast<const float2*>(s->data);
    if (c128 && im) k_expect_pair_c128<true><<<nb, RED_T, 0, s->stream>>>(d2, N / 2, b, x, z, part);
    else if (c128) k_expect_pair_c128<false><<<nb, RED_T, 0, s->stream>>>(d2, N / 2, b, x, z, part);
    else if (im) k_expect_pair_c64<true><<<nb, RED_T, 0, s->stream>>>(f2, N / 2, b, x, z, part);
    else k_expect_pair_c64<false><<<nb, RED_T, 0, s->stream>>>(f2, N / 2, b, x, z, part);
  }
  k_final2<<<1, RED_T, 0, s->stream>>>(part, nb, s->scratch + QC_SCR_MISC);
  qc_status st = check_launch("expect", 2);
  if (st) return st;
  double h[2];
  cudaError_t e = cudaMemcpyAsync(h, s->scratch + QC_SCR_MISC, sizeof h, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "expect readback");
  // h from the pair sums (times 2: both members of each pair), then i^{|x&z|}
  const double r = !x ? h[0] : (im ? 0.0 : 2.0 * h[0]);
  const double i = !x ? 0.0 : (im ? 2.0 * h[0] : 0.0);
  const int ny = __builtin_popcountll(x & z) & 3;
  const double rr[4] = {r, -i, -r, i}, ii[4] = {i, r, -i, -r};
  out_host[0] = rr[ny];
  out_host[1] = ii[ny];
  return QC_OK;
}

// ------------------------------------------------------------ sampler ----
// w_i = trunc(p_i * 2^62); W = inclusive prefix sum (exact integers, so the
// parallel order does not matter); shot s: target = floor(r * W_{N-1} /
// 2^64), outcome = smallest i with W_i > target.
//
// Only the per-block weight sums (one per SMP_BLOCK amplitudes) are scanned
// over the whole state.  With few shots, each shot finds its block by
// bisection over the block offsets and rescans that block's weights; with
// many shots the full CDF is written once and bisected per shot.
#define SMP_PER 8
#define SMP_T 256
#define SMP_BLOCK (SMP_PER * SMP_T)
#define SMP_BAD_P 1ull     // some p_i outside [0, 2] or NaN
#define SMP_OVERFLOW 2ull  // a weight sum above 2^64 - 1

// a + b, saturated at 2^64 - 1 (associative, so any summation order
// saturates exactly when the true sum does not fit)
__device__ __forceinline__ uint64_t sat_add(uint64_t a, uint64_t b) {
  const uint64_t s = a + b;
  return s < a ? ~0ull : s;
}

// trunc(p * 2^62) for 0 <= p <= 2 from the IEEE-754 fields, with integer
// operations only: p = m * 2^(e - 1075) with the 53-bit significand m, so
// p * 2^62 = m * 2^(e - 1013).  Sets *bad (and returns 0) for p outside
// [0, 2] or NaN, i.e. for a bit pattern above that of 2.0 (unsigned).
__device__ __forceinline__ uint64_t weight_of_p(double p, bool* bad) {
  const uint64_t b = (uint64_t)__double_as_longlong(p);
  if (b > 0x4000000000000000ull) {
    *bad = true;
    return 0;
  }
  const int e = (int)(b >> 52);
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  const int sh = e - 1013;
  if (sh >= 0) return m << sh;  // sh <= 11: m << sh <= 2^63
  return sh <= -64 ? 0ull : m >> (-sh);
}

template <typename R>
__device__ __forceinline__ uint64_t weight_of(typename CT<R>::V2 v, bool* bad) {
  return weight_of_p(prob_of<R>(v), bad);
}

// Exclusive block scan with saturating sums; *total (if given) receives the
// block total.  Exact whenever the block total fits in 64 bits.
__device__ __forceinline__ uint64_t block_excl_scan_u64(uint64_t v, uint64_t* total) {
  __shared__ uint64_t ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = sat_add(x, y);
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    uint64_t t = lane < nw ? ws[lane] : 0ull;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t = sat_add(t, y);
    }
    ws[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const uint64_t warp_off = w ? ws[w - 1] : 0ull;
  if (total) *total = ws[(blockDim.x >> 5) - 1];
  const uint64_t r = warp_off + x - v;
  __syncthreads();
  return r;
}

// Weights of the SMP_PER consecutive elements thread `t` owns in block b.
template <typename R>
__device__ __forceinline__ uint64_t thread_weights(const typename CT<R>::V2* __restrict__ s, uint64_t N, uint64_t b,
                                                   int t, uint64_t w[SMP_PER], bool* bad) {
  const uint64_t base = b * SMP_BLOCK + (uint64_t)t * SMP_PER;
  uint64_t sum = 0;
#pragma unroll
  for (int k = 0; k < SMP_PER; ++k) {
    const uint64_t i = base + k;
    w[k] = i < N ? weight_of<R>(s[i], bad) : 0ull;
    sum = sat_add(sum, w[k]);
  }
  return sum;
}

// Block b's weight sum from each thread's partial sum t, into bsum[b];
// status bit SMP_BAD_P if any thread saw an unusable probability.
__device__ __forceinline__ void block_wsum_out(uint64_t t, bool bad, uint64_t* __restrict__ bsum,
                                               uint64_t* __restrict__ status) {
  __shared__ uint64_t ws[SMP_T / 32];
  for (int o = 16; o > 0; o >>= 1) t = sat_add(t, __shfl_xor_sync(0xffffffffu, t, o));
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr((unsigned long long*)status, SMP_BAD_P);
  if (threadIdx.x == 0) {
    uint64_t a = 0;
    for (int w = 0; w < SMP_T / 32; ++w) a = sat_add(a, ws[w]);
    bsum[blockIdx.x] = a;
  }
}

// Per-block weight sums (coalesced: the saturating sum does not depend on
// which thread adds which weight); status bits for unusable probabilities.
template <typename R>
__global__ void __launch_bounds__(SMP_T) k_wsum(const typename CT<R>::V2* __restrict__ s, uint64_t N,
                                                uint64_t* __restrict__ bsum, uint64_t* __restrict__ status) {
  const uint64_t base = (uint64_t)blockIdx.x * SMP_BLOCK;
  bool bad = false;
  uint64_t t = 0;
#pragma unroll
  for (int k = 0; k < SMP_PER; ++k) {
    const uint64_t i = base + (uint64_t)k * SMP_T + threadIdx.x;
    if (i < N) t = sat_add(t, weight_of<R>(s[i], &bad));
  }
  block_wsum_out(t, bad, bsum, status);
}

// The same block sums, and the probabilities p_i written out, from one read
// of the state (the Born probability is computed once and used for both).
template <typename R>
__global__ void __launch_bounds__(SMP_T) k_probs_wsum(const typename CT<R>::V2* __restrict__ s, uint64_t N,
                                                      double* __restrict__ p, uint64_t* __restrict__ bsum,
                                                      uint64_t* __restrict__ status) {
  const uint64_t base = (uint64_t)blockIdx.x * SMP_BLOCK;
  bool bad = false;
  uint64_t t = 0;
#pragma unroll
  for (int k = 0; k < SMP_PER; ++k) {
    const uint64_t i = base + (uint64_t)k * SMP_T + threadIdx.x;
    if (i < N) {
      const double pi = prob_of<R>(s[i]);
      p[i] = pi;
      t = sat_add(t, weight_of_p(pi, &bad));
    }
  }
  block_wsum_out(t, bad, bsum, status);
}

static void launch_wsum(qc_dtype dt, const void* psi, uint64_t N, uint64_t* bsum, uint64_t* status,
                        cudaStream_t st, double* probs = nullptr) {
  const unsigned nb = (unsigned)((N + SMP_BLOCK - 1) / SMP_BLOCK);
  if (probs) {
    if (dt == QC_C128)
      k_probs_wsum<double><<<nb, SMP_T, 0, st>>>(reinterpret_cast<const double2*>(psi), N, probs, bsum, status);
    else
      k_probs_wsum<float><<<nb, SMP_T, 0, st>>>(reinterpret_cast<const float2*>(psi), N, probs, bsum, status);
    return;
  }
  if (dt == QC_C128)
    k_wsum<double><<<nb, SMP_T, 0, st>>>(reinterpret_cast<const double2*>(psi), N, bsum, status);
  else
    k_wsum<float><<<nb, SMP_T, 0, st>>>(reinterpret_cast<const float2*>(psi), N, bsum, status);
}

// Exclusive scan of the block sums in place (one block); tail[0] receives
// the total and status gets SMP_OVERFLOW if it does not fit in 64 bits.
__global__ void __launch_bounds__(1024) k_scan_bsum(uint64_t* __restrict__ bsum, uint64_t nb,
                                                    uint64_t* __restrict__ tail, uint64_t* __restrict__ status) {
  const uint64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const uint64_t lo = (uint64_t)threadIdx.x * per;
  uint64_t t = 0;
  for (uint64_t i = lo; i < lo + per && i < nb; ++i) t = sat_add(t, bsum[i]);
  uint64_t total = 0;
  uint64_t off = block_excl_scan_u64(t, &total);
  for (uint64_t i = lo; i < lo + per && i < nb; ++i) {
    const uint64_t v = bsum[i];
    bsum[i] = off;
    off += v;
  }
  if (threadIdx.x == 0) {
    if (tail) tail[0] = total;
    if (total == ~0ull) atomicOr((unsigned long long*)status, SMP_OVERFLOW);
  }
}

// Large block counts: chunks of SCAN_CHUNK block sums; one CTA per chunk
// sums it (coalesced), the chunk totals take k_scan_bsum, and one CTA per
// chunk then rewrites its block sums as exclusive offsets.
#define SCAN_T 256
#define SCAN_PER 16
#define SCAN_CHUNK (SCAN_T * SCAN_PER)

__global__ void __launch_bounds__(SCAN_T) k_chunk_sum(const uint64_t* __restrict__ bsum, uint64_t nb,
                                                      uint64_t* __restrict__ csum) {
  const uint64_t base = (uint64_t)blockIdx.x * SCAN_CHUNK;
  uint64_t t = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    const uint64_t i = base + (uint64_t)k * SCAN_T + threadIdx.x;
    if (i < nb) t = sat_add(t, bsum[i]);
  }
  uint64_t tot = 0;
  block_excl_scan_u64(t, &tot);
  if (threadIdx.x == 0) csum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T) k_chunk_scan(uint64_t* __restrict__ bsum, uint64_t nb,
                                                       const uint64_t* __restrict__ coff) {
  const uint64_t base = (uint64_t)blockIdx.x * SCAN_CHUNK + (uint64_t)threadIdx.x * SCAN_PER;
  uint64_t v[SCAN_PER];
  uint64_t t = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    v[k] = base + k < nb ? bsum[base + k] : 0ull;
    t = sat_add(t, v[k]);
  }
  uint64_t run = coff[blockIdx.x] + block_excl_scan_u64(t, nullptr);
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    if (base + k < nb) bsum[base + k] = run;
    run += v[k];
  }
}

// Exclusive offsets of the nb block sums in place, total in tail[0],
// SMP_OVERFLOW in *status if the total does not fit; csum holds
// ceil(nb / SCAN_CHUNK) words (unused when nb <= SCAN_CHUNK).
static void scan_block_sums(uint64_t* bsum, uint64_t nb, uint64_t* csum, uint64_t* tail, uint64_t* status,
                            cudaStream_t st) {
  if (nb <= SCAN_CHUNK) {
    k_scan_bsum<<<1, 1024, 0, st>>>(bsum, nb, tail, status);
    return;
  }
  const uint64_t nc = (nb + SCAN_CHUNK - 1) / SCAN_CHUNK;
  k_chunk_sum<<<(unsigned)nc, SCAN_T, 0, st>>>(bsum, nb, csum);
  k_scan_bsum<<<1, 1024, 0, st>>>(csum, nc, tail, status);
  k_chunk_scan<<<(unsigned)nc, SCAN_T, 0, st>>>(bsum, nb, csum);
}

static uint64_t scan_words(uint64_t nb) { return nb <= SCAN_CHUNK ? 0 : (nb + SCAN_CHUNK - 1) / SCAN_CHUNK; }

template <typename R>
__global__ void __launch_bounds__(SMP_T) k_wcdf(const typename CT<R>::V2* __restrict__ s, uint64_t N,
                                                const uint64_t* __restrict__ boff, uint64_t* __restrict__ cdf) {
  uint64_t w[SMP_PER];
  bool bad = false;
  const uint64_t t = thread_weights<R>(s, N, blockIdx.x, threadIdx.x, w, &bad);
  uint64_t run = boff[blockIdx.x] + block_excl_scan_u64(t, nullptr);
  const uint64_t base = (uint64_t)blockIdx.x * SMP_BLOCK + (uint64_t)threadIdx.x * SMP_PER;
#pragma unroll
  for (int k = 0; k < SMP_PER; ++k) {
    run += w[k];
    if (base + k < N) cdf[base + k] = run;
  }
}

__device__ __forceinline__ uint64_t shot_target(int64_t sh, uint64_t seed, uint64_t total) {
  uint32_t x[4];
  philox4x32_10((uint32_t)(uint64_t)sh, (uint32_t)((uint64_t)sh >> 32), 0u, 0u, (uint32_t)seed,
                (uint32_t)(seed >> 32), x);
  const uint64_t r = ((uint64_t)x[0] << 32) | x[1];
  return __umul64hi(r, total);
}

// Many shots: bisection of the full CDF.
__global__ void k_sample(const uint64_t* __restrict__ cdf, uint64_t N, uint64_t seed, int64_t shots,
                         uint64_t* __restrict__ out) {
  const uint64_t total = cdf[N - 1];
  for (int64_t sh = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sh < shots;
       sh += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t target = shot_target(sh, seed, total);
    uint64_t lo = 0, hi = N - 1;  // answer in [lo, hi]; cdf[N-1] = total > target
    while (lo < hi) {
      const uint64_t mid = lo + ((hi - lo) >> 1);
      if (cdf[mid] > target) hi = mid;
      else lo = mid + 1;
    }
    out[sh] = lo;
  }
}

// Few shots: one CTA per shot finds the block holding the target (the last
// block whose exclusive offset is <= target) and rescans its weights.
template <typename R>
__global__ void __launch_bounds__(SMP_T) k_sample_local(const typename CT<R>::V2* __restrict__ s, uint64_t N,
                                                        const uint64_t* __restrict__ boff, uint64_t nb,
                                                        const uint64_t* __restrict__ tail, uint64_t seed,
                                                        int64_t shots, uint64_t* __restrict__ out) {
  const uint64_t total = tail[0];
  for (int64_t sh = blockIdx.x; sh < shots; sh += gridDim.x) {
    const uint64_t target = shot_target(sh, seed, total);
    uint64_t lo = 0, hi = nb - 1;  // boff[0] = 0 <= target
    while (lo < hi) {
      const uint64_t mid = hi - ((hi - lo) >> 1);
      if (boff[mid] <= target) lo = mid;
      else hi = mid - 1;
    }
    uint64_t w[SMP_PER];
    bool bad = false;
    const uint64_t t = thread_weights<R>(s, N, lo, threadIdx.x, w, &bad);
    uint64_t run = boff[lo] + block_excl_scan_u64(t, nullptr);
    const uint64_t base = lo * SMP_BLOCK + (uint64_t)threadIdx.x * SMP_PER;
    if (run <= target && target < run + t) {
#pragma unroll
      for (int k = 0; k < SMP_PER; ++k) {
        const uint64_t prev = run;
        run += w[k];
        if (prev <= target && target < run) out[sh] = base + k;
      }
    }
  }
}

qc_status launch_sample(const qc_state* s, uint64_t seed, int64_t shots, uint64_t* out, double* probs) {
  const uint64_t N = 1ull << s->n;
  const uint64_t nb = (N + SMP_BLOCK - 1) / SMP_BLOCK;
  const bool local = (uint64_t)shots <= nb;
  // [cdf (many shots only)] [block offsets nb] [total] [status] [chunk sums]
  const uint64_t words = (local ? 0 : N) + nb + 2 + scan_words(nb);
  uint64_t* buf = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&buf, words * sizeof(uint64_t), s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sampler buffer");
  uint64_t* cdf = buf;
  uint64_t* bsum = buf + (local ? 0 : N);
  uint64_t* tail = bsum + nb;
  uint64_t* status = tail + 1;
  uint64_t* csum = status + 1;
  e = cudaMemsetAsync(status, 0, sizeof(uint64_t), s->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(buf, s->stream);
    return cuda_fail(e, "sampler status reset");
  }
  launch_wsum(s->dt, s->data, N, bsum, status, s->stream, probs);
  scan_block_sums(bsum, nb, csum, tail, status, s->stream);
  qc_status st = check_launch("sample weights", nb <= SCAN_CHUNK ? 2 : 4);
  uint64_t h[2] = {0, 0};
  if (!st) {
    e = cudaMemcpyAsync(h, tail, sizeof h, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "sampler total readback");
  }
  if (!st && (h[1] || h[0] == 0 || h[0] > (1ull << 63))) {
    set_error("sampling needs every |C_i|^2 in [0, 2] and 0 < sum trunc(|C_i|^2 2^62) <= 2^63 "
              "(status %llu, total %llu)", (unsigned long long)h[1], (unsigned long long)h[0]);
    st = QC_EINVAL;
  }
  if (!st) {
    if (local) {
      const unsigned g = (unsigned)std::min<int64_t>(shots, (int64_t)sm_count() * 8);
      if (s->dt == QC_C128)
        k_sample_local<double><<<g, SMP_T, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), N, bsum, nb,
                                                           tail, seed, shots, out);
      else
        k_sample_local<float><<<g, SMP_T, 0, s->stream>>>(reinterpret_cast<const float2*>(s->data), N, bsum, nb,
                                                          tail, seed, shots, out);
      st = check_launch("sample", 1);
    } else {
      if (s->dt == QC_C128)
        k_wcdf<double><<<(unsigned)nb, SMP_T, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), N, bsum, cdf);
      else
        k_wcdf<float><<<(unsigned)nb, SMP_T, 0, s->stream>>>(reinterpret_cast<const float2*>(s->data), N, bsum, cdf);
      const unsigned g = (unsigned)std::min<int64_t>((shots + 255) / 256, (int64_t)sm_count() * 8);
      k_sample<<<g, 256, 0, s->stream>>>(cdf, N, seed, shots, out);
      st = check_launch("sample", 2);
    }
  }
  cudaFreeAsync(buf, s->stream);
  return st;
}

// ------------------------------------------- sampler without allocation --
// Scratch for qc_sample_noalloc, resident on every device that loads this
// library until the process exits: the integer CDF of up to 2^20
// amplitudes, the per-block weight sums and a status word.
#define NA_MAX_N QC_SAMPLE_NOALLOC_MAX_QUBITS
#define NA_CDF (1ull << NA_MAX_N)
#define NA_BSUM ((NA_CDF + SMP_BLOCK - 1) / SMP_BLOCK)
static __device__ __align__(256) uint64_t g_noalloc_scratch[NA_CDF + NA_BSUM + 32];

// Device address of the scratch per device (host code only sees a host-side
// stand-in for the symbol, so the address is looked up once per device).
// Atomic slots: first calls from several host threads may race to fill one;
// they store the same value.
static std::atomic<uint64_t*> g_noalloc_ptr[64];

// Status bits: 1 = some p_i outside [0, 2] (or NaN, from k_wsum), 2 = total
// weight zero or above 2^63.
__global__ void k_noalloc_total(const uint64_t* __restrict__ cdf, uint64_t N, uint64_t* __restrict__ status) {
  const uint64_t total = cdf[N - 1];
  if (total == 0 || total > (1ull << 63)) atomicOr((unsigned long long*)status, 2ull);
}

}  // namespace qc

using namespace qc;

QC_API qc_status qc_sample_noalloc(const void* psi_dev, int n, qc_dtype dt, uint64_t seed, int64_t shots,
                                   uint64_t* out_dev, void* stream) {
  clear_error();
  if (n < 1 || n > NA_MAX_N) {
    set_error("qc_sample_noalloc: n = %d out of range [1, %d] (its fixed scratch holds 2^%d amplitudes)", n,
              NA_MAX_N, NA_MAX_N);
    return QC_EINVAL;
  }
  if (dt != QC_C128 && dt != QC_C64) {
    set_error("unknown dtype %d", (int)dt);
    return QC_EINVAL;
  }
  if (!psi_dev || shots < 0 || (shots > 0 && !out_dev)) {
    set_error("qc_sample_noalloc: NULL state, negative shots or NULL output");
    return QC_EINVAL;
  }
  if (shots == 0) return QC_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "qc_sample_noalloc: device");
  if (dev < 0 || dev >= 64) {
    set_error("qc_sample_noalloc: device ordinal %d not supported", dev);
    return QC_EINVAL;
  }
  uint64_t* cdf = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!cdf) {  // first call on this device: look up the scratch address
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "qc_sample_noalloc: scratch address");
    cdf = reinterpret_cast<uint64_t*>(ptr);
    g_noalloc_ptr[dev].store(cdf, std::memory_order_release);
  }
  uint64_t* bsum = cdf + NA_CDF;
  uint64_t* status = bsum + NA_BSUM;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t N = 1ull << n;
  const uint64_t nb = (N + SMP_BLOCK - 1) / SMP_BLOCK;
  e = cudaMemsetAsync(status, 0, sizeof(uint64_t), st);  // the previous call's status is stale
  if (e != cudaSuccess) return cuda_fail(e, "qc_sample_noalloc: status reset");
  launch_wsum(dt, psi_dev, N, bsum, status, st);
  k_scan_bsum<<<1, 1024, 0, st>>>(bsum, nb, nullptr, status);
  if (dt == QC_C128)
    k_wcdf<double><<<(unsigned)nb, SMP_T, 0, st>>>(reinterpret_cast<const double2*>(psi_dev), N, bsum, cdf);
  else
    k_wcdf<float><<<(unsigned)nb, SMP_T, 0, st>>>(reinterpret_cast<const float2*>(psi_dev), N, bsum, cdf);
  k_noalloc_total<<<1, 1, 0, st>>>(cdf, N, status);
  qc_status rs = check_launch("qc_sample_noalloc: cdf", 4);
  if (rs) return rs;
  uint64_t hstat = 0;
  e = cudaMemcpyAsync(&hstat, status, sizeof hstat, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "qc_sample_noalloc: status readback");
  if (hstat) {
    set_error("qc_sample_noalloc: probabilities unusable (status %llu: need every |C_i|^2 in [0, 2] and "
              "0 < sum trunc(p_i 2^62) <= 2^63)", (unsigned long long)hstat);
    return QC_EINVAL;
  }
  const unsigned g = (unsigned)std::min<int64_t>((shots + 255) / 256, (int64_t)sm_count() * 8);
  k_sample<<<g, 256, 0, st>>>(cdf, N, seed, shots, out_dev);
  return check_launch("qc_sample_noalloc: sample", 1);
}
