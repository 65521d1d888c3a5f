// Reductions with FP64 accumulation: the amplitude sum (for Grover's mean),
// the norm sum |C|^2 (sec. 2), Born-rule probabilities, Pauli expectation
// values, and the seeded integer-CDF measurement sampler.
//
// Partial sums go to per-block slots in the state's scratch and are added
// in block order by one final block, so every result is deterministic for a
// given launch shape.  complex64 squares are formed exactly with the FP32
// two-product (x*x = p + e, e = fma(x, x, -p)) and accumulated as float
// pairs over short runs before they are added in FP64.
#include <algorithm>
#include <cmath>

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

// ---------------------------------------------------------------- sum ----
template <typename R>
__global__ void __launch_bounds__(RED_T) k_sum(const typename CT<R>::V2* __restrict__ s, uint64_t N,
                                               double* __restrict__ part) {
  double a = 0.0, b = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) {
    const auto v = s[i];
    a += (double)v.x;
    b += (double)v.y;
  }
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

qc_status launch_sum(qc_state* s) {
  const uint64_t N = 1ull << s->n;
  const unsigned nb = std::min<unsigned>(grid_for(N, RED_T * 4, 8), RED_MAXB);
  double* part = s->scratch + QC_SCR_PARTIALS;
  if (s->dt == QC_C128)
    k_sum<double><<<nb, RED_T, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), N, part);
  else
    k_sum<float><<<nb, RED_T, 0, s->stream>>>(reinterpret_cast<const float2*>(s->data), N, part);
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

// complex64: exact FP32 squares, float-pair runs of 8 vectors (16 amps),
// FP64 across runs.
__global__ void __launch_bounds__(RED_T) k_norm_c64(const float4* __restrict__ s, uint64_t N2,
                                                    double* __restrict__ part) {
  double acc = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  while (i < N2) {
    float hs = 0.f, hc = 0.f;
#pragma unroll 1
    for (int r = 0; r < 8 && i < N2; ++r, i += G) {
      const float4 v = s[i];
      const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float p = x[k] * x[k];
        ff_acc(hs, hc, p, fmaf(x[k], x[k], -p));
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
// p_i = re*re + im*im, each product and the sum rounded on its own (the
// same operations as the FP64 reference; complex64 inputs are widened
// first, which makes the products exact).
template <typename R>
__device__ __forceinline__ double prob_of(typename CT<R>::V2 v) {
  const double re = (double)v.x, im = (double)v.y;
  return __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
}

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
// <psi|P|psi> = sum_j conj(C[j^x]) i^{|x&z|} (-1)^{|j&z|} C[j].
template <typename R>
__global__ void __launch_bounds__(RED_T) k_expect(const typename CT<R>::V2* __restrict__ s, uint64_t N,
                                                  uint64_t x, uint64_t z, double* __restrict__ part) {
  double ar = 0.0, ai = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += G) {
    const auto v = s[j];
    const auto w = s[j ^ x];
    double vr = (double)v.x, vi = (double)v.y;
    if (__popcll(j & z) & 1) {
      vr = -vr;
      vi = -vi;
    }
    const double wr = (double)w.x, wi = (double)w.y;
    ar = fma(wr, vr, ar);
    ar = fma(wi, vi, ar);
    ai = fma(wr, vi, ai);
    ai = fma(-wi, vr, ai);
  }
  block_sum2(ar, ai);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ar;
    part[2 * blockIdx.x + 1] = ai;
  }
}

qc_status reduce_expect(const qc_state* s, uint64_t x, uint64_t z, double* out_host) {
  const uint64_t N = 1ull << s->n;
  double* part = s->scratch + QC_SCR_PARTIALS;
  const unsigned nb = std::min<unsigned>(grid_for(N, RED_T * 4, 8), RED_MAXB);
  if (s->dt == QC_C128)
    k_expect<double><<<nb, RED_T, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), N, x, z, part);
  else
    k_expect<float><<<nb, RED_T, 0, s->stream>>>(reinterpret_cast<const float2*>(s->data), N, x, z, part);
  k_final2<<<1, RED_T, 0, s->stream>>>(part, nb, s->scratch + QC_SCR_MISC);
  qc_status st = check_launch("expect", 2);
  if (st) return st;
  double h[2];
  cudaError_t e = cudaMemcpyAsync(h, s->scratch + QC_SCR_MISC, sizeof h, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "expect readback");
  // multiply by i^{|x&z|}
  const int ny = __builtin_popcountll(x & z) & 3;
  const double r = h[0], i = h[1];
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

// Per-block weight sums; status bits for unusable probabilities.
template <typename R>
__global__ void __launch_bounds__(SMP_T) k_wsum(const typename CT<R>::V2* __restrict__ s, uint64_t N,
                                                uint64_t* __restrict__ bsum, uint64_t* __restrict__ status) {
  // coalesced: the sum does not depend on which thread adds which weight
  const uint64_t base = (uint64_t)blockIdx.x * SMP_BLOCK;
  bool bad = false;
  uint64_t t = 0;
#pragma unroll
  for (int k = 0; k < SMP_PER; ++k) {
    const uint64_t i = base + (uint64_t)k * SMP_T + threadIdx.x;
    if (i < N) t = sat_add(t, weight_of<R>(s[i], &bad));
  }
  uint64_t tot = 0;
  block_excl_scan_u64(t, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr((unsigned long long*)status, SMP_BAD_P);
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

qc_status launch_sample(const qc_state* s, uint64_t seed, int64_t shots, uint64_t* out) {
  const uint64_t N = 1ull << s->n;
  const uint64_t nb = (N + SMP_BLOCK - 1) / SMP_BLOCK;
  const bool local = (uint64_t)shots <= nb;
  // [cdf (many shots only)] [block offsets nb] [total] [status]
  const uint64_t words = (local ? 0 : N) + nb + 2;
  uint64_t* buf = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&buf, words * sizeof(uint64_t), s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sampler buffer");
  uint64_t* cdf = buf;
  uint64_t* bsum = buf + (local ? 0 : N);
  uint64_t* tail = bsum + nb;
  uint64_t* status = tail + 1;
  e = cudaMemsetAsync(status, 0, sizeof(uint64_t), s->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(buf, s->stream);
    return cuda_fail(e, "sampler status reset");
  }
  if (s->dt == QC_C128)
    k_wsum<double><<<(unsigned)nb, SMP_T, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), N, bsum, status);
  else
    k_wsum<float><<<(unsigned)nb, SMP_T, 0, s->stream>>>(reinterpret_cast<const float2*>(s->data), N, bsum, status);
  k_scan_bsum<<<1, 1024, 0, s->stream>>>(bsum, nb, tail, status);
  qc_status st = check_launch("sample weights", 2);
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
static uint64_t* g_noalloc_ptr[64] = {nullptr};

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
  if (!g_noalloc_ptr[dev]) {  // first call on this device: look up the scratch address
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "qc_sample_noalloc: scratch address");
    g_noalloc_ptr[dev] = reinterpret_cast<uint64_t*>(ptr);
  }
  uint64_t* cdf = g_noalloc_ptr[dev];
  uint64_t* bsum = cdf + NA_CDF;
  uint64_t* status = bsum + NA_BSUM;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t N = 1ull << n;
  const uint64_t nb = (N + SMP_BLOCK - 1) / SMP_BLOCK;
  e = cudaMemsetAsync(status, 0, sizeof(uint64_t), st);  // the previous call's status is stale
  if (e != cudaSuccess) return cuda_fail(e, "qc_sample_noalloc: status reset");
  if (dt == QC_C128) {
    const double2* d = reinterpret_cast<const double2*>(psi_dev);
    k_wsum<double><<<(unsigned)nb, SMP_T, 0, st>>>(d, N, bsum, status);
    k_scan_bsum<<<1, 1024, 0, st>>>(bsum, nb, nullptr, status);
    k_wcdf<double><<<(unsigned)nb, SMP_T, 0, st>>>(d, N, bsum, cdf);
  } else {
    const float2* d = reinterpret_cast<const float2*>(psi_dev);
    k_wsum<float><<<(unsigned)nb, SMP_T, 0, st>>>(d, N, bsum, status);
    k_scan_bsum<<<1, 1024, 0, st>>>(bsum, nb, nullptr, status);
    k_wcdf<float><<<(unsigned)nb, SMP_T, 0, st>>>(d, N, bsum, cdf);
  }
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
