// Grover search (sec. 5.1).  The Grover operator G = HALL . Inv . HALL .
// Oracle.  The oracle negates the marked amplitudes (Eq. oracle1) and
// HALL . Inv . HALL with Inv = 2|0><0| - I (Eq. inversion) equals
// 2|s><s| - I, |s> = HALL|0..0>, which maps C_i -> 2 m - C_i with m the mean
// amplitude.  So one step is one read+write pass:
//   m = (S - 2 sum_{marked} C) / N      (S = sum of all amplitudes)
//   C_i -> 2 m - C_i (unmarked),  C_i -> 2 m + C_i (marked).
// The diffusion preserves the mean, so the new amplitude sum is known
// without reading the state again: S' = N (2m - m) = N m (for complex64 the
// rounded 2m is used).  S is kept in the state's device scratch and
// recomputed by a reduction only after another operation changed the state.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace qc {

struct MarkedList {
  int m;
  uint64_t idx[QC_MAX_MARKED];
};

// One block: m from the running sum and the marked amplitudes; saves the
// marked amplitudes and the next running sum.
template <typename R>
__global__ void k_grover_prep(const typename CT<R>::V2* __restrict__ s, uint64_t N, const MarkedList* __restrict__ ML,
                              double* __restrict__ scr) {
  __shared__ double red[2][256];
  double ar = 0.0, ai = 0.0;
  for (int i = threadIdx.x; i < ML->m; i += blockDim.x) {
    const auto v = s[ML->idx[i]];
    scr[QC_SCR_MARKED + 2 * i] = (double)v.x;
    scr[QC_SCR_MARKED + 2 * i + 1] = (double)v.y;
    ar += (double)v.x;
    ai += (double)v.y;
  }
  red[0][threadIdx.x] = ar;
  red[1][threadIdx.x] = ai;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double Nd = (double)N;
    const double mr = (scr[QC_SCR_SUM] - 2.0 * red[0][0]) / Nd;
    const double mi = (scr[QC_SCR_SUM + 1] - 2.0 * red[1][0]) / Nd;
    scr[QC_SCR_MEAN] = mr;
    scr[QC_SCR_MEAN + 1] = mi;
    const double tr = (double)(R)(2.0 * mr), ti = (double)(R)(2.0 * mi);
    scr[QC_SCR_SUM] = Nd * (tr - mr);
    scr[QC_SCR_SUM + 1] = Nd * (ti - mi);
  }
}

// C -> 2m - C over the whole state.  Real parts on the FP64 pipe, imaginary
// parts in double-float on the FP32 pipe, so that neither pipe limits the
// pass (GB300's FP64 rate allows under 2.5 operations per amplitude at HBM
// speed).
__device__ __forceinline__ double2 grover_c128(double2 a, double tr, ff ti) {
  return make_double2(tr - a.x, ff_to_d(ff_sub(ti, ff_from_d(a.y))));
}
// Four 16-byte loads in flight per thread, three blocks of 256 per SM (the
// launch caps the grid): on GB300 this streams random complex128 data at
// 0.96 of copy bandwidth, against 0.91 for two loads at eight blocks.
constexpr int GROVER_UNR = 4;
__global__ void __launch_bounds__(256, 4) k_grover_pass_c128(double2* __restrict__ s, uint64_t N, const double* __restrict__ scr) {
  const double tr = 2.0 * scr[QC_SCR_MEAN];
  const ff ti = ff_from_d(2.0 * scr[QC_SCR_MEAN + 1]);
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (GROVER_UNR - 1) * G < N; i += GROVER_UNR * G) {
    double2 a[GROVER_UNR];
#pragma unroll
    for (int u = 0; u < GROVER_UNR; ++u) a[u] = s[i + u * G];
#pragma unroll
    for (int u = 0; u < GROVER_UNR; ++u) s[i + u * G] = grover_c128(a[u], tr, ti);
  }
  for (; i < N; i += G) s[i] = grover_c128(s[i], tr, ti);
}

__global__ void __launch_bounds__(256) k_grover_pass_c64(float4* __restrict__ s, uint64_t N2, const double* __restrict__ scr) {
  const float tr = (float)(2.0 * scr[QC_SCR_MEAN]), ti = (float)(2.0 * scr[QC_SCR_MEAN + 1]);
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + G < N2; i += 2 * G) {
    float4 a = s[i], b = s[i + G];
    s[i] = make_float4(tr - a.x, ti - a.y, tr - a.z, ti - a.w);
    s[i + G] = make_float4(tr - b.x, ti - b.y, tr - b.z, ti - b.w);
  }
  if (i < N2) {
    float4 a = s[i];
    s[i] = make_float4(tr - a.x, ti - a.y, tr - a.z, ti - a.w);
  }
}

// Marked amplitudes: 2m + C_old.
template <typename R>
__global__ void k_grover_fix(typename CT<R>::V2* __restrict__ s, const MarkedList* __restrict__ ML,
                             const double* __restrict__ scr) {
  const double mr = scr[QC_SCR_MEAN], mi = scr[QC_SCR_MEAN + 1];
  const R tr = (R)(2.0 * mr), ti = (R)(2.0 * mi);
  for (int i = threadIdx.x; i < ML->m; i += blockDim.x) {
    const R cr = (R)scr[QC_SCR_MARKED + 2 * i], ci = (R)scr[QC_SCR_MARKED + 2 * i + 1];
    s[ML->idx[i]] = CT<R>::make(tr + cr, ti + ci);
  }
}

// Device copy of the marked list, kept in the handle and re-uploaded only
// when the list changes (the upload synchronises the stream once).
static qc_status upload_marked(qc_state* s, const uint64_t* marked, int m, MarkedList** out) {
  if (!s->marked_dev) {
    cudaError_t e = cudaMalloc(&s->marked_dev, sizeof(MarkedList));
    if (e != cudaSuccess) {
      s->marked_dev = nullptr;
      return cuda_fail(e, "marked list");
    }
    s->marked_host.clear();
  }
  const bool same = (int)s->marked_host.size() == m &&
                    std::equal(s->marked_host.begin(), s->marked_host.end(), marked);
  if (!same) {
    const size_t bytes = sizeof(int) * 2 + sizeof(uint64_t) * (size_t)m;
    MarkedList* h = nullptr;
    cudaError_t e = cudaMallocHost((void**)&h, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "marked list (host)");
    h->m = m;
    for (int i = 0; i < m; ++i) h->idx[i] = marked[i];
    e = cudaMemcpyAsync(s->marked_dev, h, bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFreeHost(h);
    if (e != cudaSuccess) {
      s->marked_host.clear();
      return cuda_fail(e, "marked list upload");
    }
    s->marked_host.assign(marked, marked + m);
  }
  *out = reinterpret_cast<MarkedList*>(s->marked_dev);
  return QC_OK;
}

static qc_status step_with(qc_state* s, const MarkedList* dml) {
  const uint64_t N = 1ull << s->n;
  const int T = 256;
  if (s->dt == QC_C128) {
    k_grover_prep<double><<<1, 256, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), N, dml, s->scratch);
    const unsigned g = std::min<unsigned>(resident_grid(k_grover_pass_c128, T, N, GROVER_UNR * T), 3u * (unsigned)sm_count());
    k_grover_pass_c128<<<g, T, 0, s->stream>>>(reinterpret_cast<double2*>(s->data), N, s->scratch);
    k_grover_fix<double><<<1, 256, 0, s->stream>>>(reinterpret_cast<double2*>(s->data), dml, s->scratch);
  } else {
    k_grover_prep<float><<<1, 256, 0, s->stream>>>(reinterpret_cast<const float2*>(s->data), N, dml, s->scratch);
    const uint64_t N2 = N / 2;
    if (N2 > 0)
      k_grover_pass_c64<<<resident_grid(k_grover_pass_c64, T, N2, 2 * T), T, 0, s->stream>>>(
          reinterpret_cast<float4*>(s->data), N2, s->scratch);
    k_grover_fix<float><<<1, 256, 0, s->stream>>>(reinterpret_cast<float2*>(s->data), dml, s->scratch);
  }
  return check_launch("grover step", 3);
}

qc_status launch_grover_step(qc_state* s, const uint64_t* marked, int m) {
  if (s->n < 2 && s->dt == QC_C64) {
    set_error("complex64 Grover needs n >= 2");
    return QC_EINVAL;
  }
  qc_status st = QC_OK;
  if (!s->sum_valid) {
    st = launch_sum(s);
    if (st) return st;
  }
  MarkedList* dml = nullptr;
  st = upload_marked(s, marked, m, &dml);
  if (st) return st;
  s->grover_partial_ready = false;  // the saved marked amplitudes are overwritten
  st = step_with(s, dml);
  s->sum_valid = (st == QC_OK);
  return st;
}

// ------------------------------------------ a state split over devices ----
// For a state split over several devices (one shard per device, the high
// index bits selecting the shard), the Grover mean needs the sum over all
// shards: each shard contributes P_r = S_r - 2 sum_{marked in r} C, the
// caller adds them (one scalar all-reduce) and hands back m = sum_r P_r / N.
// The pass itself is the single-device one.
template <typename R>
__global__ void k_grover_partial(const typename CT<R>::V2* __restrict__ s, const MarkedList* __restrict__ ML,
                                 double* __restrict__ scr) {
  __shared__ double red[2][256];
  double ar = 0.0, ai = 0.0;
  for (int i = threadIdx.x; i < ML->m; i += blockDim.x) {
    const auto v = s[ML->idx[i]];
    scr[QC_SCR_MARKED + 2 * i] = (double)v.x;
    scr[QC_SCR_MARKED + 2 * i + 1] = (double)v.y;
    ar += (double)v.x;
    ai += (double)v.y;
  }
  red[0][threadIdx.x] = ar;
  red[1][threadIdx.x] = ai;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // P_r in the misc slots
    scr[QC_SCR_MISC] = scr[QC_SCR_SUM] - 2.0 * red[0][0];
    scr[QC_SCR_MISC + 1] = scr[QC_SCR_SUM + 1] - 2.0 * red[1][0];
  }
}

// The given mean into the scratch, and the shard's next running sum
// S_r' = N_r (2m) - P_r (2m rounded as the pass rounds it).
template <typename R>
__global__ void k_grover_set_mean(double* __restrict__ scr, uint64_t N, double mr, double mi) {
  scr[QC_SCR_MEAN] = mr;
  scr[QC_SCR_MEAN + 1] = mi;
  const double tr = (double)(R)(2.0 * mr), ti = (double)(R)(2.0 * mi);
  scr[QC_SCR_SUM] = (double)N * tr - scr[QC_SCR_MISC];
  scr[QC_SCR_SUM + 1] = (double)N * ti - scr[QC_SCR_MISC + 1];
}

qc_status launch_grover_partial(qc_state* s, const uint64_t* marked, int m, double* out_host) {
  qc_status st = QC_OK;
  if (!s->sum_valid) {
    st = launch_sum(s);
    if (st) return st;
  }
  MarkedList* dml = nullptr;
  st = upload_marked(s, marked, m, &dml);
  if (st) return st;
  if (s->dt == QC_C128)
    k_grover_partial<double><<<1, 256, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), dml, s->scratch);
  else
    k_grover_partial<float><<<1, 256, 0, s->stream>>>(reinterpret_cast<const float2*>(s->data), dml, s->scratch);
  st = check_launch("grover partial sum");
  if (st) return st;
  cudaError_t e = cudaMemcpyAsync(out_host, s->scratch + QC_SCR_MISC, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                  s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "grover partial readback");
  s->grover_partial_ready = true;
  return QC_OK;
}

qc_status launch_grover_apply(qc_state* s, const uint64_t* marked, int m, const double* mean) {
  if (!s->grover_partial_ready || !s->sum_valid || (int)s->marked_host.size() != m ||
      !std::equal(s->marked_host.begin(), s->marked_host.end(), marked)) {
    set_error("qc_grover_apply_mean: call qc_grover_partial with the same marked list first");
    return QC_EINVAL;
  }
  s->grover_partial_ready = false;
  const uint64_t N = 1ull << s->n;
  const int T = 256;
  const MarkedList* dml = reinterpret_cast<const MarkedList*>(s->marked_dev);
  if (s->dt == QC_C128) {
    k_grover_set_mean<double><<<1, 1, 0, s->stream>>>(s->scratch, N, mean[0], mean[1]);
    const unsigned g = std::min<unsigned>(resident_grid(k_grover_pass_c128, T, N, GROVER_UNR * T), 3u * (unsigned)sm_count());
    k_grover_pass_c128<<<g, T, 0, s->stream>>>(reinterpret_cast<double2*>(s->data), N, s->scratch);
    k_grover_fix<double><<<1, 256, 0, s->stream>>>(reinterpret_cast<double2*>(s->data), dml, s->scratch);
  } else {
    k_grover_set_mean<float><<<1, 1, 0, s->stream>>>(s->scratch, N, mean[0], mean[1]);
    const uint64_t N2 = N / 2;
    if (N2 > 0)
      k_grover_pass_c64<<<resident_grid(k_grover_pass_c64, T, N2, 2 * T), T, 0, s->stream>>>(
          reinterpret_cast<float4*>(s->data), N2, s->scratch);
    k_grover_fix<float><<<1, 256, 0, s->stream>>>(reinterpret_cast<float2*>(s->data), dml, s->scratch);
  }
  qc_status st = check_launch("grover pass (given mean)", 3);
  s->sum_valid = (st == QC_OK);
  return st;
}

// ---------------------------------------------------- whole small run ----
// HALL|0..0> followed by `iters` Grover steps, one block, state in shared
// memory.  The mean is recomputed from the amplitudes every step.  One SM
// completes about 1.6 FP64 operations per clock, which would bound every
// step (a block-wide FP64 sum and an FP64 diffusion), so the run stays on
// the FP32 pipe: complex128 keeps the state as double-float (about 48
// bits) from the first to the last step, complex64 sums in float pairs.
template <typename R> struct SmallRun;
template <> struct SmallRun<double> {
  using E = ffc;
  __device__ static E start(double a) { return ffc_make(ff_from_d(a), ff_make(0.f, 0.f)); }
  __device__ static double2 out(E z) { return make_double2(ff_to_d(z.re), ff_to_d(z.im)); }
  __device__ static E neg(E z) { return ffc_make(ff_neg(z.re), ff_neg(z.im)); }
  __device__ static ff re(E z) { return z.re; }
  __device__ static ff im(E z) { return z.im; }
  // 2m = S 2^{1-n} (an exact power-of-two scaling of the double-float sum)
  __device__ static E two_mean(ff sr, ff si, float scale) {
    return ffc_make(ff_make(sr.hi * scale, sr.lo * scale), ff_make(si.hi * scale, si.lo * scale));
  }
  __device__ static E diffuse(E t2, E z) { return ffc_sub(t2, z); }
};
template <> struct SmallRun<float> {
  using E = Cx<float>;
  __device__ static E start(double a) { return cmake<float>((float)a, 0.f); }
  __device__ static float2 out(E z) { return make_float2(z.re, z.im); }
  __device__ static E neg(E z) { return cmake<float>(-z.re, -z.im); }
  __device__ static ff re(E z) { return ff_make(z.re, 0.f); }
  __device__ static ff im(E z) { return ff_make(z.im, 0.f); }
  __device__ static E two_mean(ff sr, ff si, float scale) {
    return cmake<float>((sr.hi + sr.lo) * scale, (si.hi + si.lo) * scale);
  }
  __device__ static E diffuse(E t2, E z) { return cmake<float>(t2.re - z.re, t2.im - z.im); }
};

__device__ __forceinline__ ff shfl_xor_ff(ff v, int o) {
  return ff_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

template <typename R>
__global__ void __launch_bounds__(1024) k_grover_small(typename CT<R>::V2* __restrict__ s, int n,
                                                       const MarkedList* __restrict__ ML, int iters) {
  using G = SmallRun<R>;
  using E = typename G::E;
  extern __shared__ __align__(16) unsigned char smraw[];
  E* sm = reinterpret_cast<E*>(smraw);
  __shared__ ff red[2][32];
  __shared__ E t2s;
  const int N = 1 << n;
  const float scale = ldexpf(1.f, 1 - n);  // 2 / N, exact
  const E a = G::start(1.0 / sqrt(ldexp(1.0, n)));
  for (int i = threadIdx.x; i < N; i += blockDim.x) sm[i] = a;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const ff zero = ff_make(0.f, 0.f);
  for (int it = 0; it < iters; ++it) {
    // oracle (Eq. oracle1)
    for (int i = threadIdx.x; i < ML->m; i += blockDim.x) {
      const uint64_t j = ML->idx[i];
      sm[j] = G::neg(sm[j]);
    }
    __syncthreads();
    // amplitude sum in double-float: per thread, across the warp, across warps
    ff sr = zero, si = zero;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const E z = sm[i];
      sr = ff_add(sr, G::re(z));
      si = ff_add(si, G::im(z));
    }
    for (int o = 16; o > 0; o >>= 1) {
      sr = ff_add(sr, shfl_xor_ff(sr, o));
      si = ff_add(si, shfl_xor_ff(si, o));
    }
    if (lane == 0) {
      red[0][warp] = sr;
      red[1][warp] = si;
    }
    __syncthreads();
    if (warp == 0) {
      ff r = lane < nw ? red[0][lane] : zero, q = lane < nw ? red[1][lane] : zero;
      for (int o = 16; o > 0; o >>= 1) {
        r = ff_add(r, shfl_xor_ff(r, o));
        q = ff_add(q, shfl_xor_ff(q, o));
      }
      if (lane == 0) t2s = G::two_mean(r, q, scale);
    }
    __syncthreads();
    // diffusion: C -> 2m - C (HALL . Inv . HALL)
    const E t2 = t2s;
    for (int i = threadIdx.x; i < N; i += blockDim.x) sm[i] = G::diffuse(t2, sm[i]);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) s[i] = G::out(sm[i]);
}

qc_status launch_grover_run(qc_state* s, const uint64_t* marked, int m, int iters) {
  MarkedList* dml = nullptr;
  qc_status st = upload_marked(s, marked, m, &dml);
  if (st) return st;
  const bool small = (s->dt == QC_C128) ? (s->n <= 13) : (s->n <= 14);
  if (small) {
    const size_t smem = ((size_t)1 << s->n) * amp_bytes(s->dt);
    if (s->dt == QC_C128) {
      cudaFuncSetAttribute(k_grover_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
      k_grover_small<double><<<1, 1024, smem, s->stream>>>(reinterpret_cast<double2*>(s->data), s->n, dml, iters);
    } else {
      cudaFuncSetAttribute(k_grover_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
      k_grover_small<float><<<1, 1024, smem, s->stream>>>(reinterpret_cast<float2*>(s->data), s->n, dml, iters);
    }
    st = check_launch("grover run (shared memory)");
    s->sum_valid = false;
  } else {
    st = launch_fill_uniform(s);  // HALL|0..0>; records the amplitude sum
    for (int it = 0; it < iters && !st; ++it) st = step_with(s, dml);
    s->sum_valid = (st == QC_OK);
  }
  return st;
}

}  // namespace qc
