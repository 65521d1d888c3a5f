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
__global__ void __launch_bounds__(256) k_grover_pass_c128(double2* __restrict__ s, uint64_t N, const double* __restrict__ scr) {
  const double tr = 2.0 * scr[QC_SCR_MEAN];
  const ff ti = ff_from_d(2.0 * scr[QC_SCR_MEAN + 1]);
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + G < N; i += 2 * G) {
    double2 a = s[i], b = s[i + G];
    s[i] = grover_c128(a, tr, ti);
    s[i + G] = grover_c128(b, tr, ti);
  }
  if (i < N) s[i] = grover_c128(s[i], tr, ti);
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
    k_grover_pass_c128<<<resident_grid(k_grover_pass_c128, T, N, 2 * T), T, 0, s->stream>>>(
        reinterpret_cast<double2*>(s->data), N, s->scratch);
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
  st = step_with(s, dml);
  s->sum_valid = (st == QC_OK);
  return st;
}

// ---------------------------------------------------- whole small run ----
// HALL|0..0> followed by `iters` Grover steps, one block, state in shared
// memory.  The mean is recomputed from the amplitudes every step (FP64).
template <typename R>
__global__ void __launch_bounds__(1024) k_grover_small(typename CT<R>::V2* __restrict__ s, int n,
                                                       const MarkedList* __restrict__ ML, int iters) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Cx<R>* sm = reinterpret_cast<Cx<R>*>(smraw);
  __shared__ double red[2][32];
  __shared__ double mean[2];
  const int N = 1 << n;
  const R a = (R)(1.0 / sqrt(ldexp(1.0, n)));
  for (int i = threadIdx.x; i < N; i += blockDim.x) sm[i] = cmake<R>(a, (R)0);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int it = 0; it < iters; ++it) {
    // oracle (Eq. oracle1)
    for (int i = threadIdx.x; i < ML->m; i += blockDim.x) {
      const uint64_t j = ML->idx[i];
      sm[j] = cmake<R>(-sm[j].re, -sm[j].im);
    }
    __syncthreads();
    double ar = 0.0, ai = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      ar += (double)sm[i].re;
      ai += (double)sm[i].im;
    }
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) {
      red[0][warp] = ar;
      red[1][warp] = ai;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tr = 0.0, ti = 0.0;
      for (int w = 0; w < nw; ++w) {
        tr += red[0][w];
        ti += red[1][w];
      }
      mean[0] = tr / (double)N;
      mean[1] = ti / (double)N;
    }
    __syncthreads();
    const R t2r = (R)(2.0 * mean[0]), t2i = (R)(2.0 * mean[1]);
    for (int i = threadIdx.x; i < N; i += blockDim.x) sm[i] = cmake<R>(t2r - sm[i].re, t2i - sm[i].im);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) s[i] = CT<R>::make(sm[i].re, sm[i].im);
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
