// The ensemble density matrix of complex64 states (sec. 6.1)
//   rho[i][j] = sum_a P_a C_a(i) C_a(j)^*
// as a tensor-core contraction.  With the row vector of amplitude index i
//   A_i = (sqrt(P_a) Re C_a(i))_a ++ (sqrt(P_a) Im C_a(i))_a     (K = 2B reals)
// and, per column j, Bre_j = A_j and Bim_j = (-sqrt(P_a) Im C_a(j))_a ++
// (sqrt(P_a) Re C_a(j))_a,
//   Re rho[i][j] = A_i . Bre_j,   Im rho[i][j] = A_i . Bim_j,
// so a 128 x 32 tile of rho is one real GEMM with M = 128, N = 64 (Bre and
// Bim of 32 columns interleaved, giving rho's own (re, im) row layout) and
// K = 2B.  The operands are cut into bf16 digit slices (slices.cuh) with one
// scale per amplitude index; the leading digit products sum exactly in the
// FP32 accumulators (128 products below 2^16 each), so the result keeps
// FP32-class accuracy without the tensor cores' truncation bias (the same
// scheme as the dense block in dense.cu).
//
// k_rho_digits writes every operand tile once, already in the canonical
// shared-memory layout, to a workspace; k_rho_tc then fetches the 8 digit
// slices of a tile with cp.async.bulk (one mbarrier with a transaction
// count), issues 32 MMAs per 64-wide K chunk into three accumulators in
// tensor memory and writes its 128 x 32 complex entries.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "slices.cuh"
#include "tc5.cuh"

namespace qc {

#define RT_T 256
#define RT_NA 3  // a0, a1, a2
#define RT_NB 5  // b0, b1, b2, 2^-8 b1, 2^-8 b2
#define RT_CHUNK_BYTES (RT_NA * TC5_A_SLICE + RT_NB * TC5_B_SLICE)  // 88 KiB per K chunk
#define RT_SMEM (RT_CHUNK_BYTES + 64)
#define RT_TMEM_COLS 256  // three 64-column accumulators
#define RT_SPIN (1u << 20)

struct RhoDims {
  uint64_t N;       // amplitudes per state
  int B;            // states in the batch
  int nkc;          // K chunks of 64 (K = 2B padded)
  uint64_t nib;     // 128-row blocks of rho
  uint64_t njb;     // 32-column blocks of rho
};

__device__ __forceinline__ uint64_t a_tile(const RhoDims& d, int s, uint64_t ib, int kc) {
  return ((uint64_t)s * d.nib + ib) * d.nkc + kc;  // in units of TC5_A_SLICE
}
__device__ __forceinline__ uint64_t b_tile(const RhoDims& d, int s, uint64_t jb, int kc) {
  return ((uint64_t)s * d.njb + jb) * d.nkc + kc;  // in units of TC5_B_SLICE
}

__device__ __forceinline__ uint16_t bf16_rn(float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  return *reinterpret_cast<const uint16_t*>(&h);
}

// One warp per amplitude index i: the K = 2B reals of A_i (lane l holds
// k = l, l + 32, ...), their largest magnitude, and the digits written to
// the A tiles, the Bre row 2 (i mod 32) and the Bim row 2 (i mod 32) + 1 of
// column block i / 32.  Indices past N (padding of the last blocks) get
// zeros.
__global__ void __launch_bounds__(256) k_rho_digits(const float2* __restrict__ psi, const float* __restrict__ sqrtP,
                                                    RhoDims d, uint16_t* __restrict__ Aop,
                                                    uint16_t* __restrict__ Bop, uint8_t* __restrict__ Erow) {
  const int lane = threadIdx.x & 31;
  const uint64_t nrows = d.nib * TC5_M;
  const int K = 2 * d.B, KP = 64 * d.nkc;
  for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nrows;
       i += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
    float x[4];
    uint32_t mx = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = lane + 32 * q;
      float v = 0.f;
      if (k < K && i < d.N) {
        const int a = k < d.B ? k : k - d.B;
        const float2 c = psi[(uint64_t)a * d.N + i];
        v = sqrtP[a] * (k < d.B ? c.x : c.y);
      }
      x[q] = v;
      mx = max(mx, __float_as_uint(v) & 0x7FFFFFFFu);
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const uint32_t E = slice_exp(mx);
    const float sc = slice_scale(E);
    if (lane == 0) Erow[i] = (uint8_t)E;
    const uint64_t ib = i >> 7, jb = i >> 5;
    const int r = (int)(i & 127), nn = 2 * (int)(i & 31);
    const bool has_b = jb < d.njb;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = lane + 32 * q;
      if (k >= KP) continue;
      float a0, a1, a2;
      slice_digits(x[q], sc, a0, a1, a2);
      const uint16_t h[5] = {bf16_rn(a0), bf16_rn(a1), bf16_rn(a2), bf16_rn(a1 * 0.00390625f),
                             bf16_rn(__uint_as_float((uint32_t)bf16_rn(a2) << 16) * 0.00390625f)};
      const int kc = k >> 6, kk = k & 63;
#pragma unroll
      for (int s = 0; s < RT_NA; ++s)
        Aop[a_tile(d, s, ib, kc) * (TC5_A_SLICE / 2) + tc5_canon_off(r, kk) / 2] = h[s];
      if (has_b) {
        // Bre_i[k] = A_i[k]; Bim_i[k'] = -A_i[k] for k' = k - B (k >= B), +A_i[k] for k' = k + B (k < B)
#pragma unroll
        for (int s = 0; s < RT_NB; ++s)
          Bop[b_tile(d, s, jb, kc) * (TC5_B_SLICE / 2) + tc5_canon_off(nn, kk) / 2] = h[s];
        if (k < K) {
          const int k2 = k < d.B ? k + d.B : k - d.B;
          const uint16_t sg = k < d.B ? 0 : 0x8000;  // exact negation of a bf16
          const int kc2 = k2 >> 6, kk2 = k2 & 63;
#pragma unroll
          for (int s = 0; s < RT_NB; ++s)
            Bop[b_tile(d, s, jb, kc2) * (TC5_B_SLICE / 2) + tc5_canon_off(nn + 1, kk2) / 2] = (uint16_t)(h[s] ^ sg);
        }
      }
    }
    if (has_b)  // Bim's padding columns k2 in [K, KP) take zeros
      for (int k2 = K + lane; k2 < KP; k2 += 32) {
        const int kc2 = k2 >> 6, kk2 = k2 & 63;
#pragma unroll
        for (int s = 0; s < RT_NB; ++s)
          Bop[b_tile(d, s, jb, kc2) * (TC5_B_SLICE / 2) + tc5_canon_off(nn + 1, kk2) / 2] = 0;
      }
  }
}

// One CTA per 128 x 32 tile of rho.
__global__ void __launch_bounds__(RT_T, 2) k_rho_tc(const uint16_t* __restrict__ Aop, const uint16_t* __restrict__ Bop,
                                                   const uint8_t* __restrict__ Erow, RhoDims d,
                                                   float2* __restrict__ rho, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char rsm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(rsm + RT_CHUNK_BYTES);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2);
  __shared__ int stop;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint64_t jb = blockIdx.x, ib = blockIdx.y;
  const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(rsm);
  const uint32_t bar_ld = (uint32_t)__cvta_generic_to_shared(bars), bar_mma = bar_ld + 8;
  if (tid == 0) {
    stop = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_ld));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_mma));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(tmem_holder)),
                 "n"(RT_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_holder;
  uint32_t ph_ld = 0, ph_mma = 0;
  for (int kc = 0; kc < d.nkc; ++kc) {
    if (tid == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar_ld), "r"(RT_CHUNK_BYTES)
                   : "memory");
      for (int s = 0; s < RT_NA; ++s) {
        const uint16_t* src = Aop + a_tile(d, s, ib, kc) * (TC5_A_SLICE / 2);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                s_base + (uint32_t)(s * TC5_A_SLICE)),
            "l"(src), "r"(TC5_A_SLICE), "r"(bar_ld)
            : "memory");
      }
      for (int s = 0; s < RT_NB; ++s) {
        const uint16_t* src = Bop + b_tile(d, s, jb, kc) * (TC5_B_SLICE / 2);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                s_base + (uint32_t)(RT_NA * TC5_A_SLICE + s * TC5_B_SLICE)),
            "l"(src), "r"(TC5_B_SLICE), "r"(bar_ld)
            : "memory");
      }
    }
    if (!tc5_mbar_wait(bar_ld, ph_ld, RT_SPIN)) {
      if (tid == 0) {
        atomicExch(status, 1);
        tc5_mbar_wait(bar_ld, ph_ld, RT_SPIN);  // copies still in flight: one more bounded wait
      }
      stop = 1;
    }
    ph_ld ^= 1u;
    __syncthreads();
    if (stop) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      // acc0 = a0 b0; acc1 = a0 b1 + a1 b0;
      // acc2 = a0 b2 + a2 b0 + a1 (2^-8 b1) + a1 (2^-8 b2) + a2 (2^-8 b1)
      const int pa[8] = {0, 0, 1, 0, 2, 1, 1, 2}, pb[8] = {0, 1, 0, 2, 0, 3, 4, 3};
      const int acc_of[8] = {0, 1, 1, 2, 2, 2, 2, 2};
      for (int t = 0; t < 8; ++t) {
        const bool first = kc == 0 && (t == 0 || t == 1 || t == 3);
        for (int s = 0; s < TC5_K / 16; ++s)
          tc5_mma_bf16(tmem + acc_of[t] * TC5_N,
                       tc5_smem_desc(s_base + pa[t] * TC5_A_SLICE + s * 2 * TC5_LBO),
                       tc5_smem_desc(s_base + RT_NA * TC5_A_SLICE + pb[t] * TC5_B_SLICE + s * 2 * TC5_LBO),
                       (first && s == 0) ? 0u : 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar_mma)
                   : "memory");
    }
    // the MMAs have read this chunk before the next one overwrites it
    if (!tc5_mbar_wait(bar_mma, ph_mma, RT_SPIN)) {
      if (tid == 0) {
        atomicExch(status, 1);
        tc5_mbar_wait(bar_mma, ph_mma, RT_SPIN);  // MMAs still in flight: one more bounded wait
      }
      stop = 1;
    }
    ph_mma ^= 1u;
    __syncthreads();
    if (stop) break;
  }
  if (!stop) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const int row = tid & 127, hf = tid >> 7;
    const uint64_t i = ib * TC5_M + row;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 32 * hf;
    const float ui = slice_unscale(Erow[i]);
    const uint64_t j0 = jb * 32 + 16 * hf;  // this thread's 16 columns
    const uint4 ej4 = *reinterpret_cast<const uint4*>(Erow + j0);
    const uint8_t* ej = reinterpret_cast<const uint8_t*>(&ej4);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float y[16], t1[16];
      tc5_tmem_ld16(lane_base + TC5_N + 16 * h, y);
      tc5_tmem_ld16(lane_base + 2 * TC5_N + 16 * h, t1);
#pragma unroll
      for (int c = 0; c < 16; ++c) t1[c] = __fadd_rn(y[c], t1[c]);  // acc1 + acc2
      tc5_tmem_ld16(lane_base + 16 * h, y);                          // acc0
#pragma unroll
      for (int c = 0; c < 16; ++c)
        y[c] = __fmul_rn(__fmul_rn(__fmaf_rn(t1[c], 0.00390625f, y[c]), ui), slice_unscale(ej[8 * h + c / 2]));
      if (i < d.N) {
        float4* dst = reinterpret_cast<float4*>(rho + i * d.N + j0 + 8 * h);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (j0 + 8 * h + 2 * q < d.N) dst[q] = make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(RT_TMEM_COLS));
}

// rho of a complex64 batch of B <= 64 states on the tensor cores (K = 2B <=
// 128: one row of A per warp, four reals per lane); synchronous (reads the
// status word of the bounded waits).
qc_status rho_tc_c64(const float2* psi, int n, int B, const double* P_host, float2* rho, cudaStream_t s) {
  RhoDims d;
  d.N = 1ull << n;
  d.B = B;
  d.nkc = (2 * B + 63) / 64;
  d.nib = (d.N + TC5_M - 1) / TC5_M;
  d.njb = (d.N + 31) / 32;
  const size_t bytesA = (size_t)RT_NA * d.nib * d.nkc * TC5_A_SLICE;
  const size_t bytesB = (size_t)RT_NB * d.njb * d.nkc * TC5_B_SLICE;
  const size_t bytesE = (size_t)(d.nib * TC5_M + 16);
  const size_t total = bytesA + bytesB + ((bytesE + 255) / 256) * 256 + 256 + sizeof(float) * B + 16;
  char* buf = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&buf, total, s);
  if (e != cudaSuccess) return cuda_fail(e, "density matrix workspace");
  uint16_t* Aop = reinterpret_cast<uint16_t*>(buf);
  uint16_t* Bop = reinterpret_cast<uint16_t*>(buf + bytesA);
  uint8_t* E = reinterpret_cast<uint8_t*>(buf + bytesA + bytesB);
  int* status = reinterpret_cast<int*>(buf + bytesA + bytesB + ((bytesE + 255) / 256) * 256);
  float* sqrtP = reinterpret_cast<float*>(status + 64);
  std::vector<float> sp(B);
  for (int a = 0; a < B; ++a) sp[a] = (float)std::sqrt(P_host[a]);
  e = cudaMemcpyAsync(sqrtP, sp.data(), sizeof(float) * B, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(E, 0, bytesE, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(buf, s);
    return cuda_fail(e, "density matrix setup");
  }
  const uint64_t rows = d.nib * TC5_M;
  k_rho_digits<<<(unsigned)std::min<uint64_t>((rows + 7) / 8, (uint64_t)sm_count() * 16), 256, 0, s>>>(psi, sqrtP, d,
                                                                                                   Aop, Bop, E);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rho_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, RT_SMEM);
    attr = true;
  }
  k_rho_tc<<<dim3((unsigned)d.njb, (unsigned)d.nib), RT_T, RT_SMEM, s>>>(Aop, Bop, E, d, rho, status);
  qc_status st = check_launch("density matrix (tensor cores)", 2);
  if (!st) {
    int h = 0;
    e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "density matrix status");
    else if (h) {
      set_error("density matrix: an mbarrier wait timed out");
      st = QC_ETIMEOUT;
    }
  }
  cudaFreeAsync(buf, s);
  return st;
}

}  // namespace qc
