// A dense 2^k x 2^k operator on k qubits: OneOpA and TwoOpA (sec. 3-4,
// Eqs. resmat1 / resmat2) extended to k qubits, the fused "k-qubit block"
// of a circuit.  Local index l of a group has bit b on qubit qubits[b];
// group g is the assignment of the other n - k qubits, and
//   new C[g | offs[l]] = sum_l' U[l][l'] C[g | offs[l']].
//
// With the state's interleaved (re, im) layout a group is a row of 2^{k+1}
// reals and the update is one real matrix product Y = X W, with
//   W[2l][2j] = Re U[j][l],   W[2l+1][2j] = -Im U[j][l],
//   W[2l][2j+1] = Im U[j][l], W[2l+1][2j+1] = Re U[j][l]   (K = N = 2^{k+1}).
// At k = 5 that is 256 flops per amplitude, more than the FP32 pipe can
// feed at HBM speed, so complex64 k = 5 runs on the 5th-generation tensor
// cores (tcgen05 kind::f16 with bf16 inputs, FP32 accumulators in tensor
// memory).  Each operand is scaled by a power of two and cut into three
// integer-valued bf16 digits, x = 2^-s (a0 + 2^-8 a1 + 2^-16 a2); the eight
// digit products down to weight 2^-16 go to three accumulators, the first
// two of which sum integers exactly, so no product or partial sum is
// rounded toward zero and the result keeps FP32-level accuracy without
// drift.  Other k and complex128 run on CUDA cores (complex128 in
// double-float; k <= 3 in the compiled one-thread-per-group kernel).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cuda_bf16.h>

#include "common.cuh"
#include "slices.cuh"
#include "tc5.cuh"

namespace qc {


__device__ __forceinline__ uint64_t group_base(uint64_t g, const DenseMap& M) {
  for (int b = 0; b < M.k; ++b) g = insert0(g, M.pos[b]);
  return g;
}

// ------------------------------------------------------ CUDA cores -------
// A CTA stages DENSE_AMPS amplitudes (DENSE_AMPS / 2^k groups) in shared
// memory, with all DENSE_PER loads of a thread in flight before its first
// shared-memory store, then every thread forms outputs
// sum_l' U[l][l'] x[l'] with U in shared memory.
#define DENSE_T 256
#define DENSE_AMPS 2048
#define DENSE_PER (DENSE_AMPS / DENSE_T)

template <typename R> struct DenseT;
template <> struct DenseT<float> {
  typedef float2 V;
  typedef float2 S;  // shared-memory element
  static __device__ __forceinline__ S load(const V* p, uint64_t i) { return p[i]; }
  static __device__ __forceinline__ S cvt(const V& v) { return v; }
  static __device__ __forceinline__ void store(V* p, uint64_t i, const S& z) { p[i] = z; }
  static __device__ __forceinline__ S zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void mac(S& acc, const S& u, const S& x) {
    acc.x = fmaf(u.x, x.x, fmaf(-u.y, x.y, acc.x));
    acc.y = fmaf(u.x, x.y, fmaf(u.y, x.x, acc.y));
  }
  static __device__ __forceinline__ S from_d(double re, double im) { return make_float2((float)re, (float)im); }
};
template <> struct DenseT<double> {
  typedef double2 V;
  typedef ffc S;
  static __device__ __forceinline__ S cvt(const V& v) { return ffc_make(ff_from_d(v.x), ff_from_d(v.y)); }
  static __device__ __forceinline__ S load(const V* p, uint64_t i) { return cvt(p[i]); }
  static __device__ __forceinline__ void store(V* p, uint64_t i, const S& z) {
    p[i] = make_double2(ff_to_d(z.re), ff_to_d(z.im));
  }
  static __device__ __forceinline__ S zero() { return ffc_make(ff_make(0.f, 0.f), ff_make(0.f, 0.f)); }
  static __device__ __forceinline__ void mac(S& acc, const S& u, const S& x) {
    acc.re = ff_add(acc.re, ff_dot2m(u.re, x.re, u.im, x.im));
    acc.im = ff_add(acc.im, ff_dot2p(u.re, x.im, u.im, x.re));
  }
  static __device__ __forceinline__ S from_d(double re, double im) { return ffc_make(ff_from_d(re), ff_from_d(im)); }
};

// dynamic shared memory: U (4^k elements) then X (DENSE_AMPS)
template <typename R>
__global__ void __launch_bounds__(DENSE_T) k_dense(typename DenseT<R>::V* __restrict__ psi, uint64_t ngroups,
                                               const double* __restrict__ U, DenseMap M) {
  typedef DenseT<R> D;
  typedef typename D::S S;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int dim = 1 << M.k;
  S* Us = reinterpret_cast<S*>(dsm);
  S* X = Us + dim * dim;
  // transposed: Us[l' dim + l] = U[l][l'], so lanes with consecutive l read
  // consecutive words (the row-major copy would be a dim-way bank conflict)
  for (int e = threadIdx.x; e < dim * dim; e += blockDim.x) {
    const int l = e / dim, lp = e % dim;
    Us[lp * dim + l] = D::from_d(U[2 * e], U[2 * e + 1]);
  }
  const int G = DENSE_AMPS >> M.k;  // groups per iteration (k <= 6: at least 32)
  for (uint64_t g0 = (uint64_t)blockIdx.x * G; g0 < ngroups; g0 += (uint64_t)gridDim.x * G) {
    const int ng = (int)min((uint64_t)G, ngroups - g0);
    __syncthreads();  // U staged; the previous groups' outputs are written
    typename D::V v[DENSE_PER];
#pragma unroll
    for (int u = 0; u < DENSE_PER; ++u) {
      const int e = threadIdx.x + u * DENSE_T;
      const int gi = e >> M.k, l = e & (dim - 1);
      if (gi < ng) v[u] = psi[group_base(g0 + gi, M) | M.offs[l]];
    }
#pragma unroll
    for (int u = 0; u < DENSE_PER; ++u) {
      const int e = threadIdx.x + u * DENSE_T;
      if ((e >> M.k) < ng) X[e] = D::cvt(v[u]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ng * dim; e += blockDim.x) {
      const int gi = e >> M.k, l = e & (dim - 1);
      S acc = D::zero();
      const S* xr = X + gi * dim;
      for (int lp = 0; lp < dim; ++lp) D::mac(acc, Us[lp * dim + l], xr[lp]);
      D::store(psi, group_base(g0 + gi, M) | M.offs[l], acc);
    }
  }
}

// complex128 blocks of K <= 3 qubits, compiled per K, one thread per group:
// the thread loads its group's 2^K amplitudes (integer-lean conversions),
// runs all 2^{K+1} output components as running dots at once (ffacc: one
// renormalisation per four terms instead of one per complex multiply-add;
// 2^{K+1} independent chains), and writes the group back.  The operator, as
// double-float, sits in shared memory, and every lane of a warp reads the
// same entry (a broadcast).  Measured on the 24-qubit, 200-layer random
// circuit fused into 1108 three-qubit blocks: 403.7 ms, against 559.8 ms with
// k_dense (runtime loop, a renormalisation per term) and 472 ms with one
// output per thread (fewer independent chains).
template <int K>
__global__ void __launch_bounds__(DENSE_T, K == 3 ? 2 : 3) k_dense_grp(double2* __restrict__ psi, uint64_t ngroups,
                                                    const double* __restrict__ U, DenseMap M) {
  constexpr int DIM = 1 << K;
  __shared__ ffc Us[DIM * DIM];  // row-major: Us[l DIM + l'] = U[l][l']
  for (int e = threadIdx.x; e < DIM * DIM; e += blockDim.x)
    Us[e] = ffc_make(ff_from_d_fast(U[2 * e]), ff_from_d_fast(U[2 * e + 1]));
  __syncthreads();
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups;
       g += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t base = group_base(g, M);
    ffc x[DIM];
    {
      double2 v[DIM];
#pragma unroll
      for (int lp = 0; lp < DIM; ++lp) v[lp] = psi[base | M.offs[lp]];
#pragma unroll
      for (int lp = 0; lp < DIM; ++lp) x[lp] = ffc_make(ff_from_d_fast(v[lp].x), ff_from_d_fast(v[lp].y));
    }
    ffacc re[DIM], im[DIM];
#pragma unroll
    for (int l = 0; l < DIM; ++l) {
      const ffc u = Us[l * DIM];
      re[l] = ffacc_first(u.re, x[0].re);
      im[l] = ffacc_first(u.re, x[0].im);
      ffacc_add(re[l], ff_neg(u.im), x[0].im);
      ffacc_add(im[l], u.im, x[0].re);
    }
#pragma unroll
    for (int lp = 1; lp < DIM; ++lp) {
#pragma unroll
      for (int l = 0; l < DIM; ++l) {
        const ffc u = Us[l * DIM + lp];
        ffacc_add(re[l], u.re, x[lp].re);
        ffacc_add(re[l], ff_neg(u.im), x[lp].im);
        ffacc_add(im[l], u.re, x[lp].im);
        ffacc_add(im[l], u.im, x[lp].re);
        if (lp & 1) {  // four terms per component since the last
          ffacc_norm(re[l]);
          ffacc_norm(im[l]);
        }
      }
    }
#pragma unroll
    for (int l = 0; l < DIM; ++l)
      psi[base | M.offs[l]] = make_double2(ff_to_d_fast(ffacc_result(re[l])), ff_to_d_fast(ffacc_result(im[l])));
  }
}

// ----------------------------------------------------- tensor cores ------
// complex64, k = 5: rows of K = 64 reals, N = 64, tiles of M = 128 rows, on
// tcgen05 kind::f16 with bf16 digit slices (slices.cuh).  Row r of a tile
// (one group) is scaled by 2^(134 - E_r) from its largest magnitude and cut
// into digits a0, a1, a2; W^T into b0, b1, b2 with one scale per operator.
// With y = a0 + 2^-8 (a1 + a2) and v = b0 + 2^-8 (b1 + b2),
//   y v = a0 b0 + 2^-8 (a0 b1 + a1 b0)
//         + 2^-8 (a0 b2 + a2 b0 + a1 (2^-8 b1) + a1 (2^-8 b2) + a2 (2^-8 b1))
//         + 2^-16 a2 b2,
// and three FP32 accumulators in tensor memory hold
//   acc0 = sum a0 b0,  acc1 = sum a0 b1 + a1 b0   (exact integers below 2^24)
//   acc2 = the fractional terms (2^-8 b1 and 2^-8 b2 are extra W digits),
// so the output is (acc0 + 2^-8 (acc1 + acc2)) 2^(E_r - 134) 2^(E_w - 134).
// acc0 and acc1 are exact, so the tensor cores' truncating accumulation
// leaves no bias in them; acc2 is about 2^-8 of acc1 and enters 2^-8 lower
// still.  The one omitted term, 2^-16 a2 b2 (|a2|, |b2| <= 1/2), is below
// 2^-18 of a unit of y v, far under the final rounding.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices (8 bf16 along K), 128 contiguous bytes
// each; core matrices adjacent in K are 128 B apart (leading byte offset),
// 8-row groups are 8 * 128 = 1024 B apart (stride byte offset).
#define TC_M 128
#define TC_T 256  // threads: two per tile row (halves of 16 amplitudes)
#define TC_K 64
#define TC_N 64
#define TC_A_SLICE TC5_A_SLICE  // 16 KiB per A digit
#define TC_B_SLICE TC5_B_SLICE  // 8 KiB per W digit
#define TC_NA 3                       // a0, a1, a2
#define TC_NB 5                       // b0, b1, b2, 2^-8 b1, 2^-8 b2
#define TC_OP_BYTES (TC_NB * TC_B_SLICE)  // device operator: the W digits, then the W scale (float)
// Two CTAs per SM (a third does not fit: 3 x 89 KiB > 227 KiB), 256 TMEM
// columns each (three 64-column accumulators; allocations are powers of two).
#define TC_SMEM (TC_NA * TC_A_SLICE + TC_NB * TC_B_SLICE + TC_M * 4 + 64)
#define TC_TMEM_COLS 256

__device__ __forceinline__ uint32_t abs_bits(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }
__device__ __forceinline__ uint32_t max4_bits(const float4& v) {
  return max(max(abs_bits(v.x), abs_bits(v.y)), max(abs_bits(v.z), abs_bits(v.w)));
}

// Two reals into their three digits, each pair packed as bf16x2 (element
// k in the low half, at the lower address).
__device__ __forceinline__ void digits2(float x, float y, float scale, uint32_t& w0, uint32_t& w1, uint32_t& w2) {
  float a0, a1, a2, b0, b1, b2;
  slice_digits(x, scale, a0, a1, a2);
  slice_digits(y, scale, b0, b1, b2);
  __nv_bfloat162 t = __floats2bfloat162_rn(a0, b0);
  w0 = *reinterpret_cast<const uint32_t*>(&t);
  t = __floats2bfloat162_rn(a1, b1);
  w1 = *reinterpret_cast<const uint32_t*>(&t);
  t = __floats2bfloat162_rn(a2, b2);
  w2 = *reinterpret_cast<const uint32_t*>(&t);
}

// Four reals of one row into their three digit slices (8 bytes each).
__device__ __forceinline__ void stage4(const float4& v, float scale, unsigned char* A, uint32_t off) {
  uint2 d0, d1, d2;
  digits2(v.x, v.y, scale, d0.x, d1.x, d2.x);
  digits2(v.z, v.w, scale, d0.y, d1.y, d2.y);
  *reinterpret_cast<uint2*>(A + off) = d0;
  *reinterpret_cast<uint2*>(A + TC_A_SLICE + off) = d1;
  *reinterpret_cast<uint2*>(A + 2 * TC_A_SLICE + off) = d2;
}

// Persistent CTAs of 256 threads.  Per tile of 128 groups: the row maxima
// (shared-memory atomics), the digit slices of every row, 32 MMAs issued by
// thread 0 into three 128 x 64 FP32 accumulators and committed to an
// mbarrier, then every warp reads its 32 accumulator lanes back and writes
// its rows.  Wd holds the W^T digits (b0, b1, b2, 2^-8 b1, 2^-8 b2; N x K each) and
// then the W scale.  status: set to 1 if an mbarrier wait ran out (the
// kernel then stops).  spin_limit bounds each wait; no_mma = 1 issues no MMA
// and no commit, so the first wait runs out with nothing asynchronous in
// flight (the self-test of the timeout path).
__global__ void __launch_bounds__(TC_T, 2) k_dense_tc(float2* __restrict__ psi, uint64_t ngroups,
                                                   const uint16_t* __restrict__ Wd, DenseMap M,
                                                   int* __restrict__ status,
                                                   const __grid_constant__ CUtensorMap out_map, int use_tma,
                                                   uint32_t spin_limit, int no_mma) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* A = tsm;                          // TC_NA digit slices of the tile
  unsigned char* B = tsm + TC_NA * TC_A_SLICE;     // TC_NB digit slices of W^T
  uint32_t* rowmax = reinterpret_cast<uint32_t*>(B + TC_NB * TC_B_SLICE);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(rowmax + TC_M);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mbar + 1);
  __shared__ int stop;
  const int tid = threadIdx.x, warp = tid >> 5;
  // W^T digits into the canonical layout (once per CTA)
  for (int e = tid; e < TC_NB * TC_N * TC_K; e += TC_T) {
    const int s = e / (TC_N * TC_K), rc = e % (TC_N * TC_K), r = rc / TC_K, c = rc % TC_K;
    *reinterpret_cast<uint16_t*>(B + s * TC_B_SLICE + tc5_canon_off(r, c)) = Wd[e];
  }
  const float wscale = *reinterpret_cast<const float*>(Wd + TC_NB * TC_N * TC_K);
  for (int r = tid; r < TC_M; r += TC_T) rowmax[r] = 0u;
  const uint32_t mbar_a = (uint32_t)__cvta_generic_to_shared(mbar);
  if (tid == 0) {
    stop = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {  // 256 TMEM columns: the three 128 x 64 FP32 accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(tmem_holder)),
                 "n"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_holder;
  const uint32_t a_s = (uint32_t)__cvta_generic_to_shared(A), b_s = (uint32_t)__cvta_generic_to_shared(B);
  bool contig = true;
  for (int l = 0; l < 32; ++l) contig &= (M.offs[l] == (uint64_t)l);
  uint32_t phase = 0;
  const uint64_t ntiles = (ngroups + TC_M - 1) / TC_M;
  // Thread tid serves tile row `row` (its TMEM lane: warp & 3 picks the lane
  // quarter) and half `hf` of it (16 amplitudes; 32 accumulator columns).
  const int row = tid & (TC_M - 1), hf = tid >> 7;
  // contiguous targets (qubits 0..4 in order): a tile is one 32 KiB block,
  // moved by all threads together.  Chunk i of thread tid is row
  // 8 (8 hf + i) + (tid & 7), 16-byte segment 4 ((tid & 127) >> 5) +
  // ((tid >> 3) & 3): a warp reads 8 rows x 64 contiguous bytes (whole
  // sectors).
  const int crow = tid & 7, cseg = 4 * (row >> 5) + ((tid >> 3) & 3);
  // A thread's 8 float4 of a tile in registers from its load to its
  // staging; two register buffers, so tile t+2's loads are in flight during
  // tile t.
  auto fetch = [&](uint64_t tile, float4 (&R)[8], bool& rlive, uint64_t& rbase) {
    if (contig) {
      const float4* src = reinterpret_cast<const float4*>(psi) + tile * TC_M * 16;
      rlive = true;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int ii = 8 * hf + i;
        R[i] = tile * TC_M + 8 * ii + crow < ngroups ? src[(8 * ii + crow) * 16 + cseg]
                                                      : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      return;
    }
    const uint64_t g = tile * TC_M + row;
    rlive = g < ngroups;
    rbase = rlive ? group_base(g, M) : 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int l4 = 8 * hf + i;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rlive) {
        const float2 x0 = psi[rbase | M.offs[2 * l4]], x1 = psi[rbase | M.offs[2 * l4 + 1]];
        v = make_float4(x0.x, x0.y, x1.x, x1.y);
      }
      R[i] = v;
    }
  };
  // one tile: stage R, MMAs, refill R with tile + 2 grid, epilogue
  const bool tma_out = contig && use_tma;
  auto body = [&](uint64_t tile, float4 (&R)[8], bool& rlive, uint64_t& rbase) -> bool {
    const bool live = rlive;
    const uint64_t base = rbase;
    if (tma_out) {  // the previous tile's output store has read the A slices
      if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
      __syncthreads();
    }
    // row maxima (|x| bit patterns order like the values)
    if (contig) {
#pragma unroll
      for (int i = 0; i < 8; ++i) atomicMax(&rowmax[8 * (8 * hf + i) + crow], max4_bits(R[i]));
    } else {
      uint32_t mx = 0u;
#pragma unroll
      for (int i = 0; i < 8; ++i) mx = max(mx, max4_bits(R[i]));
      atomicMax(&rowmax[row], mx);
    }
    __syncthreads();
    const uint32_t Ee = slice_exp(rowmax[row]);  // the exponent of this thread's output row
#pragma unroll
    for (int i = 0; i < 8; ++i) {  // digits of two amplitudes (4 reals) per 8-byte piece of a row
      const int r = contig ? 8 * (8 * hf + i) + crow : row;
      const int k = contig ? 4 * cseg : 4 * (8 * hf + i);
      stage4(R[i], slice_scale(slice_exp(rowmax[r])), A, tc5_canon_off(r, k));
    }
    // the tensor core reads shared memory through the async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid < TC_M) rowmax[tid] = 0u;  // read by every thread above; the next tile's atomics follow the last barrier
    if (tid == 0 && !no_mma) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      // acc0 = a0 b0; acc1 = a0 b1 + a1 b0;
      // acc2 = a0 b2 + a2 b0 + a1 (2^-8 b1) + a1 (2^-8 b2) + a2 (2^-8 b1)
      const int pa[8] = {0, 0, 1, 0, 2, 1, 1, 2}, pb[8] = {0, 1, 0, 2, 0, 3, 4, 3};
      const int acc_of[8] = {0, 1, 1, 2, 2, 2, 2, 2};
      for (int t = 0; t < 8; ++t) {
        const uint32_t d = tmem + acc_of[t] * TC_N;
        const bool first = (t == 0 || t == 1 || t == 3);  // first term of its accumulator
        for (int s = 0; s < TC_K / 16; ++s)  // K = 16 bf16 per MMA: two core matrices along K
          tc5_mma_bf16(d, tc5_smem_desc(a_s + pa[t] * TC_A_SLICE + s * 2 * TC5_LBO),
                   tc5_smem_desc(b_s + pb[t] * TC_B_SLICE + s * 2 * TC5_LBO), (first && s == 0) ? 0u : 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar_a)
                   : "memory");
    }
    // tile + 2 grid's loads overlap this tile's MMAs and epilogue and the next tile
    if (tile + 2ull * gridDim.x < ntiles) fetch(tile + 2ull * gridDim.x, R, rlive, rbase);
    if (!tc5_mbar_wait(mbar_a, phase, spin_limit)) {
      if (tid == 0) atomicExch(status, 1);
      stop = 1;
    }
    phase ^= 1u;
    __syncthreads();
    if (stop) return false;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // lanes 32 (warp & 3) .. hold this warp's rows; columns 32 hf .. 32 hf + 31,
    // read and combined 16 at a time
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 32 * hf;
    const float us = slice_unscale(Ee);
    float4* stg = reinterpret_cast<float4*>(A);  // contiguous fallback: 128 rows x 16 float4, chunk c of row r at c ^ (r & 15)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float out[16], acc1[16];
      tc5_tmem_ld16(lane_base + TC_N + 16 * h, out);
      tc5_tmem_ld16(lane_base + 2 * TC_N + 16 * h, acc1);
#pragma unroll
      for (int j = 0; j < 16; ++j) acc1[j] = __fadd_rn(out[j], acc1[j]);  // acc1 + acc2
      tc5_tmem_ld16(lane_base + 16 * h, out);  // acc0
#pragma unroll
      for (int j = 0; j < 16; ++j) out[j] = __fmul_rn(__fmul_rn(__fmaf_rn(acc1[j], 0.00390625f, out[j]), wscale), us);
      if (tma_out) {
        // rows into two 128 x 32-float boxes (the A slices are free: the
        // MMAs are done) in the tensor map's 128-byte swizzle (16-byte chunk
        // c of row r at chunk c ^ (r & 7), so a warp's 32 rows hit every
        // bank)
        unsigned char* box = A + hf * (TC_M * 128);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = 4 * h + j;
          *reinterpret_cast<float4*>(box + row * 128 + ((c ^ (row & 7)) << 4)) =
              make_float4(out[4 * j], out[4 * j + 1], out[4 * j + 2], out[4 * j + 3]);
        }
      } else if (contig) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = 8 * hf + 4 * h + j;
          stg[row * 16 + (c ^ (row & 15))] = make_float4(out[4 * j], out[4 * j + 1], out[4 * j + 2], out[4 * j + 3]);
        }
      } else if (live) {
#pragma unroll
        for (int l = 0; l < 8; ++l)
          psi[base | M.offs[16 * hf + 8 * h + l]] = make_float2(out[2 * l], out[2 * l + 1]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    if (tma_out) {
      // one tensor store per box writes the rows back (rows past the state
      // are clipped by the map)
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      if (tid == 0) {
#pragma unroll
        for (int hb = 0; hb < 2; ++hb)
          asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                           reinterpret_cast<uint64_t>(&out_map)),
                       "r"(32 * hb), "r"((int)(tile * TC_M)), "r"(a_s + (uint32_t)(hb * TC_M * 128))
                       : "memory");
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
      }
    } else if (contig) {  // rows through shared memory
      __syncthreads();
      float4* dst = reinterpret_cast<float4*>(psi) + tile * TC_M * 16;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = 8 * (8 * hf + i) + crow;
        if (tile * TC_M + r < ngroups) dst[r * 16 + cseg] = stg[r * 16 + (cseg ^ (r & 15))];
      }
    }
    __syncthreads();  // every lane is read before the next tile's MMAs overwrite TMEM
    return true;
  };
  float4 RA[8], RB[8];
  bool la = false, lb = false;
  uint64_t ba = 0, bb = 0;
  if (blockIdx.x < ntiles) fetch(blockIdx.x, RA, la, ba);
  if (blockIdx.x + gridDim.x < ntiles) fetch(blockIdx.x + gridDim.x, RB, lb, bb);
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += 2ull * gridDim.x) {
    if (!body(tile, RA, la, ba)) break;
    if (tile + gridDim.x < ntiles && !body(tile + gridDim.x, RB, lb, bb)) break;
  }
  // an MMA that a timed-out wait left in flight: one more bounded wait
  if (stop && tid == 0 && !no_mma) tc5_mbar_wait(mbar_a, phase ^ 1u, spin_limit);
  // output stores in flight finish before the CTA (and its shared memory) ends
  if (tma_out && tid == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(TC_TMEM_COLS));
}

}  // namespace qc

using namespace qc;

// -------------------------------------------------------------- host ----
namespace qc {

qc_status dense_map(int n, int k, const int* qubits, DenseMap* M) {
  if (k < 1 || k > DENSE_MAX_K || k > n || !qubits) {
    set_error("dense block: k = %d must be in 1..%d and <= n = %d", k, DENSE_MAX_K, n);
    return QC_EINVAL;
  }
  *M = DenseMap{};
  M->k = k;
  uint64_t seen = 0;
  for (int b = 0; b < k; ++b) {
    if (qubits[b] < 0 || qubits[b] >= n || ((seen >> qubits[b]) & 1)) {
      set_error("dense block: qubit %d out of range or repeated", qubits[b]);
      return QC_EINVAL;
    }
    seen |= 1ull << qubits[b];
    M->pos[b] = qubits[b];
  }
  std::sort(M->pos, M->pos + k);
  for (int l = 0; l < (1 << k); ++l) {
    uint64_t o = 0;
    for (int b = 0; b < k; ++b)
      if ((l >> b) & 1) o |= 1ull << qubits[b];
    M->offs[l] = o;
  }
  return QC_OK;
}

bool dense_uses_tc(qc_dtype dt, int k) { return dt == QC_C64 && k == 5; }

size_t dense_op_bytes(qc_dtype dt, int k) {
  return dense_uses_tc(dt, k) ? TC_OP_BYTES + 16 : sizeof(double) * 2 * (size_t)(1 << k) * (1 << k);
}

// The device form of U.  For the tensor cores: W^T (W^T[nn][kk], nn the
// output real 2j or 2j+1, kk the input real 2l or 2l+1) as float, cut into
// the digit slices b0, b1, b2, 2^-8 b1, 2^-8 b2 (bf16, N x K each) with one scale
// 2^(134 - E_w) from the largest |entry|, followed by 2^(E_w - 134) as a
// float.  Otherwise U itself.
void dense_pack(qc_dtype dt, int k, const double* U, void* host_out) {
  const int dim = 1 << k;
  if (!dense_uses_tc(dt, k)) {
    memcpy(host_out, U, sizeof(double) * 2 * dim * dim);
    return;
  }
  std::vector<float> wt((size_t)TC_N * TC_K);
  for (int j = 0; j < dim; ++j)
    for (int l = 0; l < dim; ++l) {
      const double ur = U[2 * (j * dim + l)], ui = U[2 * (j * dim + l) + 1];
      const float vals[4] = {(float)ur, (float)-ui, (float)ui, (float)ur};  // (2j,2l) (2j,2l+1) (2j+1,2l) (2j+1,2l+1)
      const int rr[4] = {2 * j, 2 * j, 2 * j + 1, 2 * j + 1}, cc[4] = {2 * l, 2 * l + 1, 2 * l, 2 * l + 1};
      for (int q = 0; q < 4; ++q) wt[rr[q] * TC_K + cc[q]] = vals[q];
    }
  uint32_t mx = 0;
  for (float w : wt) mx = std::max(mx, ff_fbits(w) & 0x7FFFFFFFu);
  const uint32_t Ew = slice_exp(mx);
  const float sc = slice_scale(Ew);
  uint16_t* out = reinterpret_cast<uint16_t*>(host_out);
  const size_t S = (size_t)TC_N * TC_K;
  for (size_t e = 0; e < S; ++e) {
    float b0, b1, b2;
    slice_digits(wt[e], sc, b0, b1, b2);
    out[e] = bf16_bits_rn(b0);
    out[S + e] = bf16_bits_rn(b1);
    out[2 * S + e] = bf16_bits_rn(b2);
    out[3 * S + e] = bf16_bits_rn(b1 * 0.00390625f);  // exact: b1 is a small integer
    out[4 * S + e] = bf16_bits_rn(bf16_value(out[2 * S + e]) * 0.00390625f);  // exact: a power-of-two scaling
  }
  const float ws = slice_unscale(Ew);
  memcpy(reinterpret_cast<unsigned char*>(host_out) + TC_OP_BYTES, &ws, sizeof ws);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (looked up
// once; null if the driver does not provide it).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  }
  return fn;
}

// The state as a 2-D float tensor of 64-float rows (one group of 32
// amplitudes each), stored back by boxes of 128 rows x 32 floats with the
// 128-byte swizzle; false if it cannot be encoded (the kernel then stages
// its output through shared memory with ordinary stores).
static bool dense_out_map(const qc_state* s, uint64_t ngroups, CUtensorMap* tm) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (!fn || (reinterpret_cast<uintptr_t>(s->data) & 15)) return false;
  const cuuint64_t gdim[2] = {(cuuint64_t)TC_K, (cuuint64_t)ngroups};
  const cuuint64_t gstride[1] = {(cuuint64_t)TC_K * sizeof(float)};
  const cuuint32_t box[2] = {32, TC_M};
  const cuuint32_t estr[2] = {1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, s->data, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Launches one block on the state's stream (no allocation, no sync);
// dev_op holds dense_pack's output; status (tensor cores) is a device word
// that a timed-out wait sets to 1.
qc_status dense_launch(qc_state* s, const DenseMap& M, const void* dev_op, int* status, uint32_t spin_limit,
                       int no_mma) {
  const int k = M.k, dim = 1 << k;
  const uint64_t ngroups = 1ull << (s->n - k);
  if (dense_uses_tc(s->dt, k)) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_dense_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
      attr = true;
    }
    const uint64_t ntiles = (ngroups + TC_M - 1) / TC_M;
    const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)sm_count() * 2);
    bool contig = true;  // targets 0..4 in order: a group is 32 contiguous amplitudes
    for (int l = 0; l < dim; ++l) contig &= (M.offs[l] == (uint64_t)l);
    CUtensorMap tm;
    memset(&tm, 0, sizeof tm);
    const int use_tma = contig && dense_out_map(s, ngroups, &tm);
    k_dense_tc<<<grid, TC_T, TC_SMEM, s->stream>>>(reinterpret_cast<float2*>(s->data), ngroups,
                                                     reinterpret_cast<const uint16_t*>(dev_op), M, status, tm,
                                                     use_tma, spin_limit, no_mma);
  } else if (s->dt == QC_C64) {
    const size_t smem = sizeof(float2) * ((size_t)dim * dim + DENSE_AMPS);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_dense<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(float2) * (64 * 64 + DENSE_AMPS)));
      attr = true;
    }
    const uint64_t G = DENSE_AMPS >> M.k;
    const unsigned grid = resident_grid(k_dense<float>, DENSE_T, (int64_t)((ngroups + G - 1) / G), 1, smem);
    k_dense<float><<<grid, DENSE_T, smem, s->stream>>>(reinterpret_cast<float2*>(s->data), ngroups,
                                                    reinterpret_cast<const double*>(dev_op), M);
  } else if (k <= 3) {
    double2* d = reinterpret_cast<double2*>(s->data);
    const double* op = reinterpret_cast<const double*>(dev_op);
    switch (k) {
#define QC_DENSE_GRP(KK)                                                                    \
  case KK: {                                                                                \
    const unsigned grid = resident_grid(k_dense_grp<KK>, DENSE_T, (int64_t)ngroups, DENSE_T); \
    k_dense_grp<KK><<<grid, DENSE_T, 0, s->stream>>>(d, ngroups, op, M);                      \
    break;                                                                                  \
  }
      QC_DENSE_GRP(1) QC_DENSE_GRP(2) QC_DENSE_GRP(3)
#undef QC_DENSE_GRP
    }
  } else {
    const size_t smem = sizeof(ffc) * ((size_t)dim * dim + DENSE_AMPS);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_dense<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(ffc) * (64 * 64 + DENSE_AMPS)));
      attr = true;
    }
    const uint64_t G = DENSE_AMPS >> M.k;
    const unsigned grid = resident_grid(k_dense<double>, DENSE_T, (int64_t)((ngroups + G - 1) / G), 1, smem);
    k_dense<double><<<grid, DENSE_T, smem, s->stream>>>(reinterpret_cast<double2*>(s->data), ngroups,
                                                     reinterpret_cast<const double*>(dev_op), M);
  }
  s->sum_valid = false;
  return QC_OK;
}

}  // namespace qc

// One dense block, synchronous for the tensor cores (to read the status
// word); spin_limit and no_mma as in dense_launch.
static qc_status apply_dense_impl(qc_state* s, int k, const int* qubits, const double* U, uint32_t spin_limit,
                                  int no_mma) {
  qc_status st = check_state(s);
  if (st) return st;
  if (!U) {
    set_error("qc_apply_dense: U is NULL");
    return QC_EINVAL;
  }
  DenseMap M;
  st = dense_map(s->n, k, qubits, &M);
  if (st) return st;
  const int dim = 1 << k;
  for (int e = 0; e < 2 * dim * dim; ++e)
    if (!std::isfinite(U[e])) {
      set_error("qc_apply_dense: non-finite operator entry");
      return QC_EINVAL;
    }
  const size_t ob = dense_op_bytes(s->dt, k);
  std::vector<unsigned char> host(ob);
  dense_pack(s->dt, k, U, host.data());
  void* dbuf = nullptr;
  cudaError_t e = cudaMallocAsync(&dbuf, ob + 16, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dense operator buffer");
  int* status = reinterpret_cast<int*>(reinterpret_cast<char*>(dbuf) + ob);
  e = cudaMemcpyAsync(dbuf, host.data(), ob, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(dbuf, s->stream);
    return cuda_fail(e, "dense operator upload");
  }
  dense_launch(s, M, dbuf, status, spin_limit, no_mma);
  st = check_launch(dense_uses_tc(s->dt, k) ? "dense block (tensor cores)" : "dense block", 1);
  if (!st && dense_uses_tc(s->dt, k)) {
    int hstat = 0;
    e = cudaMemcpyAsync(&hstat, status, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "dense block status");
    else if (hstat) {
      set_error("dense block: an mbarrier wait timed out");
      st = QC_ETIMEOUT;
    }
  }
  cudaFreeAsync(dbuf, s->stream);
  return st;
}

QC_API qc_status qc_apply_dense(qc_state* s, int k, const int* qubits, const double* U) {
  clear_error();
  return apply_dense_impl(s, k, qubits, U, QC_TC_SPIN_LIMIT, 0);
}

QC_API qc_status qc_dense_timeout_selftest(qc_state* s, uint32_t spin_limit) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (s->dt != QC_C64 || s->n < 5 || spin_limit < 1 || spin_limit > QC_TC_SPIN_LIMIT) {
    set_error("qc_dense_timeout_selftest: needs a complex64 state of >= 5 qubits and 1 <= spin_limit <= %u",
              QC_TC_SPIN_LIMIT);
    return QC_EINVAL;
  }
  // identity block on qubits 0..4: any operator would do, none is applied
  std::vector<double> I(2 * 32 * 32, 0.0);
  for (int d = 0; d < 32; ++d) I[2 * (d * 32 + d)] = 1.0;
  const int q[5] = {0, 1, 2, 3, 4};
  return apply_dense_impl(s, 5, q, I.data(), spin_limit, 1);
}

// ------------------------------------------------- Hamiltonian step ------
// psi <- [1 - i dt (H1 + H2)] psi (sec. 7; hbar = 1): every one- or
// two-body term adds (-i dt h) applied to a snapshot of the state taken
// before the step -- one accumulating pass per term, the paper's repeated
// OneOpA / TwoOpA.
namespace qc {

struct HMat {
  double v[32];  // -i dt h, row-major dim x dim, (re, im)
};

template <typename R>
__global__ void __launch_bounds__(256) k_hterm(typename DenseT<R>::V* __restrict__ dst,
                                               const typename DenseT<R>::V* __restrict__ src, uint64_t ngroups,
                                               DenseMap M, HMat A) {
  typedef DenseT<R> D;
  typedef typename D::S S;
  const int dim = 1 << M.k;  // 2 or 4
  S a[16];
  for (int e = 0; e < dim * dim; ++e) a[e] = D::from_d(A.v[2 * e], A.v[2 * e + 1]);
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += G) {
    const uint64_t base = group_base(g, M);
    S x[4];
    for (int l = 0; l < dim; ++l) x[l] = D::load(src, base | M.offs[l]);
    for (int l = 0; l < dim; ++l) {
      S acc = D::load(dst, base | M.offs[l]);
      for (int lp = 0; lp < dim; ++lp) D::mac(acc, a[l * dim + lp], x[lp]);
      D::store(dst, base | M.offs[l], acc);
    }
  }
}

}  // namespace qc

QC_API qc_status qc_hamiltonian_step(qc_state* s, double dt, const qc_hterm* terms, int n_terms) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (n_terms < 0 || (n_terms > 0 && !terms) || !std::isfinite(dt)) {
    set_error("qc_hamiltonian_step: bad term list or dt");
    return QC_EINVAL;
  }
  std::vector<DenseMap> maps(n_terms);
  std::vector<HMat> mats(n_terms);
  for (int t = 0; t < n_terms; ++t) {
    const qc_hterm& T = terms[t];
    if ((T.k != 1 && T.k != 2) || T.k > s->n) {
      set_error("qc_hamiltonian_step: term %d has k = %d (1 or 2 qubits)", t, T.k);
      return QC_EINVAL;
    }
    DenseMap& M = maps[t];
    M = DenseMap{};
    M.k = T.k;
    for (int b = 0; b < T.k; ++b) {
      if (T.qubits[b] < 0 || T.qubits[b] >= s->n || (b == 1 && T.qubits[1] == T.qubits[0])) {
        set_error("qc_hamiltonian_step: term %d qubit %d out of range or repeated", t, T.qubits[b]);
        return QC_EINVAL;
      }
      M.pos[b] = T.qubits[b];
    }
    std::sort(M.pos, M.pos + T.k);
    const int dim = 1 << T.k;
    for (int l = 0; l < dim; ++l) {
      uint64_t o = 0;
      for (int b = 0; b < T.k; ++b)
        if ((l >> b) & 1) o |= 1ull << T.qubits[b];
      M.offs[l] = o;
    }
    for (int e = 0; e < dim * dim; ++e) {
      const double hr = T.h[2 * e], hi = T.h[2 * e + 1];
      if (!std::isfinite(hr) || !std::isfinite(hi)) {
        set_error("qc_hamiltonian_step: term %d has a non-finite entry", t);
        return QC_EINVAL;
      }
      mats[t].v[2 * e] = dt * hi;       // (-i dt)(hr + i hi) = dt hi - i dt hr
      mats[t].v[2 * e + 1] = -dt * hr;
    }
  }
  if (n_terms == 0) return QC_OK;
  const uint64_t N = 1ull << s->n;
  const size_t bytes = (s->dt == QC_C128 ? 16 : 8) * (size_t)N;
  void* snap = nullptr;
  cudaError_t e = cudaMallocAsync(&snap, bytes, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(snap, s->data, bytes, cudaMemcpyDeviceToDevice, s->stream);
  if (e != cudaSuccess) {
    if (snap) cudaFreeAsync(snap, s->stream);
    return cuda_fail(e, "Hamiltonian step snapshot");
  }
  for (int t = 0; t < n_terms; ++t) {
    const uint64_t ng = N >> maps[t].k;
    if (s->dt == QC_C128)
      k_hterm<double><<<resident_grid(k_hterm<double>, 256, (int64_t)ng, 256), 256, 0, s->stream>>>(
          reinterpret_cast<double2*>(s->data), reinterpret_cast<const double2*>(snap), ng, maps[t], mats[t]);
    else
      k_hterm<float><<<resident_grid(k_hterm<float>, 256, (int64_t)ng, 256), 256, 0, s->stream>>>(
          reinterpret_cast<float2*>(s->data), reinterpret_cast<const float2*>(snap), ng, maps[t], mats[t]);
  }
  st = check_launch("Hamiltonian step", n_terms);
  cudaFreeAsync(snap, s->stream);
  s->sum_valid = false;
  return st;
}
