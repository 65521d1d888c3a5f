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
// cores (tcgen05, TF32 inputs, FP32 accumulator in tensor memory) with the
// operands split hi + lo ("3xTF32": A_hi B_hi + A_hi B_lo + A_lo B_hi), which
// keeps FP32-level accuracy.  Other k and complex128 run on CUDA cores
// (complex128 in double-float).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

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

// ----------------------------------------------------- tensor cores ------
// complex64, k = 5: rows of K = 64 reals, N = 64, tiles of M = 128 rows.
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, 128 contiguous bytes each; core matrices
// adjacent in K are 128 B apart (leading byte offset), 8-row groups are
// 16 * 128 = 2048 B apart (stride byte offset).
#define TC_M 128
#define TC_T 256  // threads: two per tile row (halves of 16 amplitudes)
#define TC_K 64
#define TC_N 64
#define TC_LBO 128
#define TC_SBO 2048
#define TC_A_BYTES (TC_M * TC_K * 4)  // 32 KiB
#define TC_B_BYTES (TC_N * TC_K * 4)  // 16 KiB
#define TC_SMEM (2 * TC_A_BYTES + 2 * TC_B_BYTES + 64)
#define TC_SPIN_LIMIT (1u << 20)  // polls of try_wait; a tile takes microseconds

__device__ __forceinline__ uint32_t canon_off(int r, int k) {  // byte offset of (row r, column k)
  return (uint32_t)((r >> 3) * TC_SBO + (k >> 2) * TC_LBO + (r & 7) * 16 + (k & 3) * 4);
}

// hi = x rounded to TF32 (11 significant bits, ties away from zero, by
// integer arithmetic on the pattern); lo = x - hi exactly
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  lo = x - hi;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(TC_LBO >> 4) << 16) | ((uint64_t)(TC_SBO >> 4) << 32) |
         (1ull << 46);  // descriptor version 1, no swizzle (layout 0)
}

// kind::tf32, D = F32, A = B = TF32, both K-major, N = 64, M = 128
#define TC_IDESC ((1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24))

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(TC_IDESC), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < TC_SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 32 consecutive accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// One persistent CTA of 128 threads per tile stream.  Thread t stages row
// t of each 128-group tile (split into TF32 hi and lo), thread 0 issues the
// 3 x 8 MMAs of the tile into a 128 x 64 FP32 accumulator in tensor memory
// and commits them to an mbarrier, every warp reads its 32 accumulator
// lanes back and writes its rows.  Wt holds W^T (N x K) split hi, lo.
// status: set to 1 if an mbarrier wait ran out (the kernel then stops).
__global__ void __launch_bounds__(TC_T, 2) k_dense_tc(float2* __restrict__ psi, uint64_t ngroups,
                                                   const float* __restrict__ Wt_hi, const float* __restrict__ Wt_lo,
                                                   DenseMap M, int* __restrict__ status,
                                                   const __grid_constant__ CUtensorMap out_map, int use_tma) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* A_hi = tsm;
  unsigned char* A_lo = tsm + TC_A_BYTES;
  unsigned char* B_hi = tsm + 2 * TC_A_BYTES;
  unsigned char* B_lo = B_hi + TC_B_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(B_lo + TC_B_BYTES);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mbar + 1);
  __shared__ int stop;
  const int tid = threadIdx.x, warp = tid >> 5;
  // W^T into the canonical layout (once per CTA)
  for (int e = tid; e < TC_N * TC_K; e += TC_T) {
    const int r = e / TC_K, c = e % TC_K;
    *reinterpret_cast<float*>(B_hi + canon_off(r, c)) = Wt_hi[e];
    *reinterpret_cast<float*>(B_lo + canon_off(r, c)) = Wt_lo[e];
  }
  const uint32_t mbar_a = (uint32_t)__cvta_generic_to_shared(mbar);
  if (tid == 0) {
    stop = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {  // 64 TMEM columns: the 128 x 64 FP32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;\n" ::"r"(
        (uint32_t)__cvta_generic_to_shared(tmem_holder)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_holder;
  const uint32_t a_hi = (uint32_t)__cvta_generic_to_shared(A_hi), a_lo = (uint32_t)__cvta_generic_to_shared(A_lo);
  const uint32_t b_hi = (uint32_t)__cvta_generic_to_shared(B_hi), b_lo = (uint32_t)__cvta_generic_to_shared(B_lo);
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
  // sectors) and a quarter-warp writes one contiguous 128-byte run of the
  // K-major layout.
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
    if (tma_out) {  // the previous tile's output store has read A_hi
      if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {  // two amplitudes (4 reals) per core-matrix row
      const float4 v = R[i];
      float4 h, lo;
      tf32_split(v.x, h.x, lo.x);
      tf32_split(v.y, h.y, lo.y);
      tf32_split(v.z, h.z, lo.z);
      tf32_split(v.w, h.w, lo.w);
      const uint32_t off =
          contig ? canon_off(8 * (8 * hf + i) + crow, 4 * cseg) : canon_off(row, 4 * (8 * hf + i));
      *reinterpret_cast<float4*>(A_hi + off) = h;
      *reinterpret_cast<float4*>(A_lo + off) = lo;
    }
    // the tensor core reads shared memory through the async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t as[3] = {a_hi, a_hi, a_lo}, bs[3] = {b_hi, b_lo, b_hi};
      uint32_t acc = 0;
      for (int t = 0; t < 3; ++t)
        for (int s = 0; s < TC_K / 8; ++s) {  // K = 8 TF32 per MMA: two core matrices along K
          mma_tf32(tmem, smem_desc(as[t] + s * 2 * TC_LBO), smem_desc(bs[t] + s * 2 * TC_LBO), acc);
          acc = 1;
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar_a)
                   : "memory");
    }
    // tile + 2 grid's loads overlap this tile's MMAs and epilogue and the next tile
    if (tile + 2ull * gridDim.x < ntiles) fetch(tile + 2ull * gridDim.x, R, rlive, rbase);
    if (!mbar_wait(mbar_a, phase)) {
      if (tid == 0) atomicExch(status, 1);
      stop = 1;
    }
    phase ^= 1u;
    __syncthreads();
    if (stop) return false;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // lanes 32 (warp & 3) .. hold this warp's rows; columns 32 hf .. 32 hf + 31
    float out[32];
    tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 32 * hf, out);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    if (tma_out) {
      // rows into two 128 x 32-float boxes (A_hi is free: the MMAs are done)
      // in the tensor map's 128-byte swizzle (16-byte chunk c of row r at
      // chunk c ^ (r & 7), so a warp's 32 rows hit every bank), then one
      // tensor store per box writes them back as plain rows (rows past the
      // state are clipped by the map)
      unsigned char* box = A_hi + hf * (TC_M * 128);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        *reinterpret_cast<float4*>(box + row * 128 + ((j ^ (row & 7)) << 4)) =
            make_float4(out[4 * j], out[4 * j + 1], out[4 * j + 2], out[4 * j + 3]);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      if (tid == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
          asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                           reinterpret_cast<uint64_t>(&out_map)),
                       "r"(32 * h), "r"((int)(tile * TC_M)), "r"(a_hi + (uint32_t)(h * TC_M * 128))
                       : "memory");
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
      }
    } else if (contig) {  // rows through shared memory (A_hi is free: the MMAs are done)
#pragma unroll
      for (int l4 = 0; l4 < 8; ++l4)
        *reinterpret_cast<float4*>(A_hi + canon_off(row, 4 * (8 * hf + l4))) =
            make_float4(out[4 * l4], out[4 * l4 + 1], out[4 * l4 + 2], out[4 * l4 + 3]);
      __syncthreads();
      float4* dst = reinterpret_cast<float4*>(psi) + tile * TC_M * 16;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int ii = 8 * hf + i;
        if (tile * TC_M + 8 * ii + crow < ngroups)
          dst[(8 * ii + crow) * 16 + cseg] = *reinterpret_cast<const float4*>(A_hi + canon_off(8 * ii + crow, 4 * cseg));
      }
    } else if (live) {
#pragma unroll
      for (int l = 0; l < 16; ++l) psi[base | M.offs[16 * hf + l]] = make_float2(out[2 * l], out[2 * l + 1]);
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
  if (stop && tid == 0) mbar_wait(mbar_a, phase ^ 1u);
  // output stores in flight finish before the CTA (and its shared memory) ends
  if (tma_out && tid == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;\n" ::"r"(tmem));
}

}  // namespace qc

using namespace qc;

// -------------------------------------------------------------- host ----
namespace qc {

static uint32_t tf32_hi_bits(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  return (b + 0x1000u) & 0xFFFFE000u;
}

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
  return dense_uses_tc(dt, k) ? 2 * sizeof(float) * TC_N * TC_K : sizeof(double) * 2 * (size_t)(1 << k) * (1 << k);
}

// The device form of U: W^T split into TF32 hi and lo for the tensor cores
// (W^T[n][kk], n the output real 2j or 2j+1, kk the input real 2l or
// 2l+1), else U itself.
void dense_pack(qc_dtype dt, int k, const double* U, void* host_out) {
  const int dim = 1 << k;
  if (!dense_uses_tc(dt, k)) {
    memcpy(host_out, U, sizeof(double) * 2 * dim * dim);
    return;
  }
  float* hi = reinterpret_cast<float*>(host_out);
  float* lo = hi + TC_N * TC_K;
  for (int j = 0; j < dim; ++j)
    for (int l = 0; l < dim; ++l) {
      const double ur = U[2 * (j * dim + l)], ui = U[2 * (j * dim + l) + 1];
      const float vals[4] = {(float)ur, (float)-ui, (float)ui, (float)ur};  // (2j,2l) (2j,2l+1) (2j+1,2l) (2j+1,2l+1)
      const int rr[4] = {2 * j, 2 * j, 2 * j + 1, 2 * j + 1}, cc[4] = {2 * l, 2 * l + 1, 2 * l, 2 * l + 1};
      for (int q = 0; q < 4; ++q) {
        const float x = vals[q];
        const uint32_t hb = tf32_hi_bits(x);
        float h;
        memcpy(&h, &hb, 4);
        hi[rr[q] * TC_K + cc[q]] = h;
        lo[rr[q] * TC_K + cc[q]] = x - h;
      }
    }
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
qc_status dense_launch(qc_state* s, const DenseMap& M, const void* dev_op, int* status) {
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
                                                     reinterpret_cast<const float*>(dev_op),
                                                     reinterpret_cast<const float*>(dev_op) + TC_N * TC_K, M, status,
                                                     tm, use_tma);
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

QC_API qc_status qc_apply_dense(qc_state* s, int k, const int* qubits, const double* U) {
  clear_error();
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
  dense_launch(s, M, dbuf, status);
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
