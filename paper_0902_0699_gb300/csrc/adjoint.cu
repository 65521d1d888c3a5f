// Parameterised circuits on a batch of states and the adjoint gradient of
// E = <psi|H|psi> (not part of the QCMPI paper).
//
// The gate list is first compiled into passes: two consecutive rotations on
// the same qubit become one pass, and a full CNOT ring CNOT(0,1), CNOT(1,2),
// .., CNOT(n-1,0) -- a permutation of basis indices (prefix parity) --
// becomes one gather pass; any other gate is a pass of its own.  Batch
// element b is grid.y, so each block builds its element's matrices once.
//
// Forward: psi_b = U_G .. U_1 |0..0>.  Backward: lambda = H psi (one gather
// pass over the Pauli terms), E = Re <psi|lambda>, then the passes are
// walked in reverse; a rotation pass reads psi_j and lambda_j, accumulates
// Im <lambda_j|P_j|psi_j> -- the derivative of U_j = exp(-i theta P_j / 2)
// gives dE/dtheta_j = 2 Re <lambda_j|(-i/2) P_j|psi_j> = Im <lambda_j|P_j|psi_j>
// -- and applies U_j^dagger to both.  No intermediate state is stored: psi
// is uncomputed instead of checkpointed.
//
// Accumulation is FP64: complex128 with FMA in double; complex64 products
// are formed exactly with the FP32 two-product and summed as float pairs
// over short runs before they are added in double.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace qc {

#define ADJ_T 256
#define ADJ_GX_MAX 256

struct GateDev {
  int kind, q0, q1, param;
};

// Rotation matrices exp(-i theta P / 2) for P = X, Y, Z; H.
template <typename R>
__device__ __forceinline__ Mat2<R> gate_matrix(int kind, double theta) {
  Mat2<R> U;
  double s, c;
  sincos(0.5 * theta, &s, &c);
  const R cr = (R)c, sr = (R)s;
  const R z = (R)0;
  if (kind == QC_G_RX) {
    U.m[0] = cmake<R>(cr, z);
    U.m[1] = cmake<R>(z, -sr);
    U.m[2] = cmake<R>(z, -sr);
    U.m[3] = cmake<R>(cr, z);
  } else if (kind == QC_G_RY) {
    U.m[0] = cmake<R>(cr, z);
    U.m[1] = cmake<R>(-sr, z);
    U.m[2] = cmake<R>(sr, z);
    U.m[3] = cmake<R>(cr, z);
  } else if (kind == QC_G_RZ) {
    U.m[0] = cmake<R>(cr, -sr);
    U.m[1] = cmake<R>(z, z);
    U.m[2] = cmake<R>(z, z);
    U.m[3] = cmake<R>(cr, sr);
  } else {  // H
    const R h = (R)0.70710678118654752440;
    U.m[0] = cmake<R>(h, z);
    U.m[1] = cmake<R>(h, z);
    U.m[2] = cmake<R>(h, z);
    U.m[3] = cmake<R>(-h, z);
  }
  return U;
}

// The block's matrix for (kind, theta), or the product U_b U_a of two: one
// thread evaluates the FP64 sines and cosines (costly on GB300's FP64 pipe)
// and the block reads the result from shared memory.
template <typename R>
__device__ __forceinline__ Mat2<R> block_matrix(int ka, double tha, int kb = -1, double thb = 0.0) {
  __shared__ Mat2<double> sh;
  if (threadIdx.x == 0) {
    const Mat2<double> A = gate_matrix<double>(ka, tha);
    if (kb < 0) {
      sh = A;
    } else {
      const Mat2<double> Bm = gate_matrix<double>(kb, thb);
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) sh.m[2 * r + c] = cmul2(Bm.m[2 * r], A.m[c], Bm.m[2 * r + 1], A.m[2 + c]);
    }
  }
  __syncthreads();
  Mat2<R> U;
  for (int k = 0; k < 4; ++k) U.m[k] = cmake<R>((R)sh.m[k].re, (R)sh.m[k].im);
  __syncthreads();  // sh may be rewritten by a second call in the same kernel
  return U;
}

template <typename R>
__device__ __forceinline__ void apply_any(int kind, const Mat2<R>& U, Cx<R>& a0, Cx<R>& a1) {
  if (kind == QC_G_RY) apply2<R, MK_REAL>(U, a0, a1);
  else if (kind == QC_G_RZ) apply2<R, MK_DIAG>(U, a0, a1);
  else if (kind == QC_G_H) apply2<R, MK_HAD>(U, a0, a1);
  else if (kind == QC_G_CNOT) apply2<R, MK_SWAPX>(U, a0, a1);
  else apply2<R, MK_GENERAL>(U, a0, a1);
}

// Pair enumeration of one gate: 1q gates insert a zero at q0; CNOT inserts
// zeros at both qubits and sets the control bit.
__device__ __forceinline__ uint64_t gate_pair(const GateDev& g, uint64_t p, uint64_t& partner) {
  if (g.kind == QC_G_CNOT) {
    const int lo = min(g.q0, g.q1), hi = max(g.q0, g.q1);
    const uint64_t i0 = insert0(insert0(p, lo), hi) | (1ull << g.q0);
    partner = i0 | (1ull << g.q1);
    return i0;
  }
  const uint64_t i0 = insert0(p, g.q0);
  partner = i0 | (1ull << g.q0);
  return i0;
}

// ----------------------------------------------------- accumulators ------
template <typename R> struct Acc;
template <> struct Acc<double> {
  double a = 0.0;
  __device__ void add(double x, double y) { a = fma(x, y, a); }
  __device__ void sub(double x, double y) { a = fma(-x, y, a); }
  __device__ void flush() {}
  __device__ double value() const { return a; }
};
// complex64: products exact as float pairs (two-product), summed as a float
// pair with two-sum (relative error ~ terms * 2^-48), converted to double
// once per thread -- no FP64 instruction in the loop.
template <> struct Acc<float> {
  double a = 0.0;
  float s = 0.f, c = 0.f;
  __device__ void put(float p, float e) {
    const float t = s + p;
    const float bp = t - s;
    c += ((s - (t - bp)) + (p - bp)) + e;
    s = t;
  }
  __device__ void add(float x, float y) {
    const float p = x * y;
    put(p, fmaf(x, y, -p));
  }
  __device__ void sub(float x, float y) {
    const float p = -x * y;
    put(p, fmaf(-x, y, -p));
  }
  __device__ void flush() {
    a += (double)s + (double)c;
    s = c = 0.f;
  }
  __device__ double value() const { return a; }
};

// Accumulate Im <l|P|p> over one pair for the generator P of a rotation.
template <typename R>
__device__ __forceinline__ void acc_generator(Acc<R>& acc, int kind, const Cx<R>& p0, const Cx<R>& p1,
                                              const Cx<R>& l0, const Cx<R>& l1) {
  // Im(conj(a) b) = a.re b.im - a.im b.re
  if (kind == QC_G_RZ) {  // Z: conj(l0) p0 - conj(l1) p1
    acc.add(l0.re, p0.im); acc.sub(l0.im, p0.re);
    acc.sub(l1.re, p1.im); acc.add(l1.im, p1.re);
  } else if (kind == QC_G_RX) {  // X: conj(l0) p1 + conj(l1) p0
    acc.add(l0.re, p1.im); acc.sub(l0.im, p1.re);
    acc.add(l1.re, p0.im); acc.sub(l1.im, p0.re);
  } else {  // Y: conj(l0)(-i p1) + conj(l1)(i p0); Im(conj(a)(-i b)) = -Re(conj(a) b)
    acc.sub(l0.re, p1.re); acc.sub(l0.im, p1.im);
    acc.add(l1.re, p0.re); acc.add(l1.im, p0.im);
  }
}

__device__ __forceinline__ double block_reduce(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  __syncthreads();
  return t;
}

// ------------------------------------------------------------ forward ----
template <typename R>
__global__ void __launch_bounds__(ADJ_T) k_fwd_gate(typename CT<R>::V2* __restrict__ psi, int n, GateDev g,
                                                    const double* __restrict__ theta, int64_t stride) {
  using IO = AmpIO<R>;
  const int b = blockIdx.y;
  typename CT<R>::V2* s = psi + ((uint64_t)b << n);
  const double th = (g.kind <= QC_G_RZ) ? theta[(int64_t)b * stride + g.param] : 0.0;
  const Mat2<R> U = block_matrix<R>(g.kind, th);
  const uint64_t np = (g.kind == QC_G_CNOT) ? (1ull << (n - 2)) : (1ull << (n - 1));
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t i1;
    const uint64_t i0 = gate_pair(g, p, i1);
    Cx<R> a0 = IO::ld(s + i0), a1 = IO::ld(s + i1);
    apply_any<R>(g.kind, U, a0, a1);
    IO::st(s + i0, a0);
    IO::st(s + i1, a1);
  }
}

// Two rotations on one qubit, ga then gb: one pass with M = U_b U_a.
template <typename R>
__global__ void __launch_bounds__(ADJ_T) k_fwd_rot2(typename CT<R>::V2* __restrict__ psi, int n, GateDev ga,
                                                    GateDev gb, const double* __restrict__ theta, int64_t stride) {
  using IO = AmpIO<R>;
  const int b = blockIdx.y;
  typename CT<R>::V2* s = psi + ((uint64_t)b << n);
  const Mat2<R> M = block_matrix<R>(ga.kind, theta[(int64_t)b * stride + ga.param], gb.kind,
                                    theta[(int64_t)b * stride + gb.param]);
  const int q = ga.q0;
  const uint64_t np = 1ull << (n - 1);
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = insert0(p, q), i1 = i0 | (1ull << q);
    Cx<R> a0 = IO::ld(s + i0), a1 = IO::ld(s + i1);
    apply2<R, MK_GENERAL>(M, a0, a1);
    IO::st(s + i0, a0);
    IO::st(s + i1, a1);
  }
}

// The same pass for complex64 with 16-byte accesses: an item is two
// neighbouring pairs (q >= 1: amplitudes i0, i0+1 and i0 + 2^q, i0 + 2^q + 1)
// or one pair (q = 0: amplitudes 2v, 2v+1 in one vector); four items per
// trip on three blocks per SM (eight-byte loads, one pair per trip, streamed
// the 64-state batch at 0.78 of copy bandwidth on GB300).
constexpr int FWD_UNR = 4;
__device__ __forceinline__ void rot_v(const Mat2<float>& M, float4& A, float4& B) {
  Cx<float> a0 = cmake(A.x, A.y), c0 = cmake(A.z, A.w), a1 = cmake(B.x, B.y), c1 = cmake(B.z, B.w);
  apply2<float, MK_GENERAL>(M, a0, a1);
  apply2<float, MK_GENERAL>(M, c0, c1);
  A = make_float4(a0.re, a0.im, c0.re, c0.im);
  B = make_float4(a1.re, a1.im, c1.re, c1.im);
}
__global__ void __launch_bounds__(ADJ_T, 4) k_fwd_rot2_c64(float2* __restrict__ psi, int n, GateDev ga, GateDev gb,
                                                           const double* __restrict__ theta, int64_t stride) {
  const int b = blockIdx.y;
  float2* s = psi + ((uint64_t)b << n);
  const Mat2<float> M = block_matrix<float>(ga.kind, theta[(int64_t)b * stride + ga.param], gb.kind,
                                            theta[(int64_t)b * stride + gb.param]);
  const int q = ga.q0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) {
    float4* w = reinterpret_cast<float4*>(s);
    const uint64_t items = 1ull << (n - 1);
    for (; v + (FWD_UNR - 1) * G < items; v += FWD_UNR * G) {
      float4 A[FWD_UNR];
#pragma unroll
      for (int u = 0; u < FWD_UNR; ++u) A[u] = w[v + u * G];
#pragma unroll
      for (int u = 0; u < FWD_UNR; ++u) {
        Cx<float> a0 = cmake(A[u].x, A[u].y), a1 = cmake(A[u].z, A[u].w);
        apply2<float, MK_GENERAL>(M, a0, a1);
        w[v + u * G] = make_float4(a0.re, a0.im, a1.re, a1.im);
      }
    }
    for (; v < items; v += G) {
      const float4 A = w[v];
      Cx<float> a0 = cmake(A.x, A.y), a1 = cmake(A.z, A.w);
      apply2<float, MK_GENERAL>(M, a0, a1);
      w[v] = make_float4(a0.re, a0.im, a1.re, a1.im);
    }
    return;
  }
  const uint64_t items = 1ull << (n - 2), st = 1ull << q;
  for (; v + (FWD_UNR - 1) * G < items; v += FWD_UNR * G) {
    uint64_t i0[FWD_UNR];
    float4 A[FWD_UNR], B[FWD_UNR];
#pragma unroll
    for (int u = 0; u < FWD_UNR; ++u) {
      i0[u] = insert0(2 * (v + u * G), q);
      A[u] = *reinterpret_cast<const float4*>(s + i0[u]);
      B[u] = *reinterpret_cast<const float4*>(s + (i0[u] | st));
    }
#pragma unroll
    for (int u = 0; u < FWD_UNR; ++u) {
      rot_v(M, A[u], B[u]);
      *reinterpret_cast<float4*>(s + i0[u]) = A[u];
      *reinterpret_cast<float4*>(s + (i0[u] | st)) = B[u];
    }
  }
  for (; v < items; v += G) {
    const uint64_t i0 = insert0(2 * v, q);
    float4 A = *reinterpret_cast<const float4*>(s + i0), B = *reinterpret_cast<const float4*>(s + (i0 | st));
    rot_v(M, A, B);
    *reinterpret_cast<float4*>(s + i0) = A;
    *reinterpret_cast<float4*>(s + (i0 | st)) = B;
  }
}

// CNOT ring CNOT(0,1) .. CNOT(n-2,n-1), CNOT(n-1,0) as a basis permutation
// j -> A(j): A(j)_k = j_0 ^ .. ^ j_k for k >= 1 and A(j)_0 = j_1 ^ .. ^ j_{n-1}.
__device__ __forceinline__ uint64_t ring_fwd(uint64_t x, int n) {
  const uint64_t mask = (n >= 64) ? ~0ull : ((1ull << n) - 1ull);
  uint64_t p = x;
  p ^= (p << 1) & mask;
  p ^= (p << 2) & mask;
  p ^= (p << 4) & mask;
  p ^= (p << 8) & mask;
  p ^= (p << 16) & mask;
  p ^= (p << 32) & mask;
  const uint64_t top = (p >> (n - 1)) & 1ull;
  return (p & ~1ull) | (top ^ (x & 1ull));
}
// inverse: x_k = y_k ^ y_{k-1} (k >= 1), x_0 = y_0, then bits 0 and 1 take y_{n-1}
__device__ __forceinline__ uint64_t ring_inv(uint64_t y, int n) {
  const uint64_t mask = (n >= 64) ? ~0ull : ((1ull << n) - 1ull);
  uint64_t x = (y ^ (y << 1)) & mask;
  if ((y >> (n - 1)) & 1ull) x ^= 3ull;
  return x;
}

// out[j] = in[src(j)] for every batch element; forward: the ring maps
// psi'[A(x)] = psi[x], so out[y] = in[A^{-1}(y)]; inverse: out[x] = in[A(x)].
template <typename R>
__global__ void __launch_bounds__(ADJ_T) k_ring(const typename CT<R>::V2* __restrict__ in,
                                                typename CT<R>::V2* __restrict__ out, int n, int inverse) {
  const int b = blockIdx.y;
  const typename CT<R>::V2* s = in + ((uint64_t)b << n);
  typename CT<R>::V2* d = out + ((uint64_t)b << n);
  const uint64_t N = 1ull << n;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (uint64_t)gridDim.x * blockDim.x)
    d[j] = s[inverse ? ring_fwd(j, n) : ring_inv(j, n)];
}

template <typename R>
__global__ void k_zero_state_batch(typename CT<R>::V2* __restrict__ psi, int n, int B) {
  const uint64_t N = 1ull << n, tot = N * (uint64_t)B;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (uint64_t)gridDim.x * blockDim.x)
    psi[i] = CT<R>::make((R)((i & (N - 1)) == 0 ? 1 : 0), (R)0);
}

// Sum partial[b][0..gx) in order into out[b * ostride + ooff].
__global__ void k_final_batch(const double* __restrict__ part, int gx, double* __restrict__ out, int64_t ostride,
                              int64_t ooff) {
  const int b = blockIdx.x;
  double t = 0.0;
  for (int i = threadIdx.x; i < gx; i += blockDim.x) t += part[(int64_t)b * gx + i];
  t = block_reduce(t);
  if (threadIdx.x == 0) out[(int64_t)b * ostride + ooff] = t;
}

// ------------------------------------------------------------ backward ---
// One gate: accumulate Im <lam|P|psi> (rotations), apply U^dagger to both.
template <typename R>
__global__ void __launch_bounds__(ADJ_T) k_bwd_gate(typename CT<R>::V2* __restrict__ psi,
                                                    typename CT<R>::V2* __restrict__ lam, int n, GateDev g,
                                                    const double* __restrict__ theta, int64_t stride,
                                                    double* __restrict__ part) {
  using IO = AmpIO<R>;
  const int b = blockIdx.y;
  typename CT<R>::V2* s = psi + ((uint64_t)b << n);
  typename CT<R>::V2* l = lam + ((uint64_t)b << n);
  const bool rot = g.kind <= QC_G_RZ;
  const double th = rot ? -theta[(int64_t)b * stride + g.param] : 0.0;  // U^dagger
  const Mat2<R> U = block_matrix<R>(g.kind, th);
  const uint64_t np = (g.kind == QC_G_CNOT) ? (1ull << (n - 2)) : (1ull << (n - 1));
  Acc<R> acc;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t i1;
    const uint64_t i0 = gate_pair(g, p, i1);
    Cx<R> p0 = IO::ld(s + i0), p1 = IO::ld(s + i1);
    Cx<R> l0 = IO::ld(l + i0), l1 = IO::ld(l + i1);
    if (rot) acc_generator<R>(acc, g.kind, p0, p1, l0, l1);
    apply_any<R>(g.kind, U, p0, p1);
    apply_any<R>(g.kind, U, l0, l1);
    IO::st(s + i0, p0);
    IO::st(s + i1, p1);
    IO::st(l + i0, l0);
    IO::st(l + i1, l1);
  }
  if (rot) {
    acc.flush();
    const double t = block_reduce(acc.value());
    if (threadIdx.x == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = t;
  }
}

// Two rotations ga then gb (forward order) on one qubit, walked backwards:
// gradient of gb, undo gb, gradient of ga, undo ga -- one pass.
template <typename R>
__global__ void __launch_bounds__(ADJ_T) k_bwd_rot2(typename CT<R>::V2* __restrict__ psi,
                                                    typename CT<R>::V2* __restrict__ lam, int n, GateDev ga,
                                                    GateDev gb, const double* __restrict__ theta, int64_t stride,
                                                    double* __restrict__ part_a, double* __restrict__ part_b) {
  using IO = AmpIO<R>;
  const int b = blockIdx.y;
  typename CT<R>::V2* s = psi + ((uint64_t)b << n);
  typename CT<R>::V2* l = lam + ((uint64_t)b << n);
  const Mat2<R> Ua = block_matrix<R>(ga.kind, -theta[(int64_t)b * stride + ga.param]);
  const Mat2<R> Ub = block_matrix<R>(gb.kind, -theta[(int64_t)b * stride + gb.param]);
  const int q = ga.q0;
  const uint64_t np = 1ull << (n - 1);
  Acc<R> acca, accb;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = insert0(p, q), i1 = i0 | (1ull << q);
    Cx<R> p0 = IO::ld(s + i0), p1 = IO::ld(s + i1);
    Cx<R> l0 = IO::ld(l + i0), l1 = IO::ld(l + i1);
    acc_generator<R>(accb, gb.kind, p0, p1, l0, l1);
    apply_any<R>(gb.kind, Ub, p0, p1);
    apply_any<R>(gb.kind, Ub, l0, l1);
    acc_generator<R>(acca, ga.kind, p0, p1, l0, l1);
    apply_any<R>(ga.kind, Ua, p0, p1);
    apply_any<R>(ga.kind, Ua, l0, l1);
    IO::st(s + i0, p0);
    IO::st(s + i1, p1);
    IO::st(l + i0, l0);
    IO::st(l + i1, l1);
  }
  acca.flush();
  accb.flush();
  const double ta = block_reduce(acca.value());
  const double tb = block_reduce(accb.value());
  if (threadIdx.x == 0) {
    part_a[(int64_t)b * gridDim.x + blockIdx.x] = ta;
    part_b[(int64_t)b * gridDim.x + blockIdx.x] = tb;
  }
}

// lam = H psi = sum_k c_k P_k psi, P_k = i^{|x&z|} X^x Z^z:
// (P psi)[j] = i^{|x&z|} (-1)^{|(j^x)&z|} psi[j^x].
struct TermsDev {
  int nt;
  uint64_t x[64], z[64];
  double c[64];
};

template <typename R>
__global__ void __launch_bounds__(ADJ_T) k_apply_h(const typename CT<R>::V2* __restrict__ psi,
                                                   typename CT<R>::V2* __restrict__ lam, int n,
                                                   const TermsDev* __restrict__ T) {
  const int b = blockIdx.y;
  const typename CT<R>::V2* s = psi + ((uint64_t)b << n);
  typename CT<R>::V2* l = lam + ((uint64_t)b << n);
  const uint64_t N = 1ull << n;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (uint64_t)gridDim.x * blockDim.x) {
    R ar = 0, ai = 0;
    for (int k = 0; k < T->nt; ++k) {
      const uint64_t x = T->x[k], z = T->z[k];
      const auto v = s[j ^ x];
      R vr = v.x, vi = v.y;
      if (__popcll((j ^ x) & z) & 1) {
        vr = -vr;
        vi = -vi;
      }
      const int ny = __popcll(x & z) & 3;
      R wr = vr, wi = vi;  // times i^ny
      if (ny == 1) { wr = -vi; wi = vr; }
      else if (ny == 2) { wr = -vr; wi = -vi; }
      else if (ny == 3) { wr = vi; wi = -vr; }
      const R c = (R)T->c[k];
      ar = fma(c, wr, ar);
      ai = fma(c, wi, ai);
    }
    l[j] = CT<R>::make(ar, ai);
  }
}

// Re <psi|lam> per batch element (block partials).
template <typename R>
__global__ void __launch_bounds__(ADJ_T) k_energy(const typename CT<R>::V2* __restrict__ psi,
                                                  const typename CT<R>::V2* __restrict__ lam, int n,
                                                  double* __restrict__ part) {
  const int b = blockIdx.y;
  const typename CT<R>::V2* s = psi + ((uint64_t)b << n);
  const typename CT<R>::V2* l = lam + ((uint64_t)b << n);
  const uint64_t N = 1ull << n;
  Acc<R> acc;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (uint64_t)gridDim.x * blockDim.x) {
    const auto v = s[j], w = l[j];
    acc.add(v.x, w.x);
    acc.add(v.y, w.y);
  }
  acc.flush();
  const double t = block_reduce(acc.value());
  if (threadIdx.x == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = t;
}

// ------------------------------------------------------------ host side --
enum AdjOpKind { AOP_GATE = 0, AOP_ROT2 = 1, AOP_RING = 2 };
struct AdjOp {
  int kind;
  GateDev a, b;
};

static GateDev gdev(const qc_gate& g) { return GateDev{g.kind, g.q0, g.q1, g.param}; }

// Compile the gate list into passes (see the file comment).
static std::vector<AdjOp> compile_ops(const qc_gate* gates, int ng, int n) {
  std::vector<AdjOp> ops;
  int i = 0;
  while (i < ng) {
    bool ring = (i + n <= ng) && n >= 2;
    for (int k = 0; ring && k < n; ++k)
      ring = gates[i + k].kind == QC_G_CNOT && gates[i + k].q0 == k && gates[i + k].q1 == (k + 1) % n;
    if (ring) {
      ops.push_back(AdjOp{AOP_RING, GateDev{QC_G_CNOT, 0, 1, 0}, GateDev{QC_G_CNOT, 0, 1, 0}});
      i += n;
      continue;
    }
    if (i + 1 < ng && gates[i].kind <= QC_G_RZ && gates[i + 1].kind <= QC_G_RZ && gates[i].q0 == gates[i + 1].q0) {
      ops.push_back(AdjOp{AOP_ROT2, gdev(gates[i]), gdev(gates[i + 1])});
      i += 2;
      continue;
    }
    ops.push_back(AdjOp{AOP_GATE, gdev(gates[i]), gdev(gates[i])});
    ++i;
  }
  return ops;
}

static qc_status check_circuit(int n, qc_dtype dt, int B, const qc_gate* gates, int n_gates, int64_t stride,
                               int n_params) {
  if (n < 2 || n > 30) {
    set_error("n = %d out of range [2, 30]", n);
    return QC_EINVAL;
  }
  if (dt != QC_C128 && dt != QC_C64) {
    set_error("unknown dtype %d", (int)dt);
    return QC_EINVAL;
  }
  if (B < 1 || B > 65535) {
    set_error("batch B = %d out of range [1, 65535]", B);
    return QC_EINVAL;
  }
  if (n_gates < 0 || (n_gates > 0 && !gates)) {
    set_error("bad gate list");
    return QC_EINVAL;
  }
  for (int i = 0; i < n_gates; ++i) {
    const qc_gate& g = gates[i];
    if (g.kind < QC_G_RX || g.kind > QC_G_H || g.q0 < 0 || g.q0 >= n) {
      set_error("gate %d: bad kind %d or qubit %d", i, g.kind, g.q0);
      return QC_EINVAL;
    }
    if (g.kind == QC_G_CNOT && (g.q1 < 0 || g.q1 >= n || g.q1 == g.q0)) {
      set_error("gate %d: bad CNOT target %d", i, g.q1);
      return QC_EINVAL;
    }
    if (g.kind <= QC_G_RZ && (g.param < 0 || g.param >= stride || (n_params > 0 && g.param >= n_params))) {
      set_error("gate %d: parameter index %d out of range", i, g.param);
      return QC_EINVAL;
    }
  }
  return QC_OK;
}

// Blocks per batch element: all blocks of the (gx, B) grid resident at once.
template <typename R>
static unsigned gx_for(int n, int B) {
  const uint64_t pairs = 1ull << (n - 1);
  uint64_t gx = (pairs + ADJ_T - 1) / ADJ_T;
  const int res = std::min(resident_blocks((const void*)k_bwd_rot2<R>, ADJ_T, 0),
                           resident_blocks((const void*)k_fwd_gate<R>, ADJ_T, 0));
  const uint64_t cap = std::max<uint64_t>(1, (uint64_t)sm_count() * res / (uint64_t)B);
  gx = std::min<uint64_t>(gx, std::min<uint64_t>(cap, ADJ_GX_MAX));
  return (unsigned)std::max<uint64_t>(gx, 1);
}

// Buffers rotate among the caller's psi and lam and one workspace.
template <typename R>
struct Bufs {
  typename CT<R>::V2* psi;
  typename CT<R>::V2* lam;
  typename CT<R>::V2* spare;
};

// Forward passes; the result is in bufs.psi (which may be the workspace).
template <typename R>
static int forward_passes(const std::vector<AdjOp>& ops, int n, int B, const double* theta, int64_t stride,
                          Bufs<R>& bf, cudaStream_t st) {
  const dim3 grid(gx_for<R>(n, B), B);
  // complex64 rotation pairs: three blocks per SM over the whole batch
  const uint64_t vitems = n >= 2 ? (1ull << (n - 2)) : 1ull;
  const unsigned gxv = (unsigned)std::max<uint64_t>(
      1, std::min<uint64_t>((vitems + FWD_UNR * ADJ_T - 1) / (FWD_UNR * ADJ_T), 3ull * sm_count() / (uint64_t)B));
  const uint64_t tot = (uint64_t)B << n;
  k_zero_state_batch<R><<<grid_for(tot, ADJ_T, 8), ADJ_T, 0, st>>>(bf.psi, n, B);
  int nk = 1;
  for (const AdjOp& op : ops) {
    if (op.kind == AOP_RING) {
      k_ring<R><<<grid, ADJ_T, 0, st>>>(bf.psi, bf.spare, n, 0);
      std::swap(bf.psi, bf.spare);
    } else if (op.kind == AOP_ROT2) {
      if constexpr (sizeof(R) == 4) {
        if (n >= 2) {
          k_fwd_rot2_c64<<<dim3(gxv, B), ADJ_T, 0, st>>>(reinterpret_cast<float2*>(bf.psi), n, op.a, op.b, theta,
                                                         stride);
          ++nk;
          continue;
        }
      }
      k_fwd_rot2<R><<<grid, ADJ_T, 0, st>>>(bf.psi, n, op.a, op.b, theta, stride);
    } else {
      k_fwd_gate<R><<<grid, ADJ_T, 0, st>>>(bf.psi, n, op.a, theta, stride);
    }
    ++nk;
  }
  return nk;
}

static bool has_ring(const std::vector<AdjOp>& ops) {
  for (const AdjOp& o : ops)
    if (o.kind == AOP_RING) return true;
  return false;
}

template <typename R>
static qc_status forward_impl(int n, int B, const qc_gate* gates, int n_gates, const double* theta,
                              int64_t stride, void* psi, cudaStream_t st) {
  using V2 = typename CT<R>::V2;
  const std::vector<AdjOp> ops = compile_ops(gates, n_gates, n);
  const size_t bytes = ((size_t)B << n) * sizeof(V2);
  V2* ws = nullptr;
  if (has_ring(ops)) {
    cudaError_t e = cudaMallocAsync((void**)&ws, bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "forward workspace");
  }
  Bufs<R> bf{reinterpret_cast<V2*>(psi), nullptr, ws};
  int nk = forward_passes<R>(ops, n, B, theta, stride, bf, st);
  if (bf.psi != reinterpret_cast<V2*>(psi)) {
    cudaMemcpyAsync(psi, bf.psi, bytes, cudaMemcpyDeviceToDevice, st);
  }
  if (ws) cudaFreeAsync(ws, st);
  return check_launch("circuit forward", nk);
}

template <typename R>
static qc_status adjoint_impl(int n, int B, const qc_gate* gates, int n_gates, const double* theta,
                              int64_t stride, const qc_pauli_term* H, int n_terms, void* psi, void* lam,
                              double* energy, double* grad, cudaStream_t st) {
  using V2 = typename CT<R>::V2;
  const std::vector<AdjOp> ops = compile_ops(gates, n_gates, n);
  const size_t bytes = ((size_t)B << n) * sizeof(V2);
  const unsigned gx = gx_for<R>(n, B);
  const dim3 grid(gx, B);
  // workspace: Hamiltonian terms, two partial arrays, one state buffer
  TermsDev* dT = nullptr;
  double* part = nullptr;
  V2* ws = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&dT, sizeof(TermsDev), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&part, sizeof(double) * 2 * (size_t)gx * B, st);
  if (e == cudaSuccess && has_ring(ops)) e = cudaMallocAsync((void**)&ws, bytes, st);
  TermsDev* hT = nullptr;
  if (e == cudaSuccess) e = cudaMallocHost((void**)&hT, sizeof(TermsDev));
  if (e != cudaSuccess) {
    if (dT) cudaFreeAsync(dT, st);
    if (part) cudaFreeAsync(part, st);
    if (ws) cudaFreeAsync(ws, st);
    return cuda_fail(e, "adjoint workspace");
  }
  double* part_b = part + (size_t)gx * B;
  hT->nt = n_terms;
  for (int k = 0; k < n_terms; ++k) {
    hT->x[k] = H[k].xmask;
    hT->z[k] = H[k].zmask;
    hT->c[k] = H[k].coeff;
  }
  e = cudaMemcpyAsync(dT, hT, sizeof(TermsDev), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)B * stride, st);
  qc_status s = QC_OK;
  if (e != cudaSuccess) s = cuda_fail(e, "adjoint setup");
  if (!s) {
    Bufs<R> bf{reinterpret_cast<V2*>(psi), reinterpret_cast<V2*>(lam), ws};
    // the forward pass may rotate psi into the workspace; lam stays put
    Bufs<R> fb{bf.psi, nullptr, bf.spare};
    int nk = forward_passes<R>(ops, n, B, theta, stride, fb, st);
    bf.psi = fb.psi;
    bf.spare = fb.spare;
    k_apply_h<R><<<grid, ADJ_T, 0, st>>>(bf.psi, bf.lam, n, dT);
    k_energy<R><<<grid, ADJ_T, 0, st>>>(bf.psi, bf.lam, n, part);
    k_final_batch<<<B, ADJ_T, 0, st>>>(part, gx, energy, 1, 0);
    nk += 3;
    for (int i = (int)ops.size() - 1; i >= 0; --i) {
      const AdjOp& op = ops[i];
      if (op.kind == AOP_RING) {
        k_ring<R><<<grid, ADJ_T, 0, st>>>(bf.psi, bf.spare, n, 1);
        std::swap(bf.psi, bf.spare);
        k_ring<R><<<grid, ADJ_T, 0, st>>>(bf.lam, bf.spare, n, 1);
        std::swap(bf.lam, bf.spare);
        nk += 2;
      } else if (op.kind == AOP_ROT2) {
        k_bwd_rot2<R><<<grid, ADJ_T, 0, st>>>(bf.psi, bf.lam, n, op.a, op.b, theta, stride, part, part_b);
        k_final_batch<<<B, ADJ_T, 0, st>>>(part_b, gx, grad, stride, op.b.param);
        k_final_batch<<<B, ADJ_T, 0, st>>>(part, gx, grad, stride, op.a.param);
        nk += 3;
      } else {
        k_bwd_gate<R><<<grid, ADJ_T, 0, st>>>(bf.psi, bf.lam, n, op.a, theta, stride, part);
        ++nk;
        if (op.a.kind <= QC_G_RZ) {
          k_final_batch<<<B, ADJ_T, 0, st>>>(part, gx, grad, stride, op.a.param);
          ++nk;
        }
      }
    }
    s = check_launch("adjoint", nk);
  }
  e = cudaStreamSynchronize(st);  // the pinned term list is freed below
  cudaFreeHost(hT);
  cudaFreeAsync(dT, st);
  cudaFreeAsync(part, st);
  if (ws) cudaFreeAsync(ws, st);
  if (!s && e != cudaSuccess) s = cuda_fail(e, "adjoint");
  return s;
}

static qc_status check_param_once(const qc_gate* gates, int n_gates) {
  // each angle may drive at most one gate (the gradient slot is written,
  // not accumulated)
  std::vector<int> seen;
  for (int i = 0; i < n_gates; ++i)
    if (gates[i].kind <= QC_G_RZ) seen.push_back(gates[i].param);
  std::sort(seen.begin(), seen.end());
  for (size_t i = 1; i < seen.size(); ++i)
    if (seen[i] == seen[i - 1]) {
      set_error("parameter %d drives more than one gate", seen[i]);
      return QC_EINVAL;
    }
  return QC_OK;
}

}  // namespace qc

using namespace qc;

QC_API qc_status qc_circuit_forward(int n, qc_dtype dt, int B, const qc_gate* gates, int n_gates,
                                    const double* theta_dev, int64_t theta_stride, void* psi_dev, void* stream) {
  clear_error();
  qc_status s = check_circuit(n, dt, B, gates, n_gates, theta_stride, 0);
  if (s) return s;
  if (!psi_dev || (!theta_dev && n_gates > 0)) {
    set_error("NULL device buffer");
    return QC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return dt == QC_C128 ? forward_impl<double>(n, B, gates, n_gates, theta_dev, theta_stride, psi_dev, st)
                       : forward_impl<float>(n, B, gates, n_gates, theta_dev, theta_stride, psi_dev, st);
}

QC_API qc_status qc_adjoint_grad(int n, qc_dtype dt, int B, const qc_gate* gates, int n_gates,
                                 const double* theta_dev, int64_t theta_stride, int n_params,
                                 const qc_pauli_term* H, int n_terms, void* psi_dev, void* lam_dev,
                                 double* energy_dev, double* grad_dev, void* stream) {
  clear_error();
  qc_status s = check_circuit(n, dt, B, gates, n_gates, theta_stride, n_params);
  if (!s) s = check_param_once(gates, n_gates);
  if (s) return s;
  if (n_params < 0 || n_params > theta_stride) {
    set_error("n_params = %d out of range [0, theta_stride]", n_params);
    return QC_EINVAL;
  }
  if (!H || n_terms < 1 || n_terms > 64) {
    set_error("need 1..64 Hamiltonian terms");
    return QC_EINVAL;
  }
  for (int k = 0; k < n_terms; ++k)
    if ((n < 64 && ((H[k].xmask | H[k].zmask) >> n)) || !std::isfinite(H[k].coeff)) {
      set_error("Hamiltonian term %d has bits at or above n or a non-finite coefficient", k);
      return QC_EINVAL;
    }
  if (!psi_dev || !lam_dev || !energy_dev || !grad_dev || (!theta_dev && n_gates > 0)) {
    set_error("NULL device buffer");
    return QC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return dt == QC_C128 ? adjoint_impl<double>(n, B, gates, n_gates, theta_dev, theta_stride, H, n_terms,
                                              psi_dev, lam_dev, energy_dev, grad_dev, st)
                       : adjoint_impl<float>(n, B, gates, n_gates, theta_dev, theta_stride, H, n_terms,
                                             psi_dev, lam_dev, energy_dev, grad_dev, st);
}
