// Single-gate kernels: one-qubit operators (OneOpA, Eq. resmat1),
// controlled operators / CNOT / CPHASEK (Eq. resmat2, Eq. cphasek) and SWAP,
// plus state fills.  Each is one streaming read+write pass over the
// amplitudes the gate touches, with 128-bit loads and stores and
// grid-stride loops sized to the resident blocks.
//
// complex64 operators compute in FP32.  complex128 operators with real
// arithmetic (general, real, diagonal, anti-diagonal, Hadamard) split their
// products between the FP64 pipe (a few operations per pair) and
// double-float on the FP32 pipe (ff.cuh): on GB300 the FP64 pipe does 0.5
// Top/s, fewer than 2.5 FP64 operations per amplitude in the time one HBM
// pass takes at 30 qubits.  Exchanges (X, CNOT, SWAP) and the phases -1, +i,
// -i are exact moves and sign flips; other phases use one FP64 complex
// multiply on the touched quarter.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace qc {

// Operator as passed to the gate kernels: the native matrix, and for
// complex128 its double-float split.
template <typename R> struct GateArg;
template <> struct GateArg<float> {
  Mat2<float> U;
};
template <> struct GateArg<double> {
  Mat2<double> U;
  Mat2ff F;
};

// complex128 operators with products on both pipes: 4 FP64 operations per
// pair (GB300's FP64 pipe completes about 6 per pair in the time a 30-qubit
// read+write pass takes at 0.8 of HBM), the rest in double-float on the FP32
// pipe.  The FP64 part is one output component (general: Re b0) or the
// real parts (real operators) or one output (diagonal, anti-diagonal).
// The real part of the first output on the FP64 pipe, the other three as
// four-term double-float dots, with the integer-lean conversions (the kernel
// is bound by issue, not by memory).
__device__ __forceinline__ void apply_general_c128(const GateArg<double>& G, Cx<double>& a0, Cx<double>& a1) {
  const Mat2<double>& U = G.U;
  double r0 = U.m[0].re * a0.re;
  r0 = fma(-U.m[0].im, a0.im, r0);
  r0 = fma(U.m[1].re, a1.re, r0);
  r0 = fma(-U.m[1].im, a1.im, r0);
  const ff x0r = ff_from_d_fast(a0.re), x0i = ff_from_d_fast(a0.im);
  const ff x1r = ff_from_d_fast(a1.re), x1i = ff_from_d_fast(a1.im);
  const Mat2ff& F = G.F;
  const ff i0 = ff_dot4(F.m[0].re, x0i, F.m[0].im, x0r, F.m[1].re, x1i, F.m[1].im, x1r);
  const ff r1 = ff_dot4(F.m[2].re, x0r, ff_neg(F.m[2].im), x0i, F.m[3].re, x1r, ff_neg(F.m[3].im), x1i);
  const ff i1 = ff_dot4(F.m[2].re, x0i, F.m[2].im, x0r, F.m[3].re, x1i, F.m[3].im, x1r);
  a0 = cmake<double>(r0, ff_to_d_fast(i0));
  a1 = cmake<double>(ff_to_d_fast(r1), ff_to_d_fast(i1));
}
__device__ __forceinline__ void apply_real_c128(const GateArg<double>& G, Cx<double>& a0, Cx<double>& a1) {
  const double u00 = G.U.m[0].re, u01 = G.U.m[1].re, u10 = G.U.m[2].re, u11 = G.U.m[3].re;
  const double r0 = fma(u01, a1.re, u00 * a0.re), r1 = fma(u11, a1.re, u10 * a0.re);
  const ff x0i = ff_from_d(a0.im), x1i = ff_from_d(a1.im);
  const Mat2ff& F = G.F;
  const ff i0 = ff_dot2p(F.m[0].re, x0i, F.m[1].re, x1i), i1 = ff_dot2p(F.m[2].re, x0i, F.m[3].re, x1i);
  a0 = cmake<double>(r0, ff_to_d(i0));
  a1 = cmake<double>(r1, ff_to_d(i1));
}
// one complex product in FP64 (u a), the other in double-float
__device__ __forceinline__ Cx<double> cmul_fp64(Cx<double> u, Cx<double> a) {
  return cmake<double>(fma(-u.im, a.im, u.re * a.re), fma(u.im, a.re, u.re * a.im));
}
__device__ __forceinline__ Cx<double> cmul_ffd(const ffc& u, Cx<double> a) {
  const ffc z = ffc_mul(u, ffc_from_d(a.re, a.im));
  return cmake<double>(ff_to_d(z.re), ff_to_d(z.im));
}

template <typename R, int KIND>
__device__ __forceinline__ void apply_gate(const GateArg<R>& G, Cx<R>& a0, Cx<R>& a1) {
  if constexpr (sizeof(R) == 8 && KIND == MK_GENERAL) {
    apply_general_c128(G, a0, a1);
  } else if constexpr (sizeof(R) == 8 && KIND == MK_REAL) {
    apply_real_c128(G, a0, a1);
  } else if constexpr (sizeof(R) == 8 && KIND == MK_DIAG) {
    a0 = cmul_fp64(G.U.m[0], a0);
    a1 = cmul_ffd(G.F.m[3], a1);
  } else if constexpr (sizeof(R) == 8 && KIND == MK_ANTI) {
    const Cx<double> b0 = cmul_fp64(G.U.m[1], a1);
    a1 = cmul_ffd(G.F.m[2], a0);
    a0 = b0;
  } else if constexpr (sizeof(R) == 8 && KIND == MK_HAD) {
    // both pipes: real parts in FP64 (1.5 FP64 operations per amplitude),
    // imaginary parts in double-float on the FP32 pipe
    const double h = G.U.m[0].re;
    const double q = h * a1.re;
    const double r0 = fma(h, a0.re, q), r1 = fma(h, a0.re, -q);
    const ff x0 = ff_from_d(a0.im), x1 = ff_from_d(a1.im), hf = G.F.m[0].re;
    a0 = cmake<R>(r0, ff_to_d(ff_mul(ff_add(x0, x1), hf)));
    a1 = cmake<R>(r1, ff_to_d(ff_mul(ff_sub(x0, x1), hf)));
  } else if constexpr (sizeof(R) == 8 && uses_ff(KIND)) {
    ffc b0 = ffc_from_d(a0.re, a0.im), b1 = ffc_from_d(a1.re, a1.im);
    apply2_ff<KIND>(G.F, b0, b1);
    a0 = cmake<R>(ff_to_d(b0.re), ff_to_d(b0.im));
    a1 = cmake<R>(ff_to_d(b1.re), ff_to_d(b1.im));
  } else {
    apply2<R, KIND>(G.U, a0, a1);
  }
}

// Enumeration of the pairs a gate updates.  Pair p maps to index i0 by
// inserting zero bits at positions p0 < p1 (NINS = 1 or 2) and or-ing in
// `setm` (the control bit); its partner is i1 = i0 | 2^t.
template <int NINS>
__device__ __forceinline__ uint64_t pair_base(uint64_t p, int p0, int p1, uint64_t setm) {
  uint64_t i = insert0(p, p0);
  if (NINS == 2) i = insert0(i, p1);
  return i | setm;
}

// Scalar form: one pair per work item, 16-byte (c128) or 8-byte (c64)
// accesses.  UNR items are processed per loop trip so that 2 UNR loads are
// in flight before the first use (4 for complex128).  The register budget
// of four blocks per SM is declared: with it the complex128 exchange (CNOT)
// streams at 0.93-0.95 of copy bandwidth on GB300, without it at 0.82-0.86
// (same register count, different schedule).
// Register budget: four blocks per SM (64 registers), except the complex128
// diagonal and anti-diagonal kinds, whose products are split between FP64
// and double-float and which declare three (85 registers) -- the launcher
// runs three per SM for complex128 anyway, and under 64 registers they spill
// 100+ bytes.
// complex128 general operator: two pairs per loop trip on four blocks per SM
// (issue bound: more warps, fewer registers).  With the integer-lean
// conversions, measured on one box at 30 qubits: 5.90 ms per gate, 0.859 of
// the measured copy bandwidth, against 7.27 ms (0.697) with four pairs on
// three blocks and the general conversions; with four pairs on three blocks
// and the lean conversions 7.11 ms.
// complex128 Hadamard and exchange: eight pairs per loop trip (sixteen
// 16-byte loads in flight per thread) on two blocks per SM.  Measured on one
// box against four pairs on three blocks: H 5.455 against 5.53 ms, CNOT
// 2.884 against 2.899 ms at 30 qubits; the phase kinds, which read only the
// bit-1 half, ran slower that way (1.631 against 1.602 ms) and keep four.
template <int KIND>
struct PairWide {
  static constexpr bool value = KIND == MK_HAD || KIND == MK_SWAPX;
};
template <typename R, int KIND>
struct PairUnroll {
  static constexpr int value =
      sizeof(R) == 8 ? (PairWide<KIND>::value ? 8 : (KIND == MK_GENERAL ? 2 : 4)) : 2;
};
template <typename R, int KIND>
struct PairBlocks {
  static constexpr int value =
      (sizeof(R) == 8 && PairWide<KIND>::value) ? 2 :
      (sizeof(R) == 8 && (KIND == MK_DIAG || KIND == MK_ANTI)) ? 3 : 4;
};
template <typename R, int KIND, int NINS>
__global__ void __launch_bounds__(256, PairBlocks<R, KIND>::value)
    k_pairs(typename CT<R>::V2* __restrict__ s, uint64_t npairs, int p0, int p1, uint64_t setm, int t, GateArg<R> G) {
  using IO = AmpIO<R>;
  constexpr bool B1 = touches_bit1_only(KIND);
  constexpr int UNR = PairUnroll<R, KIND>::value;
  const uint64_t st = 1ull << t;
  const uint64_t GS = (uint64_t)gridDim.x * blockDim.x;
  uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; p + (UNR - 1) * GS < npairs; p += UNR * GS) {
    uint64_t i[UNR];
    Cx<R> a[UNR], b[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      i[u] = pair_base<NINS>(p + u * GS, p0, p1, setm);
      a[u] = B1 ? cmake<R>(0, 0) : IO::ld(s + i[u]);
      b[u] = IO::ld(s + (i[u] | st));
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      apply_gate<R, KIND>(G, a[u], b[u]);
      if (!B1) IO::st(s + i[u], a[u]);
      IO::st(s + (i[u] | st), b[u]);
    }
  }
  for (; p < npairs; p += GS) {
    const uint64_t i0 = pair_base<NINS>(p, p0, p1, setm);
    Cx<R> a0 = cmake<R>(0, 0);
    if (!B1) a0 = IO::ld(s + i0);
    Cx<R> a1 = IO::ld(s + (i0 | st));
    apply_gate<R, KIND>(G, a0, a1);
    if (!B1) IO::st(s + i0, a0);
    IO::st(s + (i0 | st), a1);
  }
}

// complex64, all inserted bit positions >= 1: two neighbouring pairs per
// work item share 16-byte loads (amplitudes i0, i0+1 and i1, i1+1).  Four
// items per loop trip (eight loads in flight per thread) on three blocks per
// SM: on GB300 the exchange (CNOT) then streams at 0.95-0.97 of copy
// bandwidth, against 0.77 with one item per trip at eight blocks.
constexpr int V2_UNR = 4;
template <int KIND>
__device__ __forceinline__ void apply_v2(const GateArg<float>& G, float4& A, float4& B) {
  Cx<float> a0 = cmake(A.x, A.y), c0 = cmake(A.z, A.w);
  Cx<float> a1 = cmake(B.x, B.y), c1 = cmake(B.z, B.w);
  apply2<float, KIND>(G.U, a0, a1);
  apply2<float, KIND>(G.U, c0, c1);
  A = make_float4(a0.re, a0.im, c0.re, c0.im);
  B = make_float4(a1.re, a1.im, c1.re, c1.im);
}
template <int KIND, int NINS>
__global__ void __launch_bounds__(256, 4) k_pairs_v2(float2* __restrict__ s, uint64_t nitems, int p0, int p1,
                                                     uint64_t setm, int t, GateArg<float> G) {
  constexpr bool B1 = touches_bit1_only(KIND);
  const uint64_t st = 1ull << t;
  const uint64_t GS = (uint64_t)gridDim.x * blockDim.x;
  uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; v + (V2_UNR - 1) * GS < nitems; v += V2_UNR * GS) {
    uint64_t i0[V2_UNR];
    float4 A[V2_UNR], B[V2_UNR];
#pragma unroll
    for (int u = 0; u < V2_UNR; ++u) {
      i0[u] = pair_base<NINS>(2 * (v + u * GS), p0, p1, setm);
      A[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!B1) A[u] = *reinterpret_cast<const float4*>(s + i0[u]);
      B[u] = *reinterpret_cast<const float4*>(s + (i0[u] | st));
    }
#pragma unroll
    for (int u = 0; u < V2_UNR; ++u) {
      apply_v2<KIND>(G, A[u], B[u]);
      if (!B1) *reinterpret_cast<float4*>(s + i0[u]) = A[u];
      *reinterpret_cast<float4*>(s + (i0[u] | st)) = B[u];
    }
  }
  for (; v < nitems; v += GS) {
    const uint64_t i0 = pair_base<NINS>(2 * v, p0, p1, setm);
    float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B;
    if (!B1) A = *reinterpret_cast<const float4*>(s + i0);
    B = *reinterpret_cast<const float4*>(s + (i0 | st));
    apply_v2<KIND>(G, A, B);
    if (!B1) *reinterpret_cast<float4*>(s + i0) = A;
    *reinterpret_cast<float4*>(s + (i0 | st)) = B;
  }
}

// complex64, one-qubit gate on t = 0: the pair (2q, 2q+1) is one 16-byte
// vector.
template <int KIND>
__global__ void __launch_bounds__(256) k_pairs_t0(float2* __restrict__ s, uint64_t npairs, GateArg<float> G) {
  const uint64_t GS = (uint64_t)gridDim.x * blockDim.x;
  float4* v4 = reinterpret_cast<float4*>(s);
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += GS) {
    float4 A = v4[p];
    Cx<float> a0 = cmake(A.x, A.y), a1 = cmake(A.z, A.w);
    apply2<float, KIND>(G.U, a0, a1);
    v4[p] = make_float4(a0.re, a0.im, a1.re, a1.im);
  }
}

template <typename R, int KIND>
static void launch_kind(qc_state* s, int nins, int p0, int p1, uint64_t setm, int t, const GateArg<R>& G) {
  using V2 = typename CT<R>::V2;
  const uint64_t npairs = (1ull << s->n) >> nins;
  V2* d = reinterpret_cast<V2*>(s->data);
  const int T = 256;
  if constexpr (sizeof(R) == 4) {
    if (nins == 1 && t == 0) {
      auto k = k_pairs_t0<KIND>;
      k<<<resident_grid(k, T, npairs, T), T, 0, s->stream>>>(d, npairs, G);
      return;
    }
    if (p0 >= 1 && npairs >= 2) {
      const uint64_t items = npairs / 2;
      auto k = (nins == 1) ? k_pairs_v2<KIND, 1> : k_pairs_v2<KIND, 2>;
      const unsigned g = std::min<unsigned>(resident_grid(k, T, items, V2_UNR * T), 3u * (unsigned)sm_count());
      k<<<g, T, 0, s->stream>>>(d, items, p0, p1, setm, t, G);
      return;
    }
  }
  auto k = (nins == 1) ? k_pairs<R, KIND, 1> : k_pairs<R, KIND, 2>;
  unsigned g = resident_grid(k, T, npairs, PairUnroll<R, KIND>::value * T);
  // complex128: three blocks per SM (24 warps, 96 16-byte loads in flight
  // per warp) stream best on GB300; a fourth adds DRAM contention (H: 0.92-
  // 0.95 of copy bandwidth with three, 0.89-0.91 with four).
  if (sizeof(R) == 8) g = std::min<unsigned>(g, (KIND == MK_GENERAL ? 4u : 3u) * (unsigned)sm_count());
  k<<<g, T, 0, s->stream>>>(d, npairs, p0, p1, setm, t, G);
}

template <typename R>
static GateArg<R> gate_arg(const double* Uh);
template <>
GateArg<float> gate_arg<float>(const double* Uh) {
  GateArg<float> G;
  G.U = mat_from_host<float>(Uh);
  return G;
}
template <>
GateArg<double> gate_arg<double>(const double* Uh) {
  GateArg<double> G;
  G.U = mat_from_host<double>(Uh);
  G.F = mat2ff_from_host(Uh);
  return G;
}

template <typename R>
static void launch_pairs(qc_state* s, int nins, int p0, int p1, uint64_t setm, int t, const double* Uh) {
  const GateArg<R> G = gate_arg<R>(Uh);
  switch (classify(Uh)) {
    case MK_IDENT: return;
    case MK_GENERAL: launch_kind<R, MK_GENERAL>(s, nins, p0, p1, setm, t, G); return;
    case MK_REAL: launch_kind<R, MK_REAL>(s, nins, p0, p1, setm, t, G); return;
    case MK_DIAG: launch_kind<R, MK_DIAG>(s, nins, p0, p1, setm, t, G); return;
    case MK_PHASE1: launch_kind<R, MK_PHASE1>(s, nins, p0, p1, setm, t, G); return;
    case MK_PH_NEG: launch_kind<R, MK_PH_NEG>(s, nins, p0, p1, setm, t, G); return;
    case MK_PH_I: launch_kind<R, MK_PH_I>(s, nins, p0, p1, setm, t, G); return;
    case MK_PH_MI: launch_kind<R, MK_PH_MI>(s, nins, p0, p1, setm, t, G); return;
    case MK_ANTI: launch_kind<R, MK_ANTI>(s, nins, p0, p1, setm, t, G); return;
    case MK_SWAPX: launch_kind<R, MK_SWAPX>(s, nins, p0, p1, setm, t, G); return;
    case MK_HAD: launch_kind<R, MK_HAD>(s, nins, p0, p1, setm, t, G); return;
  }
}

qc_status launch_1q(qc_state* s, int t, const double* U) {
  if (s->dt == QC_C128) launch_pairs<double>(s, 1, t, 0, 0, t, U);
  else launch_pairs<float>(s, 1, t, 0, 0, t, U);
  s->sum_valid = false;
  return check_launch("apply_1q", classify(U) == MK_IDENT ? 0 : 1);
}

qc_status launch_ctrl(qc_state* s, int c, int t, const double* U) {
  const int p0 = std::min(c, t), p1 = std::max(c, t);
  const uint64_t setm = 1ull << c;
  if (s->dt == QC_C128) launch_pairs<double>(s, 2, p0, p1, setm, t, U);
  else launch_pairs<float>(s, 2, p0, p1, setm, t, U);
  s->sum_valid = false;
  return check_launch("apply_ctrl", classify(U) == MK_IDENT ? 0 : 1);
}

// SWAP: amplitudes with (bit a, bit b) = (1, 0) and (0, 1) trade places.
template <typename V2>
__global__ void __launch_bounds__(256) k_swap(V2* __restrict__ s, uint64_t nq, int lo, int hi, int a, int b) {
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += G) {
    const uint64_t base = insert0(insert0(q, lo), hi);
    const uint64_t ia = base | (1ull << a), ib = base | (1ull << b);
    const V2 x = s[ia], y = s[ib];
    s[ia] = y;
    s[ib] = x;
  }
}

// complex64 with both bits >= 1: two neighbouring quartets per item.
__global__ void __launch_bounds__(256) k_swap_v2(float2* __restrict__ s, uint64_t nitems, int lo, int hi, int a, int b) {
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nitems; v += G) {
    const uint64_t base = insert0(insert0(2 * v, lo), hi);
    float4* pa = reinterpret_cast<float4*>(s + (base | (1ull << a)));
    float4* pb = reinterpret_cast<float4*>(s + (base | (1ull << b)));
    const float4 x = *pa, y = *pb;
    *pa = y;
    *pb = x;
  }
}

qc_status launch_swap(qc_state* s, int a, int b) {
  const int lo = std::min(a, b), hi = std::max(a, b);
  const uint64_t nq = (1ull << s->n) >> 2;
  const int T = 256;
  if (s->dt == QC_C128) {
    k_swap<double2><<<resident_grid(k_swap<double2>, T, nq, T), T, 0, s->stream>>>(
        reinterpret_cast<double2*>(s->data), nq, lo, hi, a, b);
  } else if (lo >= 1 && nq >= 2) {
    k_swap_v2<<<resident_grid(k_swap_v2, T, nq / 2, T), T, 0, s->stream>>>(reinterpret_cast<float2*>(s->data),
                                                                            nq / 2, lo, hi, a, b);
  } else {
    k_swap<float2><<<resident_grid(k_swap<float2>, T, nq, T), T, 0, s->stream>>>(
        reinterpret_cast<float2*>(s->data), nq, lo, hi, a, b);
  }
  s->sum_valid = false;
  return check_launch("swap");
}

// ------------------------------------------------------------ fills ------
// Every amplitude = v; the running sum N * v goes to the scratch.
template <typename V2>
__global__ void k_fill(V2* __restrict__ s, uint64_t N, V2 v, double* scratch) {
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) s[i] = v;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    scratch[QC_SCR_SUM] = (double)N * (double)v.x;
    scratch[QC_SCR_SUM + 1] = (double)N * (double)v.y;
  }
}
// Writes the single nonzero amplitude and records the running sum (1) in the
// state's scratch.
template <typename V2>
__global__ void k_set_one(V2* __restrict__ s, uint64_t idx, V2 v, double* scratch) {
  s[idx] = v;
  scratch[QC_SCR_SUM] = 1.0;
  scratch[QC_SCR_SUM + 1] = 0.0;
}

qc_status launch_fill_basis(qc_state* s, uint64_t idx) {
  const size_t bytes = ((size_t)1 << s->n) * amp_bytes(s->dt);
  cudaError_t e = cudaMemsetAsync(s->data, 0, bytes, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  if (s->dt == QC_C128)
    k_set_one<double2><<<1, 1, 0, s->stream>>>(reinterpret_cast<double2*>(s->data), idx,
                                               make_double2(1.0, 0.0), s->scratch);
  else
    k_set_one<float2><<<1, 1, 0, s->stream>>>(reinterpret_cast<float2*>(s->data), idx,
                                              make_float2(1.f, 0.f), s->scratch);
  s->sum_valid = true;
  return check_launch("fill_basis");
}

qc_status launch_fill_uniform(qc_state* s) {
  const uint64_t N = 1ull << s->n;
  const double a = 1.0 / sqrt(ldexp(1.0, s->n));  // 2^{-n/2}
  const int T = 256;
  if (s->dt == QC_C128)
    k_fill<double2><<<grid_for(N, T, 8), T, 0, s->stream>>>(reinterpret_cast<double2*>(s->data), N,
                                                            make_double2(a, 0.0), s->scratch);
  else
    k_fill<float2><<<grid_for(N, T, 8), T, 0, s->stream>>>(reinterpret_cast<float2*>(s->data), N,
                                                           make_float2((float)a, 0.f), s->scratch);
  qc_status st = check_launch("fill_uniform");
  s->sum_valid = (st == QC_OK);
  return st;
}

// Real scale of every amplitude.
template <typename R>
__global__ void k_scale(typename CT<R>::V2* __restrict__ s, uint64_t N, R f) {
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) {
    auto v = s[i];
    v.x *= f;
    v.y *= f;
    s[i] = v;
  }
}

qc_status launch_scale(qc_state* s, double f) {
  const uint64_t N = 1ull << s->n;
  const int T = 256;
  if (s->dt == QC_C128)
    k_scale<double><<<grid_for(N, T, 8), T, 0, s->stream>>>(reinterpret_cast<double2*>(s->data), N, f);
  else
    k_scale<float><<<grid_for(N, T, 8), T, 0, s->stream>>>(reinterpret_cast<float2*>(s->data), N, (float)f);
  s->sum_valid = false;
  return check_launch("scale");
}

}  // namespace qc
