// Fused shared-memory tile passes.
//
// One-qubit operators on distinct pairs are independent (sec. 3, after
// Eq. resmat1), and operators on different qubits commute, so every gate
// acting on a contiguous group of qubits [lo, lo+k) can be applied in one
// pass: a CTA stages a tile -- all 2^k values of the group bits, times the
// 2^c lowest index bits kept contiguous for 128-byte rows -- in shared
// memory, applies the group's gates there, and writes the tile back.
// HALL (Eq. HALL) and layers of one-qubit operators take a few passes
// instead of n.  Hadamards are applied as unnormalised butterflies
// (a0 + a1, a0 - a1) and the pass multiplies by 2^{-p/2} once at the end.
//
// The QFT circuit of Appendix A processes qubits from the most significant
// down: Hadamard on t, then CPHASEK(t, t') for every lower t' with phase
// e^{2 pi i / 2^{t-t'+1}}.  For a group [lo, hi] the phases with t' inside
// the group are applied right after the group's Hadamard on t (a diagonal
// "ladder" e^{2 pi i x / 2^{j+1}}, x = group bits below group qubit j);
// those with t' < lo commute with the rest of the group's gates and are
// applied at the end of the pass as one twiddle factor
//   Omega_{hi+1}^{L f},  Omega_m = e^{2 pi i / 2^m},
//   L = index bits below lo, f = the group bits in reversed order.
// With L = Ltile + l (Ltile fixed per tile, l the c contiguous low bits)
// the twiddle is V[f] * Omega^{l f}: V is built once per tile from global
// root tables, Omega^{l f} (l f < 2^{c+k}) comes from a two-level table in
// shared memory, the ladder phases from a direct table.  The final SWAPs
// are one in-place blocked bit-reversal pass.
//
// complex64 tiles compute in FP32.  complex128 tiles compute in double-float
// (ff.cuh) on the FP32 pipe: the FP64 pipe of GB300 (0.5 Top/s) would
// otherwise bound every pass many times over the memory time.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "ff.cuh"

namespace qc {

enum TileOpKind { TOP_U2 = 0, TOP_QFTLEVEL = 1, TOP_HB = 2 };
#define QC_TILE_MAXOPS 36

// ------------------------------------------------ arithmetic policies ----
template <typename R> struct TA;

template <> struct TA<float> {
  using E = Cx<float>;
  using V2 = float2;
  using M = Mat2<float>;
  static M mat(const double* U) { return mat_from_host<float>(U); }
  __device__ static E from(V2 v) { return cmake<float>(v.x, v.y); }
  __device__ static V2 to(E z) { return make_float2(z.re, z.im); }
  __device__ static E add(E a, E b) { return cmake<float>(a.re + b.re, a.im + b.im); }
  __device__ static E sub(E a, E b) { return cmake<float>(a.re - b.re, a.im - b.im); }
  // first level of a radix-4 step (no renormalisation to skip in FP32)
  __device__ static E add_u(E a, E b) { return add(a, b); }
  __device__ static E sub_u(E a, E b) { return sub(a, b); }
  __device__ static E norm(E a) { return a; }
  __device__ static E mul(E a, E b) { return cmul(a, b); }
  __device__ static E times_i(E a) { return cmake<float>(-a.im, a.re); }
  __device__ static E neg(E a) { return cmake<float>(-a.re, -a.im); }
  __device__ static E root(uint64_t num, int m) {  // e^{2 pi i num / 2^m}
    double s, c;
    sincospi(ldexp((double)num, 1 - m), &s, &c);
    return cmake<float>((float)c, (float)s);
  }
  __device__ static E fromd(double re, double im) { return cmake<float>((float)re, (float)im); }
  // 2^{-p/2}, computed once per thread, and the multiplication by it
  using S = float;
  __device__ static S scale_const(int p) { return (float)exp2(-0.5 * p); }
  __device__ static E scale_by(E a, S s) { return cmake<float>(a.re * s, a.im * s); }
  __device__ static void u2(int kind, const M& U, E& a0, E& a1) {
    switch (kind) {
      case MK_GENERAL: apply2<float, MK_GENERAL>(U, a0, a1); break;
      case MK_REAL: apply2<float, MK_REAL>(U, a0, a1); break;
      case MK_DIAG: apply2<float, MK_DIAG>(U, a0, a1); break;
      case MK_PHASE1: apply2<float, MK_PHASE1>(U, a0, a1); break;
      case MK_PH_NEG: apply2<float, MK_PH_NEG>(U, a0, a1); break;
      case MK_PH_I: apply2<float, MK_PH_I>(U, a0, a1); break;
      case MK_PH_MI: apply2<float, MK_PH_MI>(U, a0, a1); break;
      case MK_ANTI: apply2<float, MK_ANTI>(U, a0, a1); break;
      case MK_SWAPX: apply2<float, MK_SWAPX>(U, a0, a1); break;
      case MK_HAD: apply2<float, MK_HAD>(U, a0, a1); break;
      default: break;
    }
  }
};

template <> struct TA<double> {
  using E = ffc;
  using V2 = double2;
  using M = Mat2ff;
  static M mat(const double* U) { return mat2ff_from_host(U); }
  // the tile passes are arithmetic bound: the integer-lean conversions
  __device__ static E from(V2 v) { return ffc_make(ff_from_d_fast(v.x), ff_from_d_fast(v.y)); }
  __device__ static V2 to(E z) { return make_double2(ff_to_d_fast(z.re), ff_to_d_fast(z.im)); }
  __device__ static E add(E a, E b) { return ffc_add(a, b); }
  __device__ static E sub(E a, E b) { return ffc_sub(a, b); }
  // first level of a radix-4 step: its sums feed the second level's adds
  // directly, so their renormalisation is left to those
  __device__ static E add_u(E a, E b) { return ffc_add_u(a, b); }
  __device__ static E sub_u(E a, E b) { return ffc_sub_u(a, b); }
  // the closing renormalisation of an unnormalised sum (fast two-sum per
  // component), for a value stored without passing through a product
  __device__ static E norm(E a) {
    float h, l;
    ffc r;
    fast_two_sum(a.re.hi, a.re.lo, h, l);
    r.re = ff_make(h, l);
    fast_two_sum(a.im.hi, a.im.lo, h, l);
    r.im = ff_make(h, l);
    return r;
  }
  __device__ static E mul(E a, E b) { return ffc_mul(a, b); }
  __device__ static E times_i(E a) { return ffc_make(ff_neg(a.im), a.re); }
  __device__ static E neg(E a) { return ffc_make(ff_neg(a.re), ff_neg(a.im)); }
  __device__ static E root(uint64_t num, int m) {
    double s, c;
    sincospi(ldexp((double)num, 1 - m), &s, &c);
    return ffc_from_d(c, s);
  }
  __device__ static E fromd(double re, double im) { return ffc_from_d(re, im); }
  // 2^{-p/2} = 2^{-floor(p/2)} (exact) times 1/sqrt(2) when p is odd
  using S = ff;
  __device__ static S scale_const(int p) {
    ff s = ff_make(ff_bitsf((uint32_t)(127 - p / 2) << 23), 0.f);
    if (p & 1) s = ff_mul(s, ff_from_d(0.70710678118654752440));
    return s;
  }
  __device__ static E scale_by(E a, S s) { return ffc_scale(a, s); }
  __device__ static void u2(int kind, const M& U, E& a0, E& a1) {
    switch (kind) {
      case MK_GENERAL: apply2_ff<MK_GENERAL>(U, a0, a1); break;
      case MK_REAL: apply2_ff<MK_REAL>(U, a0, a1); break;
      case MK_DIAG: apply2_ff<MK_DIAG>(U, a0, a1); break;
      case MK_PHASE1: apply2_ff<MK_PHASE1>(U, a0, a1); break;
      case MK_ANTI: apply2_ff<MK_ANTI>(U, a0, a1); break;
      case MK_HAD: apply2_ff<MK_HAD>(U, a0, a1); break;
      case MK_PH_NEG: a1 = ffc_make(ff_neg(a1.re), ff_neg(a1.im)); break;
      case MK_PH_I: a1 = ffc_make(ff_neg(a1.im), a1.re); break;
      case MK_PH_MI: a1 = ffc_make(a1.im, ff_neg(a1.re)); break;
      case MK_SWAPX: {
        const E t = a0;
        a0 = a1;
        a1 = t;
        break;
      }
      default: break;
    }
  }
};

template <typename R> struct TileProg {
  int nops;
  int lo, k, c;     // group [lo, lo+k), c low contiguous bits (c <= lo)
  int n;
  int twiddle;      // apply the QFT cross phase with the bits below lo
  int qft;          // the program contains QFT levels (build the ladder table)
  int nl;           // global root table split: low table has 2^nl entries
  int scale_p;      // unnormalised butterflies: multiply by 2^{-scale_p/2} at the end
  int8_t kind[QC_TILE_MAXOPS];
  int8_t q[QC_TILE_MAXOPS];   // group-relative qubit
  int8_t mk[QC_TILE_MAXOPS];  // MatKind of a TOP_U2 operator
  typename TA<R>::M U[QC_TILE_MAXOPS];
};

// Shared memory after the tile: V[2^k] (twiddle passes), LAD[lad_entries(k)]
// (QFT passes: level j's 2^j ladder phases e^{2 pi i x / 2^{j+1}} at
// LAD[2^j - 1 + x], so a warp reads consecutive entries), TWA[128], TWB[128].
#define TS_TWA 128
#define TS_TWB 128  // x < 2^{c+k} <= 2^14

// Ladder levels kept in the table.  complex128 stops at level 10 (2047
// double-float entries, 32 KiB), so the 12-qubit lowest group's pass fits
// two CTAs per SM; its level 11 phase is L_11(y) = L_10(y >> 1) times
// e^{2 pi i / 2^12} for odd y, the latter stored after the table.
template <typename R>
__host__ __device__ constexpr int lad_levels(int k) {
  return sizeof(R) == 8 ? (k < 11 ? k : 11) : k;
}
template <typename R>
__host__ __device__ constexpr int lad_entries(int k) {
  return (1 << lad_levels<R>(k)) - 1 + (k > lad_levels<R>(k) ? 1 : 0);
}

__device__ __forceinline__ uint64_t tile_global(uint64_t e, uint64_t T, int lo, int k, int c) {
  const uint64_t cm = (1ull << c) - 1ull;
  const uint64_t tmid = T & ((1ull << (lo - c)) - 1ull);
  const uint64_t thi = T >> (lo - c);
  return (e & cm) | (tmid << c) | ((e >> c) << lo) | (thi << (lo + k));
}

// Root of unity Omega_n^r from the two global tables.
template <typename R>
__device__ __forceinline__ typename TA<R>::E omega(const typename CT<R>::V2* __restrict__ tlo,
                                                   const typename CT<R>::V2* __restrict__ thi, uint64_t r, int nl) {
  const auto a = tlo[r & ((1ull << nl) - 1ull)];
  const auto b = thi[r >> nl];
  return TA<R>::mul(TA<R>::from(a), TA<R>::from(b));
}

// QR consecutive QFT levels jtop, jtop-1, .., jtop-QR+1 in one shared-memory
// round trip: each thread holds the 2^QR elements that differ in the block's
// bits in registers.  Level j (local bit lv = j - jtop + QR - 1) pairs
// elements across local bit lv; its ladder phase e^{2 pi i x / 2^{j+1}}
// uses x = group bits below j = (local bits below lv, placed above the
// block's lowest group qubit) | (the thread's group bits below the block).
template <typename R, int QR>
__device__ __forceinline__ void qft_levels_regs(typename TA<R>::E* sm, int NE, int c, int jtop,
                                                const typename TA<R>::E* LAD) {
  using A = TA<R>;
  using E = typename A::E;
  constexpr int NR = 1 << QR;
  const int jlo = jtop - QR + 1;  // the block's lowest group qubit
  const int bl = c + jlo;         // its index bit
  for (int p = threadIdx.x; p < (NE >> QR); p += blockDim.x) {
    const int base = ((p >> bl) << (bl + QR)) | (p & ((1 << bl) - 1));
    E a[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) a[i] = sm[base | (i << bl)];
    const int xlow = (base >> c) & ((1 << jlo) - 1);
#pragma unroll
    for (int lv = QR - 1; lv >= 0; --lv) {
      const int j = jlo + lv;
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        if ((i >> lv) & 1) continue;
        const int i1 = i | (1 << lv);
        const E s0 = A::add(a[i], a[i1]);
        E d = A::sub(a[i], a[i1]);
        const int x = ((i & ((1 << lv) - 1)) << jlo) | xlow;
        if (x) d = A::mul(LAD[(1 << j) - 1 + x], d);
        a[i] = s0;
        a[i1] = d;
      }
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) sm[base | (i << bl)] = a[i];
  }
}

// L_j(y) = e^{2 pi i y / 2^{j+1}}, y < 2^j, from the ladder table (levels
// below kl) or, for level kl, from level kl - 1 and the extra entry.
template <typename R>
__device__ __forceinline__ typename TA<R>::E ladder_at(const typename TA<R>::E* LAD, int kl, int j, int y) {
  if (j < kl) return LAD[(1 << j) - 1 + y];
  const typename TA<R>::E m = LAD[(1 << (j - 1)) - 1 + (y >> 1)];
  return (y & 1) ? TA<R>::mul(m, LAD[(1 << kl) - 1]) : m;
}

// Shared tables of a pass: the ladders (QFT programs) and the twiddle
// remainder tables TWA, TWB (QFT programs with a twiddle).
template <typename R>
__device__ __forceinline__ void tile_tables(const TileProg<R>& P, typename TA<R>::E* LAD, typename TA<R>::E* TWA,
                                            typename TA<R>::E* TWB, int kl) {
  using A = TA<R>;
  const int k = P.k, hi = P.lo + P.k - 1;
  if (!P.qft) return;
  // ladder tables, one per level: LAD[2^j - 1 + x] = e^{2 pi i x / 2^{j+1}}
  for (int a = threadIdx.x; a < (1 << kl) - 1; a += blockDim.x) {
    const int j = 31 - __clz(a + 1);
    LAD[a] = A::root((uint64_t)(a + 1 - (1 << j)), j + 1);
  }
  if (k > kl && threadIdx.x == 0) LAD[(1 << kl) - 1] = A::root(1, k);  // e^{2 pi i / 2^k}
  // twiddle remainder: Omega_{hi+1}^x = TWA[x & 127] * TWB[x >> 7], x < 2^{c+k}
  if (P.twiddle)
    for (int i = threadIdx.x; i < TS_TWA + TS_TWB; i += blockDim.x) {
      if (i < TS_TWA) TWA[i] = A::root((uint64_t)i, hi + 1);
      else TWB[i - TS_TWA] = A::root((uint64_t)(i - TS_TWA) << 7, hi + 1);
    }
}

// V[f] = 2^{-p/2} Omega_{hi+1}^{Ltile f} for tile T (Ltile = the tile's bits
// between c and lo).
template <typename R>
__device__ __forceinline__ void tile_twiddle_v(const TileProg<R>& P, uint64_t T, typename TA<R>::E* V,
                                               const typename CT<R>::V2* __restrict__ tlo,
                                               const typename CT<R>::V2* __restrict__ thi, typename TA<R>::S sc) {
  const int lo = P.lo, k = P.k, c = P.c, hi = lo + k - 1;
  const uint64_t Lt = (T & ((1ull << (lo - c)) - 1ull)) << c;
  for (int f = threadIdx.x; f < (1 << k); f += blockDim.x) {
    const uint64_t r = (Lt * (uint64_t)f) & ((2ull << hi) - 1ull);
    V[f] = TA<R>::scale_by(omega<R>(tlo, thi, r << (P.n - hi - 1), P.nl), sc);
  }
}

// The program's operators on the staged tile sm (2^{k+c} elements), with a
// barrier after each shared-memory round trip.  QREG: four descending QFT
// levels at a time in registers.
template <typename R, bool QREG>
__device__ __forceinline__ void tile_ops(typename TA<R>::E* sm, const TileProg<R>& P, const typename TA<R>::E* LAD,
                                         int kl) {
  using A = TA<R>;
  using E = typename A::E;
  const int c = P.c;
  const int NE = 1 << (P.k + c);
  for (int o = 0; o < P.nops; ++o) {
    const int b = c + P.q[o];
    const int kind = P.kind[o];
    // four descending QFT levels in registers (complex64: the passes are
    // bound by shared-memory traffic)
    if (QREG && kind == TOP_QFTLEVEL && o + 3 < P.nops && P.kind[o + 1] == kind &&
        P.kind[o + 2] == kind && P.kind[o + 3] == kind && P.q[o + 1] == P.q[o] - 1 &&
        P.q[o + 2] == P.q[o] - 2 && P.q[o + 3] == P.q[o] - 3) {
      qft_levels_regs<R, 4>(sm, NE, c, P.q[o], LAD);
      __syncthreads();
      o += 3;
      continue;
    }
    // two butterfly levels on neighbouring qubits: one shared-memory round
    // trip (radix 4).  QFT levels come in descending order j, j-1; plain
    // Hadamard butterflies commute, so any neighbouring pair qualifies.
    if (kind != TOP_U2 && o + 1 < P.nops && P.kind[o + 1] == kind &&
        (P.q[o + 1] == P.q[o] - 1 || (kind == TOP_HB && P.q[o + 1] == P.q[o] + 1))) {
      const int jh = max(P.q[o], P.q[o + 1]), jl = jh - 1;  // levels jh then jl
      const int bh = c + jh, bl = c + jl;
      const bool lad = (kind == TOP_QFTLEVEL);
      for (int p = threadIdx.x; p < (NE >> 2); p += blockDim.x) {
        const int e00 = (int)insert0(insert0((uint64_t)p, bl), bh);
        const int e01 = e00 | (1 << bl), e10 = e00 | (1 << bh), e11 = e01 | (1 << bh);
        const E a00 = sm[e00], a01 = sm[e01], a10 = sm[e10], a11 = sm[e11];
        // level jh on bit bh: pairs (e00, e10), (e01, e11)
        const E s0 = A::add_u(a00, a10), d0 = A::sub_u(a00, a10);
        const E s1 = A::add_u(a01, a11), d1 = A::sub_u(a01, a11);
        E t0, u0, t1, u1;
        if (lad) {
          // With L(y) = e^{2 pi i y / 2^{jh+1}} and x = group bits below jl:
          // level jh multiplies d0 by L(x) and d1 by L(x + 2^jl) = i L(x);
          // level jl multiplies its bit-1 outputs by L(2x).  So
          //   t0 = s0 + s1,  u0 = L(2x) (s0 - s1),
          //   t1 = L(x) (d0 + i d1),  u1 = L(3x) (d0 - i d1):
          // three multiplications per four amplitudes instead of four.
          const int x = (e00 >> c) & ((1 << jl) - 1);
          const E id1 = A::times_i(d1);
          t0 = A::add(s0, s1);
          // the products renormalise u0, t1, u1; without one (x = 0) the
          // closing fast two-sum does
          u0 = A::sub_u(s0, s1);
          t1 = A::add_u(d0, id1);
          u1 = A::sub_u(d0, id1);
          if (x) {
            u0 = A::mul(ladder_at<R>(LAD, kl, jh, 2 * x), u0);
            t1 = A::mul(ladder_at<R>(LAD, kl, jh, x), t1);
            const int x3 = 3 * x;  // < 1.5 2^jh; L(y + 2^jh) = -L(y)
            u1 = A::mul(ladder_at<R>(LAD, kl, jh, x3 & ((1 << jh) - 1)), u1);
            if (x3 >> jh) u1 = A::neg(u1);
          } else {
            u0 = A::norm(u0);
            t1 = A::norm(t1);
            u1 = A::norm(u1);
          }
        } else {  // plain butterflies on both bits
          t0 = A::add(s0, s1);
          u0 = A::sub(s0, s1);
          t1 = A::add(d0, d1);
          u1 = A::sub(d0, d1);
        }
        sm[e00] = t0;
        sm[e01] = u0;
        sm[e10] = t1;
        sm[e11] = u1;
      }
      __syncthreads();
      ++o;
      continue;
    }
    if (kind == TOP_U2) {
      const int mk = P.mk[o];
      for (int p = threadIdx.x; p < (NE >> 1); p += blockDim.x) {
        const int e0 = (int)insert0((uint64_t)p, b), e1 = e0 | (1 << b);
        E a0 = sm[e0], a1 = sm[e1];
        A::u2(mk, P.U[o], a0, a1);
        sm[e0] = a0;
        sm[e1] = a1;
      }
    } else {
      // unnormalised butterfly (a0 + a1, a0 - a1); for a QFT level the
      // bit-1 half then takes the ladder phase e^{2 pi i x / 2^{j+1}}
      // = omega_k^{x 2^{k-j-1}}, x = group bits below group qubit j
      const int j = P.q[o];
      const bool lad = (kind == TOP_QFTLEVEL);
      for (int p = threadIdx.x; p < (NE >> 1); p += blockDim.x) {
        const int e0 = (int)insert0((uint64_t)p, b), e1 = e0 | (1 << b);
        const E a0 = sm[e0], a1 = sm[e1];
        sm[e0] = A::add(a0, a1);
        E d = A::sub(a0, a1);
        if (lad) {
          const int x = (e0 >> c) & ((1 << j) - 1);
          if (x) d = A::mul(ladder_at<R>(LAD, kl, j, x), d);
        }
        sm[e1] = d;
      }
    }
    __syncthreads();
  }
}

// The tile back to the state: twiddle (which carries the 2^{-p/2} scale) or
// the bare scale.
template <typename R>
__device__ __forceinline__ void tile_store(typename CT<R>::V2* __restrict__ s, uint64_t T, const typename TA<R>::E* sm,
                                           const TileProg<R>& P, const typename TA<R>::E* V,
                                           const typename TA<R>::E* TWA, const typename TA<R>::E* TWB,
                                           typename TA<R>::S sc) {
  using A = TA<R>;
  using E = typename A::E;
  using V2 = typename CT<R>::V2;
  const int lo = P.lo, k = P.k, c = P.c;
  const int NE = 1 << (k + c);
  if (sizeof(R) == 8) {
    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
      E z = sm[e];
      if (P.twiddle) {
        const int f = (int)(__brev((unsigned)(e >> c)) >> (32 - k));
        const int x = (e & ((1 << c) - 1)) * f;  // < 2^{c+k}
        z = A::mul(A::mul(V[f], A::mul(TWA[x & 127], TWB[x >> 7])), z);
      } else if (P.scale_p) {
        z = A::scale_by(z, sc);
      }
      s[tile_global(e, T, lo, k, c)] = A::to(z);
    }
  } else {
    for (int e = 2 * threadIdx.x; e < NE; e += 2 * blockDim.x) {
      E z0 = sm[e], z1 = sm[e + 1];
      if (P.twiddle) {
        // e and e+1 share the group bits (c >= 1 whenever lo > 0)
        const int f = (int)(__brev((unsigned)(e >> c)) >> (32 - k));
        const int x0 = (e & ((1 << c) - 1)) * f, x1 = x0 + f;
        const E v = V[f];
        z0 = A::mul(A::mul(v, A::mul(TWA[x0 & 127], TWB[x0 >> 7])), z0);
        z1 = A::mul(A::mul(v, A::mul(TWA[x1 & 127], TWB[x1 >> 7])), z1);
      } else if (P.scale_p) {
        z0 = A::scale_by(z0, sc);
        z1 = A::scale_by(z1, sc);
      }
      const V2 w0 = A::to(z0), w1 = A::to(z1);
      *reinterpret_cast<float4*>(s + tile_global(e, T, lo, k, c)) = make_float4(w0.x, w0.y, w1.x, w1.y);
    }
  }
}

// Two CTAs per SM (64 registers): every layer program and the complex128 QFT.
template <typename R>
__global__ void __launch_bounds__(512, 2) k_tile(typename CT<R>::V2* __restrict__ s, uint64_t ntiles,
                                                 const TileProg<R> P, const typename CT<R>::V2* __restrict__ tlo,
                                                 const typename CT<R>::V2* __restrict__ thi) {
  using A = TA<R>;
  using E = typename A::E;
  using V2 = typename CT<R>::V2;
  extern __shared__ __align__(16) unsigned char smraw[];
  E* sm = reinterpret_cast<E*>(smraw);
  const int lo = P.lo, k = P.k, c = P.c;
  const int NE = 1 << (k + c);
  E* V = sm + NE;
  E* LAD = V + (P.twiddle ? (1 << k) : 0);
  const int kl = lad_levels<R>(k);  // levels in the table
  E* TWA = LAD + (P.qft ? lad_entries<R>(k) : 0);
  E* TWB = TWA + TS_TWA;
  const typename A::S sc = A::scale_const(P.scale_p);
  tile_tables<R>(P, LAD, TWA, TWB, kl);
  for (uint64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
    if (P.twiddle) tile_twiddle_v<R>(P, T, V, tlo, thi, sc);
    // load: 16-byte vectors; for complex64 two neighbouring elements (c >= 1
    // or a fully contiguous tile, so e and e+1 are neighbours in memory);
    // four 16-byte loads in flight per thread before the first shared-memory
    // store (the tile is read once; with two CTAs per SM the load phase is
    // otherwise latency bound)
    constexpr int LU = 4;
    if (sizeof(R) == 8) {
      for (int e0 = threadIdx.x; e0 < NE; e0 += LU * blockDim.x) {
        V2 v[LU];
#pragma unroll
        for (int u = 0; u < LU; ++u) {
          const int e = e0 + u * blockDim.x;
          if (e < NE) v[u] = s[tile_global(e, T, lo, k, c)];
        }
#pragma unroll
        for (int u = 0; u < LU; ++u) {
          const int e = e0 + u * blockDim.x;
          if (e < NE) sm[e] = A::from(v[u]);
        }
      }
    } else {
      for (int e0 = 2 * threadIdx.x; e0 < NE; e0 += 2 * LU * blockDim.x) {
        float4 v[LU];
#pragma unroll
        for (int u = 0; u < LU; ++u) {
          const int e = e0 + 2 * u * blockDim.x;
          if (e < NE) v[u] = *reinterpret_cast<const float4*>(s + tile_global(e, T, lo, k, c));
        }
#pragma unroll
        for (int u = 0; u < LU; ++u) {
          const int e = e0 + 2 * u * blockDim.x;
          if (e < NE) {
            sm[e] = A::from(CT<R>::make(v[u].x, v[u].y));
            sm[e + 1] = A::from(CT<R>::make(v[u].z, v[u].w));
          }
        }
      }
    }
    __syncthreads();
    tile_ops<R, false>(sm, P, LAD, kl);
    tile_store<R>(s, T, sm, P, V, TWA, TWB, sc);
    __syncthreads();
  }
}

// ------------------------------------------------ complex128 QFT passes --
// For states of at least 12 qubits every complex128 QFT pass has k + c = 12,
// so the pass is compiled per group size K: the radix-4 level pairs' bit
// positions are constants, the tile is XOR-swizzled in 16-byte elements
// (bits 0..2 take bits 3..5, which is linear over XOR, so every element of a
// radix-4 quad is one XOR away from the thread's base and the low-bit
// stages are free of bank conflicts), and a thread's eight load / store
// addresses are one base plus multiples of a per-pass stride.  The
// arithmetic is that of k_tile's QFT programs.
__device__ __forceinline__ int tsw(int e) { return e ^ ((e >> 3) & 7); }

template <int BH, int BL, int JH, int C>
__device__ __forceinline__ void qft_quad_c128(ffc* sm, const ffc* LAD, int kl) {
  using A = TA<double>;
  constexpr int NE = 1 << 12, JL = JH - 1;
  static_assert(BH == BL + 1, "neighbouring levels");
#pragma unroll
  for (int r = 0; r < (NE >> 2) / 512; ++r) {
    const int p = threadIdx.x + 512 * r;
    const int e00 = ((p >> BL) << (BL + 2)) | (p & ((1 << BL) - 1));
    const int b = tsw(e00);
    const int o01 = tsw(1 << BL), o10 = tsw(1 << BH), o11 = tsw(3 << BL);
    const ffc a00 = sm[b], a01 = sm[b ^ o01], a10 = sm[b ^ o10], a11 = sm[b ^ o11];
    const ffc s0 = A::add_u(a00, a10), d0 = A::sub_u(a00, a10);
    const ffc s1 = A::add_u(a01, a11), d1 = A::sub_u(a01, a11);
    // as in k_tile: t0 = s0 + s1, u0 = L(2x)(s0 - s1), t1 = L(x)(d0 + i d1),
    // u1 = L(3x)(d0 - i d1), L(y) = e^{2 pi i y / 2^{JH+1}}, x = group bits below JL
    const int x = (e00 >> C) & ((1 << JL) - 1);
    const ffc id1 = A::times_i(d1);
    const ffc t0 = A::add(s0, s1);
    ffc u0 = A::sub_u(s0, s1), t1 = A::add_u(d0, id1), u1 = A::sub_u(d0, id1);
    if (x) {
      u0 = A::mul(ladder_at<double>(LAD, kl, JH, 2 * x), u0);
      t1 = A::mul(ladder_at<double>(LAD, kl, JH, x), t1);
      const int x3 = 3 * x;
      u1 = A::mul(ladder_at<double>(LAD, kl, JH, x3 & ((1 << JH) - 1)), u1);
      if (x3 >> JH) u1 = A::neg(u1);
    } else {
      u0 = A::norm(u0);
      t1 = A::norm(t1);
      u1 = A::norm(u1);
    }
    sm[b] = t0;
    sm[b ^ o01] = u0;
    sm[b ^ o10] = t1;
    sm[b ^ o11] = u1;
  }
}

// level 0 alone (odd K): plain butterflies on tile bit C (no ladder below it)
template <int C>
__device__ __forceinline__ void qft_single0_c128(ffc* sm) {
  using A = TA<double>;
  constexpr int NE = 1 << 12;
#pragma unroll
  for (int r = 0; r < (NE >> 1) / 512; ++r) {
    const int p = threadIdx.x + 512 * r;
    const int e0 = ((p >> C) << (C + 1)) | (p & ((1 << C) - 1));
    const int b = tsw(e0), o = tsw(1 << C);
    const ffc a0 = sm[b], a1 = sm[b ^ o];
    sm[b] = A::add(a0, a1);
    sm[b ^ o] = A::sub(a0, a1);
  }
}

// levels JH, JH-1 as one quad stage, then the rest
template <int K, int JH>
__device__ __forceinline__ void qft_stages_c128(ffc* sm, const ffc* LAD, int kl) {
  constexpr int C = 12 - K;
  if constexpr (JH >= 1) {
    qft_quad_c128<C + JH, C + JH - 1, JH, C>(sm, LAD, kl);
    __syncthreads();
    qft_stages_c128<K, JH - 2>(sm, LAD, kl);
  } else if constexpr (JH == 0) {
    qft_single0_c128<C>(sm);
    __syncthreads();
  }
}

// Between the passes of one transform the state holds each amplitude's
// double-float parts (re.hi, re.lo, im.hi, im.lo: the same 16 bytes), so
// only the first pass converts from IEEE double, and the bit reversal that
// ends the transform converts back.
__device__ __forceinline__ ffc ffc_unpack(double2 v) {
  return ffc_make(ff_make(__int_as_float(__double2loint(v.x)), __int_as_float(__double2hiint(v.x))),
                  ff_make(__int_as_float(__double2loint(v.y)), __int_as_float(__double2hiint(v.y))));
}
__device__ __forceinline__ double2 ffc_pack(ffc z) {
  return make_double2(__hiloint2double(__float_as_int(z.re.lo), __float_as_int(z.re.hi)),
                      __hiloint2double(__float_as_int(z.im.lo), __float_as_int(z.im.hi)));
}

template <int K>
__global__ void __launch_bounds__(512, 2) k_qft_c128_k(double2* __restrict__ s, uint64_t ntiles, const TileProg<double> P,
                                                       const double2* __restrict__ tlo,
                                                       const double2* __restrict__ thi, int ld_ff, int st_ff) {
  using A = TA<double>;
  constexpr int C = 12 - K, NE = 1 << 12, PER = NE / 512;
  static_assert(C <= 9, "512-element strides stay inside the group bits");
  static_assert(PER == 8, "eight elements per thread");
  extern __shared__ __align__(16) unsigned char smraw[];
  ffc* sm = reinterpret_cast<ffc*>(smraw);
  const int lo = P.lo, hi = lo + K - 1, sh = P.n - hi - 1, nl = P.nl;
  const bool tw = P.twiddle != 0;
  ffc* LAD = sm + NE;
  constexpr int kl = lad_levels<double>(K);
  for (int a = threadIdx.x; a < (1 << kl) - 1; a += blockDim.x) {
    const int j = 31 - __clz(a + 1);
    LAD[a] = A::root((uint64_t)(a + 1 - (1 << j)), j + 1);
  }
  if (K > kl && threadIdx.x == 0) LAD[(1 << kl) - 1] = A::root(1, K);
  const typename A::S sc = A::scale_const(K);
  const int tid = threadIdx.x;
  const int st = tsw(tid);
  const uint64_t gstep = (uint64_t)(512 >> C) << lo;
  const uint64_t hm = (2ull << hi) - 1ull;
  // twiddle of element e = tid + 512 u: 2^{-K/2} Omega_{hi+1}^{m f} with
  // m = its bits below lo (the tile's bits between C and lo, then the C low
  // bits of tid: the same for all eight elements of a thread) and
  // f = brev_K(e >> C) = F + brev_3(u), F = brev_K(tid >> C) (a multiple of
  // 8).  So the eight twiddles are B g^v, v = brev_3(u), with
  // B = 2^{-K/2} Omega^{m F} and g = Omega^m: two root-table lookups and a
  // chain of seven products per thread instead of two products per element.
  const int F = (int)(__brev((unsigned)(tid >> C)) >> (32 - K));
  for (uint64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
    const uint64_t g0 = tile_global((uint64_t)tid, T, lo, K, C);
    // four 16-byte loads in flight per thread, twice
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = s[g0 + (4 * h + u) * gstep];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        sm[st ^ tsw(512 * (4 * h + u))] =
            ld_ff ? ffc_unpack(v[u]) : ffc_make(ff_from_d_fast(v[u].x), ff_from_d_fast(v[u].y));
    }
    __syncthreads();
    qft_stages_c128<K, K - 1>(sm, LAD, kl);
    // store: the twiddle (which carries the 2^{-K/2} scale), or the scale
    if (tw) {
      const uint64_t m = ((T & ((1ull << (lo - C)) - 1ull)) << C) | (uint64_t)(tid & ((1 << C) - 1));
      ffc W = A::scale_by(omega<double>(tlo, thi, ((m * (uint64_t)F) & hm) << sh, nl), sc);
      const ffc g = omega<double>(tlo, thi, (m & hm) << sh, nl);
#pragma unroll
      for (int v = 0; v < PER; ++v) {
        const int u = ((v & 1) << 2) | (v & 2) | (v >> 2);  // brev_3(v)
        const ffc z = A::mul(W, sm[st ^ tsw(512 * u)]);
        s[g0 + u * gstep] = st_ff ? ffc_pack(z) : A::to(z);
        if (v + 1 < PER) W = A::mul(W, g);
      }
    } else {
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const ffc z = A::scale_by(sm[st ^ tsw(512 * u)], sc);
        s[g0 + u * gstep] = st_ff ? ffc_pack(z) : A::to(z);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------- complex64 QFT passes --
// One CTA per SM with two 64 KiB tile buffers: the next tile's loads
// (cp.async, 16 bytes each) are in flight while the current tile is
// transformed and written back.  The group's levels run in register blocks
// of up to four levels (one shared-memory round trip each).  Within a block
// on group qubits jlo .. jlo+QR-1, level j = jlo + lv multiplies the
// difference of the pair with local low bits m by
//   L_j(x) = e^{2 pi i x / 2^{j+1}},  x = m 2^jlo + xlow,
//   L_j(x) = e^{2 pi i m / 2^{lv+1}} L_j(xlow),
// so a thread loads one ladder entry per level (its xlow is fixed) and
// multiplies it by constant roots of unity.  The shared tile is swizzled in
// 16-byte units (pairs of amplitudes stay together for the 16-byte copies):
// strided register blocks then hit at most twice the minimum number of
// shared-memory wavefronts instead of up to 16x.
__device__ __forceinline__ int qsw(int e) { return e ^ (((e >> 4) & 7) << 1); }

__device__ __forceinline__ float2 c2mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// e^{2 pi i m / 2^{lv+1}} for m < 2^lv, lv <= 3 (constants)
__device__ __forceinline__ float2 qroot(int lv, int m) {
  const float r = 0.70710678118654752f, c1 = 0.92387953251128676f, s1 = 0.38268343236508977f;
  if (lv <= 0 || m == 0) return make_float2(1.f, 0.f);
  if (lv == 1) return make_float2(0.f, 1.f);
  if (lv == 2) {
    switch (m) {
      case 1: return make_float2(r, r);
      case 2: return make_float2(0.f, 1.f);
      default: return make_float2(-r, r);
    }
  }
  switch (m) {  // lv == 3: sixteenth roots e^{2 pi i m / 16}
    case 1: return make_float2(c1, s1);
    case 2: return make_float2(r, r);
    case 3: return make_float2(s1, c1);
    case 4: return make_float2(0.f, 1.f);
    case 5: return make_float2(-s1, c1);
    case 6: return make_float2(-r, r);
    default: return make_float2(-c1, s1);
  }
}

template <int QR>
__device__ __forceinline__ void qft_block_c64(float2* sm, int NE, int c, int jtop, const float2* LAD) {
  constexpr int NR = 1 << QR;
  const int jlo = jtop - QR + 1;
  const int bl = c + jlo;
  for (int p = threadIdx.x; p < (NE >> QR); p += blockDim.x) {
    const int base = ((p >> bl) << (bl + QR)) | (p & ((1 << bl) - 1));
    float2 a[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) a[i] = sm[qsw(base | (i << bl))];
    const int xlow = (base >> c) & ((1 << jlo) - 1);
#pragma unroll
    for (int lv = QR - 1; lv >= 0; --lv) {
      const int j = jlo + lv;
      const float2 u = LAD[(1 << j) - 1 + xlow];  // L_j(xlow)
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        if ((i >> lv) & 1) continue;
        const int i1 = i | (1 << lv);
        const float2 x0 = a[i], x1 = a[i1];
        a[i] = make_float2(x0.x + x1.x, x0.y + x1.y);
        const int m = i & ((1 << lv) - 1);  // the factor e^{2 pi i m / 2^{lv+1}} L_j(xlow)
        a[i1] = c2mul(make_float2(x0.x - x1.x, x0.y - x1.y), m ? c2mul(qroot(lv, m), u) : u);
      }
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) sm[qsw(base | (i << bl))] = a[i];
  }
}

// Register blocks over levels k-1 .. 0: ceil(k/4) blocks, the larger first.
__device__ __forceinline__ void qft_levels_c64(float2* sm, int NE, int c, int k, const float2* LAD) {
  const int nb = (k + 3) >> 2;
  int j = k - 1;
  for (int b = 0; b < nb; ++b) {
    const int qr = (j + 1 + (nb - b) - 1) / (nb - b);  // balanced, larger first
    switch (qr) {
      case 4: qft_block_c64<4>(sm, NE, c, j, LAD); break;
      case 3: qft_block_c64<3>(sm, NE, c, j, LAD); break;
      case 2: qft_block_c64<2>(sm, NE, c, j, LAD); break;
      default: qft_block_c64<1>(sm, NE, c, j, LAD); break;
    }
    __syncthreads();
    j -= qr;
  }
}

// Compile-time forms for the passes of states of at least 13 qubits, where
// every tile holds 2^13 amplitudes (k + c = 13): the register blocks' bit
// positions, the swizzled offsets of a block's elements and a thread's
// copy and store offsets are constants, so the index arithmetic is one XOR
// per element.  qsw is linear over XOR, qsw(x ^ y) = qsw(x) ^ qsw(y).
template <int QR, int BL, int JLO>
__device__ __forceinline__ void qft_block_c64_ct(float2* sm, const float2* LAD) {
  constexpr int NR = 1 << QR, NE = 1 << 13;
  constexpr int C = BL - JLO;
#pragma unroll
  for (int r = 0; r < (NE >> QR) / 512; ++r) {
    const int p = threadIdx.x + 512 * r;
    const int base = ((p >> BL) << (BL + QR)) | (p & ((1 << BL) - 1));
    const int sb = qsw(base);
    float2 a[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) a[i] = sm[sb ^ qsw(i << BL)];
    const int xlow = (base >> C) & ((1 << JLO) - 1);
#pragma unroll
    for (int lv = QR - 1; lv >= 0; --lv) {
      const int j = JLO + lv;
      const float2 u = LAD[(1 << j) - 1 + xlow];  // L_j(xlow)
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        if ((i >> lv) & 1) continue;
        const int i1 = i | (1 << lv);
        const float2 x0 = a[i], x1 = a[i1];
        a[i] = make_float2(x0.x + x1.x, x0.y + x1.y);
        const int m = i & ((1 << lv) - 1);  // the factor e^{2 pi i m / 2^{lv+1}} L_j(xlow)
        a[i1] = c2mul(make_float2(x0.x - x1.x, x0.y - x1.y), m ? c2mul(qroot(lv, m), u) : u);
      }
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) sm[sb ^ qsw(i << BL)] = a[i];
  }
}

// block b of the K levels: ceil(K/4) blocks, balanced, the larger first
__host__ __device__ constexpr int qft_nblocks(int K) { return (K + 3) >> 2; }
__host__ __device__ constexpr int qft_block_size(int K, int b) {
  int j = K - 1, qr = 0;
  for (int i = 0; i <= b; ++i) {
    const int nb = qft_nblocks(K);
    qr = (j + 1 + (nb - i) - 1) / (nb - i);
    if (i < b) j -= qr;
  }
  return qr;
}
__host__ __device__ constexpr int qft_block_jlo(int K, int b) {
  int j = K - 1;
  for (int i = 0; i <= b; ++i) j -= qft_block_size(K, i);
  return j + 1;
}

// blocks B .. END-1 of the K levels, a barrier after each
template <int K, int B, int END>
__device__ __forceinline__ void qft_levels_c64_ct(float2* sm, const float2* LAD) {
  if constexpr (B < END) {
    constexpr int QR = qft_block_size(K, B), JLO = qft_block_jlo(K, B), C = 13 - K;
    qft_block_c64_ct<QR, C + JLO, JLO>(sm, LAD);
    __syncthreads();
    qft_levels_c64_ct<K, B + 1, END>(sm, LAD);
  }
}

// The last block (levels QR-1 .. 0, on tile bits C .. C+QR-1) of a twiddle
// pass, written straight to the state: element i of a thread's block has
// group bits (base >> C) | i, so its state index is the block base's plus
// i << lo, and its twiddle is W[e] V[f] with f = brev(base >> C) | brev(i).
// Consecutive threads hold consecutive low bits (2^C >= 16 amplitudes, at
// least 128 contiguous bytes per warp and element).
template <int K, int QR>
__device__ __forceinline__ void qft_last_block_store_c64(const float2* sm, const float2* LAD, const float2* W,
                                                         const float2* V, float2* __restrict__ s, uint64_t T,
                                                         int lo) {
  constexpr int NR = 1 << QR, NE = 1 << 13, C = 13 - K, BL = C;
#pragma unroll
  for (int r = 0; r < (NE >> QR) / 512; ++r) {
    const int p = threadIdx.x + 512 * r;
    const int base = ((p >> BL) << (BL + QR)) | (p & ((1 << BL) - 1));
    const int sb = qsw(base);
    float2 a[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) a[i] = sm[sb ^ qsw(i << BL)];
    // jlo = 0: every level's ladder phase is a constant root (xlow = 0)
#pragma unroll
    for (int lv = QR - 1; lv >= 0; --lv) {
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        if ((i >> lv) & 1) continue;
        const int i1 = i | (1 << lv);
        const float2 x0 = a[i], x1 = a[i1];
        a[i] = make_float2(x0.x + x1.x, x0.y + x1.y);
        const int m = i & ((1 << lv) - 1);
        const float2 d = make_float2(x0.x - x1.x, x0.y - x1.y);
        a[i1] = m ? c2mul(d, qroot(lv, m)) : d;
      }
    }
    const uint64_t g = tile_global((uint64_t)base, T, lo, K, C);
    const int fb = (int)(__brev((unsigned)(base >> C)) >> (32 - K));
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int f = fb | (int)(__brev((unsigned)i) >> (32 - K));
      s[g + ((uint64_t)i << lo)] = c2mul(c2mul(a[i], W[base | (i << BL)]), V[f]);
    }
  }
}

template <int K>
__global__ void __launch_bounds__(512, 1) k_qft_db_c64_k(float2* __restrict__ s, uint64_t ntiles, const TileProg<float> P,
                                                         const float2* __restrict__ tlo,
                                                         const float2* __restrict__ thi) {
  using A = TA<float>;
  constexpr int C = 13 - K, NE = 1 << 13;
  static_assert(C <= 10, "1024-element copy strides stay inside the group bits");
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lo = P.lo, hi = lo + K - 1;
  const bool tw = P.twiddle != 0;
  float2* buf0 = reinterpret_cast<float2*>(smraw);
  float2* buf1 = buf0 + NE;
  float2* W = buf1 + NE;
  float2* V = W + (tw ? NE : 0);
  float2* LAD = V + (tw ? (1 << K) : 0);
  const float sc = (float)exp2(-0.5 * K);
  const int e0 = 2 * threadIdx.x;
  const int se0 = qsw(e0);
  const uint64_t gstep = (uint64_t)(1024 >> C) << lo;
  // this thread's copy / store elements e0 + 1024 u share the group bits'
  // low part; their reversed group bits are f0 | brev(u) at the top
  const int f0 = (int)(__brev((unsigned)(e0 >> C)) >> (32 - K));
  auto issue = [&](uint64_t T, float2* dst) {
    const uint64_t g = tile_global((uint64_t)e0, T, lo, K, C);
#pragma unroll
    for (int u = 0; u < NE / 1024; ++u) {
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + (se0 ^ qsw(1024 * u)));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(s + g + u * gstep) : "memory");
    }
  };
  uint64_t T = blockIdx.x;
  if (T < ntiles) issue(T, buf0);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  // the pass's tables from the global root tables (powers of Omega_n), in
  // FP32: e^{2 pi i x / 2^{j+1}} = Omega_n^{x 2^{n-j-1}}
  for (int a = threadIdx.x; a < (1 << K) - 1; a += blockDim.x) {
    const int j = 31 - __clz(a + 1);
    const A::E z = omega<float>(tlo, thi, (uint64_t)(a + 1 - (1 << j)) << (P.n - j - 1), P.nl);
    LAD[a] = make_float2(z.re, z.im);
  }
  if (tw)
    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
      const int f = (int)(__brev((unsigned)(e >> C)) >> (32 - K));
      const uint64_t x = (uint64_t)((e & ((1 << C) - 1)) * f);  // < 2^13 <= 2^{hi+1}
      const A::E z = omega<float>(tlo, thi, x << (P.n - hi - 1), P.nl);
      W[e] = make_float2(z.re, z.im);
    }
  for (int it = 0; T < ntiles; T += gridDim.x, ++it) {
    float2* cur = (it & 1) ? buf1 : buf0;
    float2* nxt = (it & 1) ? buf0 : buf1;
    if (T + gridDim.x < ntiles) issue(T + gridDim.x, nxt);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    if (tw) {
      const uint64_t Lt = (T & ((1ull << (lo - C)) - 1ull)) << C;
      for (int f = threadIdx.x; f < (1 << K); f += blockDim.x) {
        const uint64_t r = (Lt * (uint64_t)f) & ((2ull << hi) - 1ull);
        const A::E z = A::scale_by(omega<float>(tlo, thi, r << (P.n - hi - 1), P.nl), sc);
        V[f] = make_float2(z.re, z.im);
      }
    }
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    if constexpr (C >= 4) {
      if (tw) {
        // every pass above the lowest group: the last block goes straight to the state
        constexpr int NB = qft_nblocks(K);
        qft_levels_c64_ct<K, 0, NB - 1>(cur, LAD);
        qft_last_block_store_c64<K, qft_block_size(K, NB - 1)>(cur, LAD, W, V, s, T, lo);
        __syncthreads();
        continue;
      }
    }
    qft_levels_c64_ct<K, 0, qft_nblocks(K)>(cur, LAD);
    const uint64_t g = tile_global((uint64_t)e0, T, lo, K, C);
#pragma unroll
    for (int u = 0; u < NE / 1024; ++u) {
      float4 z = *reinterpret_cast<const float4*>(cur + (se0 ^ qsw(1024 * u)));
      if (tw) {
        // the group bits of e0 + 1024 u are (e0 >> C) + (1024 u >> C): reversed,
        // brev(u) lands below f0's bits
        const int f = f0 | (int)(__brev((unsigned)((1024 * u) >> C)) >> (32 - K));
        const float2 v = V[f];
        const float4 w = *reinterpret_cast<const float4*>(W + e0 + 1024 * u);
        const float2 z0 = c2mul(c2mul(make_float2(z.x, z.y), make_float2(w.x, w.y)), v);
        const float2 z1 = c2mul(c2mul(make_float2(z.z, z.w), make_float2(w.z, w.w)), v);
        z = make_float4(z0.x, z0.y, z1.x, z1.y);
      } else {
        z = make_float4(z.x * sc, z.y * sc, z.z * sc, z.w * sc);
      }
      *reinterpret_cast<float4*>(s + g + u * gstep) = z;
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// P holds the pass: group [lo, lo+k), c contiguous bits, twiddle = lo > 0,
// scale_p = k.  Shared memory: two tile buffers, then (twiddle passes) the
// per-pass table W[e] = Omega_{hi+1}^{l f} (l = e's c low bits, f = its
// group bits reversed) and V[f] (per tile), then the ladder table.
__global__ void __launch_bounds__(512, 1) k_qft_db_c64(float2* __restrict__ s, uint64_t ntiles, const TileProg<float> P,
                                                       const float2* __restrict__ tlo, const float2* __restrict__ thi) {
  using A = TA<float>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lo = P.lo, k = P.k, c = P.c, hi = lo + k - 1;
  const int NE = 1 << (k + c);
  float2* buf0 = reinterpret_cast<float2*>(smraw);
  float2* buf1 = buf0 + NE;
  float2* W = buf1 + NE;
  float2* V = W + (P.twiddle ? NE : 0);
  float2* LAD = V + (P.twiddle ? (1 << k) : 0);
  const float sc = (float)exp2(-0.5 * P.scale_p);
  // 16-byte copies of amplitude pairs (e, e+1); successive ones of a thread
  // are 1024 tile elements apart
  const bool step_ok = c <= 10;
  const uint64_t gstep = step_ok ? ((uint64_t)(1024 >> c) << lo) : 0;
  auto issue = [&](uint64_t T, float2* dst) {
    const int e0 = 2 * threadIdx.x;
    uint64_t g = tile_global((uint64_t)e0, T, lo, k, c);
    for (int e = e0; e < NE; e += 1024) {
      if (!step_ok) g = tile_global((uint64_t)e, T, lo, k, c);
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + qsw(e));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(s + g) : "memory");
      g += gstep;
    }
  };
  uint64_t T = blockIdx.x;
  if (T < ntiles) issue(T, buf0);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  // ladder table: LAD[2^j - 1 + x] = e^{2 pi i x / 2^{j+1}}, j < k
  // (from the global root tables: e^{2 pi i x / 2^{j+1}} = Omega_n^{x 2^{n-j-1}})
  for (int a = threadIdx.x; a < (1 << k) - 1; a += blockDim.x) {
    const int j = 31 - __clz(a + 1);
    const A::E z = omega<float>(tlo, thi, (uint64_t)(a + 1 - (1 << j)) << (P.n - j - 1), P.nl);
    LAD[a] = make_float2(z.re, z.im);
  }
  if (P.twiddle)
    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
      const int f = (int)(__brev((unsigned)(e >> c)) >> (32 - k));
      const uint64_t x = (uint64_t)((e & ((1 << c) - 1)) * f);  // l f < 2^{c+k} <= 2^{hi+1}
      const A::E z = omega<float>(tlo, thi, x << (P.n - hi - 1), P.nl);
      W[e] = make_float2(z.re, z.im);
    }
  for (int it = 0; T < ntiles; T += gridDim.x, ++it) {
    float2* cur = (it & 1) ? buf1 : buf0;
    float2* nxt = (it & 1) ? buf0 : buf1;
    // nxt was last read by the previous tile's store, which ended at that
    // iteration's closing barrier
    if (T + gridDim.x < ntiles) issue(T + gridDim.x, nxt);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    if (P.twiddle) {
      // V[f] = 2^{-k/2} Omega_{hi+1}^{Ltile f}
      const uint64_t Lt = (T & ((1ull << (lo - c)) - 1ull)) << c;
      for (int f = threadIdx.x; f < (1 << k); f += blockDim.x) {
        const uint64_t r = (Lt * (uint64_t)f) & ((2ull << hi) - 1ull);
        const A::E z = A::scale_by(omega<float>(tlo, thi, r << (P.n - hi - 1), P.nl), sc);
        V[f] = make_float2(z.re, z.im);
      }
    }
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this thread's copies of the current tile
    __syncthreads();                                         // ... and everyone's; tables and V written
    qft_levels_c64(cur, NE, c, k, LAD);
    // store: pairs (e, e+1) share the group bits (c >= 1 whenever lo > 0)
    const int e0 = 2 * threadIdx.x;
    uint64_t g = tile_global((uint64_t)e0, T, lo, k, c);
    for (int e = e0; e < NE; e += 1024) {
      if (!step_ok) g = tile_global((uint64_t)e, T, lo, k, c);
      float4 z = *reinterpret_cast<const float4*>(cur + qsw(e));
      if (P.twiddle) {
        const int f = (int)(__brev((unsigned)(e >> c)) >> (32 - k));
        const float2 v = V[f];
        const float4 w = *reinterpret_cast<const float4*>(W + e);
        const float2 z0 = c2mul(c2mul(make_float2(z.x, z.y), make_float2(w.x, w.y)), v);
        const float2 z1 = c2mul(c2mul(make_float2(z.z, z.w), make_float2(w.z, w.w)), v);
        z = make_float4(z0.x, z0.y, z1.x, z1.y);
      } else {
        z = make_float4(z.x * sc, z.y * sc, z.z * sc, z.w * sc);
      }
      *reinterpret_cast<float4*>(s + g) = z;
      g += gstep;
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Tables of Omega^a (a < 2^nl) and Omega^{a 2^nl} (a < 2^{n-nl}),
// Omega = e^{2 pi i / 2^n}, from sincospi in double precision.
template <typename R>
__global__ void k_roots(typename CT<R>::V2* tlo, typename CT<R>::V2* thi, int n, int nl) {
  const uint64_t nlo = 1ull << nl, nhi = 1ull << (n - nl);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nlo + nhi;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const bool low = i < nlo;
    const uint64_t a = low ? i : (i - nlo);
    // angle / pi = 2 a 2^{shift} / 2^n, reduced mod 2 exactly in integers
    const int shift = low ? 0 : nl;
    const uint64_t num = (a << (shift + 1)) & ((2ull << n) - 1ull);  // mod 2^{n+1}
    const double x = ldexp((double)num, -n);
    double sn, cs;
    sincospi(x, &sn, &cs);
    if (low) tlo[a] = CT<R>::make((R)cs, (R)sn);
    else thi[a] = CT<R>::make((R)cs, (R)sn);
  }
}

// --------------------------------------------------------------------------
// Tile-size choices: c low contiguous bits give 128-byte rows; k group bits;
// the tile holds 2^{k+c} amplitudes (64 KiB: 2^12 complex128 or 2^13
// complex64 amplitudes, 128 KiB for complex64 layer groups of 10): 30
// complex128 qubits in three QFT passes, 12 + 9 + 9, 32 complex64 qubits in
// four, 13 + 7 + 6 + 6.
template <typename R> struct TileCfg;
template <> struct TileCfg<double> { static constexpr int C = 3, K = 9, BOT = 12; };
// the ladder helper reaches one level past the table (levels 0..10)
static_assert(TileCfg<double>::BOT <= 12 && TileCfg<double>::K <= 12, "complex128 groups of at most 12 qubits");
// complex64 layers: 128 KiB tiles for groups of 10 (c = 4, one CTA per SM),
// 64 KiB for smaller ones; the complex64 QFT plans groups of at most 9 above
// the lowest 13 (64 KiB tiles, two buffers in one CTA)
template <> struct TileCfg<float> { static constexpr int C = 4, K = 10, BOT = 13; };

struct Group {
  int lo, k;
};

// Groups covering qubits [0, n): the lowest group up to bot qubits (no
// separate contiguous bits needed), the others up to K, balanced.
static std::vector<Group> plan_groups_k(int n, int bot, int K) {
  std::vector<Group> g;
  const int g0 = std::min(n, bot);
  g.push_back({0, g0});
  int rest = n - g0;
  if (rest > 0) {
    const int np = (rest + K - 1) / K;
    int lo = g0;
    for (int i = 0; i < np; ++i) {
      const int k = (rest + (np - i) - 1) / (np - i);  // balanced
      g.push_back({lo, k});
      lo += k;
      rest -= k;
    }
  }
  return g;
}

template <typename R>
static std::vector<Group> plan_groups(int n) {
  return plan_groups_k(n, TileCfg<R>::BOT, TileCfg<R>::K);
}

template <typename R>
static size_t tile_smem(int k, int c, bool twiddle, bool qft) {
  using E = typename TA<R>::E;
  return sizeof(E) * (((size_t)1 << (k + c)) + (twiddle ? ((size_t)1 << k) : 0) +
                      (qft ? (size_t)lad_entries<R>(k) : 0) + TS_TWA + TS_TWB);
}

template <typename R>
static qc_status run_tile(qc_state* s, TileProg<R>& P, const typename CT<R>::V2* tlo,
                          const typename CT<R>::V2* thi) {
  using V2 = typename CT<R>::V2;
  if (P.nops == 0 && !P.twiddle) return QC_OK;
  P.n = s->n;
  const int tb = P.k + P.c;
  const uint64_t ntiles = 1ull << (s->n - tb);
  const size_t smem = tile_smem<R>(P.k, P.c, P.twiddle != 0, P.qft != 0);
  constexpr int threads = 512;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_tile<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  const unsigned grid = resident_grid(k_tile<R>, threads, (int64_t)ntiles, 1, smem);
  k_tile<R><<<grid, threads, smem, s->stream>>>(reinterpret_cast<V2*>(s->data), ntiles, P, tlo, thi);
  return check_launch("tile pass");
}

// complex128 QFT pass: the compiled kernel for 2^12-amplitude tiles, else
// the general tile program.
static bool qft_c128_compiled(const TileProg<double>& P) {
  return P.k + P.c == 12 && P.scale_p == P.k && P.nops == P.k && ((P.k >= 3 && P.k <= 9) || P.k == 12);
}

// ld_ff / st_ff: the pass reads / leaves the double-float form (compiled
// passes only; the transform's first pass reads IEEE doubles, and the bit
// reversal after its last pass converts back).
static qc_status run_qft_c128(qc_state* s, TileProg<double>& P, const double2* tlo, const double2* thi, bool ld_ff,
                              bool st_ff) {
  P.n = s->n;
  if (qft_c128_compiled(P)) {
    const uint64_t ntiles = 1ull << (s->n - 12);
    const size_t smem = sizeof(ffc) * (((size_t)1 << 12) + (size_t)lad_entries<double>(P.k));
    double2* d = reinterpret_cast<double2*>(s->data);
    switch (P.k) {
#define QC_QFT_C128(KK)                                                                             \
  case KK: {                                                                                        \
    static bool a = false;                                                                          \
    if (!a) {                                                                                       \
      cudaFuncSetAttribute(k_qft_c128_k<KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); \
      a = true;                                                                                     \
    }                                                                                               \
    const unsigned g = resident_grid(k_qft_c128_k<KK>, 512, (int64_t)ntiles, 1, smem);             \
    k_qft_c128_k<KK><<<g, 512, smem, s->stream>>>(d, ntiles, P, tlo, thi, ld_ff, st_ff);            \
    return check_launch("qft pass");                                                                \
  }
      QC_QFT_C128(3) QC_QFT_C128(4) QC_QFT_C128(5) QC_QFT_C128(6) QC_QFT_C128(7) QC_QFT_C128(8)
      QC_QFT_C128(9) QC_QFT_C128(12)
#undef QC_QFT_C128
      default: break;
    }
  }
  if (ld_ff || st_ff) return QC_EINVAL;
  return run_tile<double>(s, P, tlo, thi);
}

// complex64 QFT pass through the double-buffered kernel: two tile buffers
// plus the pass's tables.
static size_t qft_db_smem(int k, int c, bool twiddle) {
  const size_t NE = (size_t)1 << (k + c);
  return sizeof(float2) * (2 * NE + (twiddle ? NE + ((size_t)1 << k) : 0) + ((size_t)1 << k) - 1);
}

static qc_status run_qft_db_c64(qc_state* s, TileProg<float>& P, const float2* tlo, const float2* thi) {
  P.n = s->n;
  const uint64_t ntiles = 1ull << (s->n - (P.k + P.c));
  const size_t smem = qft_db_smem(P.k, P.c, P.twiddle != 0);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_qft_db_c64, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_set = true;
  }
  float2* d = reinterpret_cast<float2*>(s->data);
  // 2^13-amplitude tiles (states of at least 13 qubits): the compile-time kernels
  if (P.k + P.c == 13 && P.c == 13 - P.k && P.scale_p == P.k) {
    switch (P.k) {
#define QC_QFT_DB(KK)                                                                              \
  case KK: {                                                                                       \
    static bool a = false;                                                                         \
    if (!a) {                                                                                      \
      cudaFuncSetAttribute(k_qft_db_c64_k<KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024); \
      a = true;                                                                                    \
    }                                                                                              \
    const unsigned g = resident_grid(k_qft_db_c64_k<KK>, 512, (int64_t)ntiles, 1, smem);          \
    k_qft_db_c64_k<KK><<<g, 512, smem, s->stream>>>(d, ntiles, P, tlo, thi);                       \
    return check_launch("qft pass");                                                               \
  }
      QC_QFT_DB(3) QC_QFT_DB(4) QC_QFT_DB(5) QC_QFT_DB(6) QC_QFT_DB(7) QC_QFT_DB(8) QC_QFT_DB(9) QC_QFT_DB(13)
#undef QC_QFT_DB
      default: break;
    }
  }
  const unsigned grid = resident_grid(k_qft_db_c64, 512, (int64_t)ntiles, 1, smem);
  k_qft_db_c64<<<grid, 512, smem, s->stream>>>(d, ntiles, P, tlo, thi);
  return check_launch("qft pass");
}

// Contiguous low bits of a group's tile: at least C (128-byte rows) and, for
// small groups, enough to fill the tile to 2^TB amplitudes, so that a pass
// has few large tiles with long rows rather than many small ones (each tile
// costs a DRAM round trip before its compute).  TB: 64 KiB tiles (two CTAs
// per SM; the complex64 QFT kernel holds two of them in one CTA).  The QFT
// twiddle tables need c + k <= 14.
template <typename R>
static int tile_c(const Group& g) {
  const int TB = sizeof(R) == 8 ? 12 : 13;
  return std::min(g.lo, std::max(TileCfg<R>::C, TB - g.k));
}

template <typename R>
static void prog_init(TileProg<R>& P, const Group& g, int n) {
  P.nops = 0;
  P.lo = g.lo;
  P.k = g.k;
  P.c = tile_c<R>(g);
  P.n = n;
  P.twiddle = 0;
  P.qft = 0;
  P.nl = 0;
  P.scale_p = 0;
}

// Hadamards (operators that are exactly h [[1,1],[1,-1]] with h = 1/sqrt 2)
// become unnormalised butterflies with the scale deferred to the store.
static bool is_exact_hadamard(const double* u) {
  const double h = 1.0 / sqrt(2.0);
  return u[0] == h && u[2] == h && u[4] == h && u[6] == -h && u[1] == 0 && u[3] == 0 && u[5] == 0 && u[7] == 0;
}

template <typename R>
static qc_status layer_impl(qc_state* s, const double* U, uint64_t mask) {
  for (const Group& g : plan_groups<R>(s->n)) {
    TileProg<R> P;
    prog_init(P, g, s->n);
    for (int j = 0; j < g.k; ++j) {
      const int q = g.lo + j;
      if (!((mask >> q) & 1)) continue;
      const MatKind mk = classify(U + 8 * q);
      if (mk == MK_IDENT) continue;
      P.q[P.nops] = (int8_t)j;
      if (is_exact_hadamard(U + 8 * q)) {
        P.kind[P.nops] = TOP_HB;
        P.mk[P.nops] = 0;
        ++P.scale_p;
      } else {
        P.kind[P.nops] = TOP_U2;
        P.mk[P.nops] = (int8_t)mk;
        P.U[P.nops] = TA<R>::mat(U + 8 * q);
      }
      ++P.nops;
    }
    qc_status st = run_tile<R>(s, P, nullptr, nullptr);
    if (st) return st;
  }
  return QC_OK;
}

qc_status launch_layer(qc_state* s, const double* U, uint64_t mask) {
  s->sum_valid = false;
  // a layer of Hadamards only (HALL among them): Walsh-Hadamard passes
  bool all_h = mask != 0;
  for (int q = 0; q < s->n && all_h; ++q)
    if ((mask >> q) & 1) all_h = is_exact_hadamard(U + 8 * q);
  if (all_h && s->n >= hadamard_layer_min_qubits(s->dt)) return launch_hadamard_layer(s, mask);
  return s->dt == QC_C128 ? layer_impl<double>(s, U, mask) : layer_impl<float>(s, U, mask);
}

qc_status launch_hall(qc_state* s) {
  std::vector<double> U(8 * (size_t)s->n);
  const double h = 1.0 / sqrt(2.0);
  for (int q = 0; q < s->n; ++q) {
    double* u = U.data() + 8 * q;
    const double v[8] = {h, 0, h, 0, h, 0, -h, 0};
    for (int i = 0; i < 8; ++i) u[i] = v[i];
  }
  const uint64_t mask = (s->n >= 64) ? ~0ull : ((1ull << s->n) - 1ull);
  return launch_layer(s, U.data(), mask);
}

// ------------------------------------------------------- bit reversal ----
// In-place reversal of all n index bits.  Index = (h, m, l) with h, l of B
// bits: rev(h, m, l) = (rev l, rev m, rev h).  The block for middle value m
// (with m <= rev m) exchanges the 2^B x 2^B tiles of m and rev m through
// shared memory (rows of 2^B contiguous amplitudes, padded against bank
// conflicts).  The pass is latency bound (load both tiles, synchronise,
// store), so many small blocks beat few large ones: complex128 runs B = 4
// with 128 threads (twelve blocks per SM; 0.76 of copy bandwidth on GB300
// at 30 qubits, against 0.63 for B = 5 with 256 threads); complex64 keeps
// B = 5 with 256 threads (rows of 256 bytes).
template <typename V2, bool FF>
__device__ __forceinline__ V2 bitrev_out(V2 v) {
  if constexpr (FF) {
    const ffc z = ffc_unpack(v);
    return make_double2(ff_to_d_fast(z.re), ff_to_d_fast(z.im));
  } else {
    return v;
  }
}

// FF (complex128 only): the input holds double-float parts (the form the
// compiled QFT passes leave) and is converted to IEEE double on the way.
template <typename R, int B, int T, bool FF = false>
__global__ void __launch_bounds__(T) k_bitrev(typename CT<R>::V2* __restrict__ s, int n) {
  using V2 = typename CT<R>::V2;
  static_assert(!FF || sizeof(R) == 8, "double-float input is complex128");
  constexpr int W = 1 << B, WP = W + 1, PER = W * W / T;
  static_assert(PER * T == W * W, "whole tiles per block");
  extern __shared__ __align__(16) unsigned char smraw[];
  V2* A = reinterpret_cast<V2*>(smraw);
  V2* Bt = A + W * WP;
  const int nm = n - 2 * B;
  const uint64_t M = 1ull << nm;
  for (uint64_t m = blockIdx.x; m < M; m += gridDim.x) {
    const uint64_t mr = nm ? (__brevll((unsigned long long)m) >> (64 - nm)) : 0ull;
    if (mr < m) continue;
    // every load of both tiles in flight before the first shared-memory store
    {
      V2 va[PER], vb[PER];
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * T;
        const int h = e >> B, l = e & (W - 1);
        va[u] = s[((uint64_t)h << (n - B)) | (m << B) | (uint64_t)l];
        if (mr != m) vb[u] = s[((uint64_t)h << (n - B)) | (mr << B) | (uint64_t)l];
      }
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * T;
        const int h = e >> B, l = e & (W - 1);
        A[h * WP + l] = va[u];
        if (mr != m) Bt[h * WP + l] = vb[u];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < W * W; e += T) {
      const int h = e >> B, l = e & (W - 1);
      const int rl = (int)(__brev((unsigned)l) >> (32 - B)), rh = (int)(__brev((unsigned)h) >> (32 - B));
      // element (h, m, l) of the output is the input at rev(h, m, l)
      if (mr != m) {
        s[((uint64_t)h << (n - B)) | (m << B) | (uint64_t)l] = bitrev_out<V2, FF>(Bt[rl * WP + rh]);
        s[((uint64_t)h << (n - B)) | (mr << B) | (uint64_t)l] = bitrev_out<V2, FF>(A[rl * WP + rh]);
      } else {
        s[((uint64_t)h << (n - B)) | (m << B) | (uint64_t)l] = bitrev_out<V2, FF>(A[rl * WP + rh]);
      }
    }
    __syncthreads();
  }
}

// Small states: the whole vector through shared memory, one block.
template <typename R>
__global__ void k_bitrev_small(typename CT<R>::V2* __restrict__ s, int n) {
  using V2 = typename CT<R>::V2;
  extern __shared__ __align__(16) unsigned char smraw[];
  V2* A = reinterpret_cast<V2*>(smraw);
  const int N = 1 << n;
  for (int i = threadIdx.x; i < N; i += blockDim.x) A[i] = s[i];
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int r = n ? (int)(__brev((unsigned)i) >> (32 - n)) : 0;
    s[i] = A[r];
  }
}

template <typename R>
static qc_status bitrev_impl(qc_state* s, bool from_ff = false) {
  using V2 = typename CT<R>::V2;
  V2* d = reinterpret_cast<V2*>(s->data);
  const int n = s->n;
  constexpr int b = sizeof(R) == 8 ? 4 : 5, T = sizeof(R) == 8 ? 128 : 256;
  if (n < 2 * b) {
    if (from_ff) return QC_EINVAL;
    k_bitrev_small<R><<<1, 256, sizeof(V2) << n, s->stream>>>(d, n);
    return check_launch("bitrev small");
  }
  const size_t smem = 2 * (size_t)(1 << b) * ((1 << b) + 1) * sizeof(V2);
  const uint64_t M = 1ull << (n - 2 * b);
  if constexpr (sizeof(R) == 8) {
    if (from_ff) {
      const unsigned grid = resident_grid(k_bitrev<R, b, T, true>, T, (int64_t)M, 1, smem);
      k_bitrev<R, b, T, true><<<grid, T, smem, s->stream>>>(d, n);
      return check_launch("bitrev");
    }
  }
  if (from_ff) return QC_EINVAL;
  const unsigned grid = resident_grid(k_bitrev<R, b, T>, T, (int64_t)M, 1, smem);
  k_bitrev<R, b, T><<<grid, T, smem, s->stream>>>(d, n);
  return check_launch("bitrev");
}

template <typename R>
static qc_status qft_impl(qc_state* s) {
  using V2 = typename CT<R>::V2;
  const int n = s->n;
  const int nl = (n + 1) / 2;
  const size_t tbytes = (((size_t)1 << nl) + ((size_t)1 << (n - nl))) * sizeof(V2);
  V2* tab = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&tab, tbytes, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "qft tables");
  V2* tlo = tab;
  V2* thi = tab + ((size_t)1 << nl);
  {
    const uint64_t tot = (1ull << nl) + (1ull << (n - nl));
    k_roots<R><<<grid_for(tot, 256, 4), 256, 0, s->stream>>>(tlo, thi, n, nl);
  }
  qc_status st = check_launch("qft roots");
  // complex64: groups of at most 9 above the lowest 13 (64 KiB tiles)
  std::vector<Group> groups = sizeof(R) == 4 ? plan_groups_k(n, 13, 9) : plan_groups<R>(n);
  std::vector<TileProg<R>> progs(groups.size());
  bool all_compiled = true;  // complex128: double-float form between the passes
  for (int gi = (int)groups.size() - 1; gi >= 0; --gi) {
    const Group& g = groups[gi];
    TileProg<R>& P = progs[gi];
    prog_init(P, g, n);
    P.nl = nl;
    P.qft = 1;
    for (int j = g.k - 1; j >= 0; --j) {
      P.kind[P.nops] = TOP_QFTLEVEL;
      P.q[P.nops] = (int8_t)j;
      P.mk[P.nops] = 0;
      ++P.nops;
    }
    P.scale_p = g.k;
    P.twiddle = g.lo > 0;
    if constexpr (sizeof(R) == 8) all_compiled = all_compiled && qft_c128_compiled(P);
  }
  for (int gi = (int)groups.size() - 1; gi >= 0 && !st; --gi) {
    if constexpr (sizeof(R) == 4) st = run_qft_db_c64(s, progs[gi], tlo, thi);
    else
      st = run_qft_c128(s, progs[gi], tlo, thi, all_compiled && gi + 1 < (int)groups.size(), all_compiled);
  }
  // the bit reversal converts the complex128 passes' double-float form back
  if (!st) st = bitrev_impl<R>(s, sizeof(R) == 8 && all_compiled);
  cudaFreeAsync(tab, s->stream);
  return st;
}

qc_status launch_qft(qc_state* s) {
  s->sum_valid = false;
  return s->dt == QC_C128 ? qft_impl<double>(s) : qft_impl<float>(s);
}

}  // namespace qc
