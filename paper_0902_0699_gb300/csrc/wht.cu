// Hadamard layers (HALL, Eq. HALL, and any layer whose operators on a tile
// group are all Hadamards) as Walsh-Hadamard tile passes.
//
// A Hadamard layer on the bits B of a tile is the unnormalised butterfly
// (a0 + a1, a0 - a1) on every bit of B followed by one scaling by
// 2^{-|B|/2}.  Only additions are needed, so:
//  - complex128 tiles run in exact 64-bit fixed point.  The tile's largest
//    exponent fixes the binary point so that |B| doublings cannot overflow
//    (|v| < 2^62); the conversion rounds every value to nearest (half away
//    from zero) at 2^-51 of the tile's largest magnitude or better, the
//    butterflies are exact integer additions, and the result is rounded
//    once, to nearest, back to binary64 (odd |B|: one fixed-point product
//    by 1/sqrt 2 before that).  No FP64 instruction is issued; GB300's FP64 pipe would
//    otherwise bound the pass, and double-float butterflies cost about 20
//    FP32 operations per addition.
//  - complex64 tiles run in FP32.
// A CTA stages 2^(k+c) amplitudes (the group's k qubits times the c lowest
// index bits kept contiguous, as in tile.cu) and applies the butterflies in
// register blocks of 2^RB elements per thread (radix 8 for complex128,
// radix 16 for complex64) between shared-memory round trips.  The shared
// tile is XOR-swizzled within 128-byte rows so that the strided register
// blocks on the lowest bits are free of bank conflicts.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace qc {

#define WHT_T 512
#define WHT_MAXBITS 16

struct WhtProg {
  int lo, k, c;              // group [lo, lo+k), c low contiguous index bits (c <= lo)
  int nb;                    // butterfly bits (tile bit positions, ascending)
  int8_t bits[WHT_MAXBITS];
  long long rsqrt2;          // floor(2^62.5): the fixed-point factor 1/sqrt 2 (scaled by 2^63)
};

__device__ __forceinline__ uint64_t wht_global(uint64_t e, uint64_t T, int lo, int k, int c) {
  const uint64_t cm = (1ull << c) - 1ull;
  const uint64_t tmid = T & ((1ull << (lo - c)) - 1ull);
  const uint64_t thi = T >> (lo - c);
  return (e & cm) | (tmid << c) | ((e >> c) << lo) | (thi << (lo + k));
}

// ---------------------------------------------------------- complex128 --
// binary64 -> fixed point round(x 2^(1075 - G)) for the tile's G (see
// k_wht_c128), rounding half away from zero (symmetric, so unbiased; exact
// values need no rounding at all).  x = m 2^(ex - 1075), so the value is
// m 2^(ex - G).
__device__ __forceinline__ long long d2fix(double x, int G) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FFu);
  if (ex == 0) return 0;  // zero or subnormal (below 2^-1022): dropped
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = ex - G;
  unsigned long long v;
  if (sh >= 0) {
    v = m << sh;  // sh <= 9 - |B|: no overflow
  } else {
    const int r = -sh;
    v = r > 54 ? 0ull : ((m >> (r - 1)) + 1ull) >> 1;
  }
  return (b >> 63) ? -(long long)v : (long long)v;
}

// fixed point v 2^-F -> binary64, rounded half away from zero (results
// below 2^-1022 flush to zero)
__device__ __forceinline__ double fix2d(long long v, int F) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  unsigned long long keep = (((a << lz) >> 10) + 1ull) >> 1;  // 53 bits, rounded
  int e = 63 - lz - F + 1023;
  if (keep >> 53) {
    keep >>= 1;
    ++e;
  }
  if (e <= 0) return __longlong_as_double((long long)sgn);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)e << 52) | (keep & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ int sw16(int e) { return e ^ ((e >> 3) & 7); }  // 16-byte elements, 8 per 128 B

template <int RB>
__device__ __forceinline__ void bfly_regs(longlong2* a) {
  constexpr int NR = 1 << RB;
#pragma unroll
  for (int lv = 0; lv < RB; ++lv)
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      if ((i >> lv) & 1) continue;
      const int j = i | (1 << lv);
      const longlong2 x = a[i], y = a[j];
      a[i] = make_longlong2(x.x + y.x, x.y + y.y);
      a[j] = make_longlong2(x.x - y.x, x.y - y.y);
    }
}

// Butterflies on tile bits bits[b0 .. b0+r) (ascending positions), r <= 3:
// thread p takes the 2^r elements of index p with zeros inserted there.
template <int RB>
__device__ __forceinline__ void wht_chunk_c128(longlong2* sm, int NE, const int8_t* bits, int b0) {
  constexpr int NR = 1 << RB;
  for (int p = threadIdx.x; p < (NE >> RB); p += blockDim.x) {
    int base = p;
#pragma unroll
    for (int i = 0; i < RB; ++i) base = (int)insert0((uint64_t)base, bits[b0 + i]);
    longlong2 a[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      int e = base;
#pragma unroll
      for (int i = 0; i < RB; ++i) e |= ((j >> i) & 1) << bits[b0 + i];
      a[j] = sm[sw16(e)];
    }
    bfly_regs<RB>(a);
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      int e = base;
#pragma unroll
      for (int i = 0; i < RB; ++i) e |= ((j >> i) & 1) << bits[b0 + i];
      sm[sw16(e)] = a[j];
    }
  }
}

// 2^12 amplitudes per tile (64 KiB), 512 threads, two CTAs per SM.
__global__ void __launch_bounds__(WHT_T, 2) k_wht_c128(double2* __restrict__ s, uint64_t ntiles, const __grid_constant__ WhtProg P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  longlong2* sm = reinterpret_cast<longlong2*>(smraw);
  __shared__ int wmax[WHT_T / 32];
  __shared__ int8_t bits[WHT_MAXBITS];
  if (threadIdx.x < WHT_MAXBITS) bits[threadIdx.x] = P.bits[threadIdx.x];  // read after the first barrier
  const int NE = 1 << (P.k + P.c);
  constexpr int PER = 8;  // elements per thread at load / store (NE = 4096)
  const int L = P.nb;
  for (uint64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
    double2 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * WHT_T;
      v[u] = e < NE ? s[wht_global(e, T, P.lo, P.k, P.c)] : make_double2(0.0, 0.0);
    }
    // the tile's largest binary exponent
    int em = 0;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      em = max(em, (int)((__double_as_longlong(v[u].x) >> 52) & 0x7FF));
      em = max(em, (int)((__double_as_longlong(v[u].y) >> 52) & 0x7FF));
    }
    for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = em;
    __syncthreads();
    em = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) em = max(em, wmax[w]);
    // |x| < 2^(em - 1022); scaled by 2^(1075 - G) with G = em + L - 9 the
    // values stay below 2^(62 - L), so L doublings stay below 2^62
    const int G = em + L - 9;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * WHT_T;
      if (e < NE) sm[sw16(e)] = make_longlong2(d2fix(v[u].x, G), d2fix(v[u].y, G));
    }
    __syncthreads();
    int b0 = 0;
    for (; b0 + 3 <= L; b0 += 3) {
      wht_chunk_c128<3>(sm, NE, bits, b0);
      __syncthreads();
    }
    if (L - b0 == 2) {
      wht_chunk_c128<2>(sm, NE, bits, b0);
      __syncthreads();
    } else if (L - b0 == 1) {
      wht_chunk_c128<1>(sm, NE, bits, b0);
      __syncthreads();
    }
    // value = v 2^(G - 1075) 2^(-L/2); odd L: v / sqrt 2 in fixed point first
    // (one bit of the headroom is spent: |v| < 2^62 before, < 2^62 after)
    const int F = 1075 - G + L / 2;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * WHT_T;
      if (e < NE) {
        longlong2 z = sm[sw16(e)];
        if (L & 1) {
          z.x = __mul64hi(z.x, P.rsqrt2) << 1;
          z.y = __mul64hi(z.y, P.rsqrt2) << 1;
        }
        s[wht_global(e, T, P.lo, P.k, P.c)] = make_double2(fix2d(z.x, F), fix2d(z.y, F));
      }
    }
    __syncthreads();  // the tile is read before the next one is staged
  }
}

// ----------------------------------------------------------- complex64 --
__device__ __forceinline__ int sw8(int e) { return e ^ ((e >> 4) & 15); }  // 8-byte elements, 16 per 128 B

template <int RB>
__device__ __forceinline__ void wht_chunk_c64(float2* sm, int NE, const int8_t* bits, int b0) {
  constexpr int NR = 1 << RB;
  for (int p = threadIdx.x; p < (NE >> RB); p += blockDim.x) {
    int base = p;
#pragma unroll
    for (int i = 0; i < RB; ++i) base = (int)insert0((uint64_t)base, bits[b0 + i]);
    float2 a[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      int e = base;
#pragma unroll
      for (int i = 0; i < RB; ++i) e |= ((j >> i) & 1) << bits[b0 + i];
      a[j] = sm[sw8(e)];
    }
#pragma unroll
    for (int lv = 0; lv < RB; ++lv)
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        if ((i >> lv) & 1) continue;
        const int j = i | (1 << lv);
        const float2 x = a[i], y = a[j];
        a[i] = make_float2(x.x + y.x, x.y + y.y);
        a[j] = make_float2(x.x - y.x, x.y - y.y);
      }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      int e = base;
#pragma unroll
      for (int i = 0; i < RB; ++i) e |= ((j >> i) & 1) << bits[b0 + i];
      sm[sw8(e)] = a[j];
    }
  }
}

// 2^13 amplitudes per tile (64 KiB), 512 threads, two CTAs per SM.
__global__ void __launch_bounds__(WHT_T, 2) k_wht_c64(float2* __restrict__ s, uint64_t ntiles, const __grid_constant__ WhtProg P,
                                                      float scale) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  __shared__ int8_t bits[WHT_MAXBITS];
  if (threadIdx.x < WHT_MAXBITS) bits[threadIdx.x] = P.bits[threadIdx.x];  // read after the first barrier
  const int NE = 1 << (P.k + P.c);
  constexpr int PER = 16;  // NE = 8192
  const int L = P.nb;
  for (uint64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
    float2 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * WHT_T;
      v[u] = e < NE ? s[wht_global(e, T, P.lo, P.k, P.c)] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * WHT_T;
      if (e < NE) sm[sw8(e)] = v[u];
    }
    __syncthreads();
    int b0 = 0;
    for (; b0 + 4 <= L; b0 += 4) {
      wht_chunk_c64<4>(sm, NE, bits, b0);
      __syncthreads();
    }
    switch (L - b0) {
      case 3: wht_chunk_c64<3>(sm, NE, bits, b0); __syncthreads(); break;
      case 2: wht_chunk_c64<2>(sm, NE, bits, b0); __syncthreads(); break;
      case 1: wht_chunk_c64<1>(sm, NE, bits, b0); __syncthreads(); break;
      default: break;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * WHT_T;
      if (e < NE) {
        const float2 z = sm[sw8(e)];
        s[wht_global(e, T, P.lo, P.k, P.c)] = make_float2(z.x * scale, z.y * scale);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------ whole-group layers ----
// The common case (HALL among them): every qubit of the group is
// butterflied, i.e. the top L bits of the 2^TB-element tile.  The bit
// positions are then compile-time, and the shared tile is padded (one
// element after every 128 bytes) instead of swizzled: an element's address
// pad(e) = e + (e >> r) is additive over disjoint index bits, so every
// element of a register block is the thread's base address plus a constant
// offset, and blocks of elements 2^b apart still hit distinct bank groups.
// The global addresses of a thread's PER elements are one base plus
// multiples of a per-pass stride.
template <int SH>
__host__ __device__ __forceinline__ int padded(int e) { return e + (e >> SH); }

// insert RB zero bits at position B0 of p
template <int B0, int RB>
__device__ __forceinline__ int ins_bits(int p) {
  return ((p >> B0) << (B0 + RB)) | (p & ((1 << B0) - 1));
}

template <int TB, int B0, int RB>
__device__ __forceinline__ void wht_block_c128(longlong2* sm) {
  constexpr int NR = 1 << RB;
  for (int p = threadIdx.x; p < ((1 << TB) >> RB); p += WHT_T) {
    const int base = padded<3>(ins_bits<B0, RB>(p));
    longlong2 a[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) a[j] = sm[base + padded<3>(j << B0)];
    bfly_regs<RB>(a);
#pragma unroll
    for (int j = 0; j < NR; ++j) sm[base + padded<3>(j << B0)] = a[j];
  }
}

template <int L>
__global__ void __launch_bounds__(WHT_T, 2) k_wht_c128_top(double2* __restrict__ s, uint64_t ntiles, int lo, int k,
                                                            int c, long long rsqrt2) {
  constexpr int TB = 12, NE = 1 << TB, PER = NE / WHT_T;
  extern __shared__ __align__(16) unsigned char smraw[];
  longlong2* sm = reinterpret_cast<longlong2*>(smraw);
  __shared__ int wmax[WHT_T / 32];
  const int tid = threadIdx.x;
  const uint64_t gstep = c <= 9 ? ((uint64_t)(WHT_T >> c) << lo) : 0;
  const int st = padded<3>(tid);
  for (uint64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
    const uint64_t g0 = wht_global((uint64_t)tid, T, lo, k, c);
    double2 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u)
      v[u] = s[c <= 9 ? g0 + u * gstep : wht_global((uint64_t)(tid + u * WHT_T), T, lo, k, c)];
    int em = 0;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      em = max(em, (int)((__double_as_longlong(v[u].x) >> 52) & 0x7FF));
      em = max(em, (int)((__double_as_longlong(v[u].y) >> 52) & 0x7FF));
    }
    for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
    if ((tid & 31) == 0) wmax[tid >> 5] = em;
    __syncthreads();
    em = 0;
#pragma unroll
    for (int w = 0; w < WHT_T / 32; ++w) em = max(em, wmax[w]);
    const int G = em + L - 9;  // as in k_wht_c128: L doublings stay below 2^62
    // a thread's eight elements tid + 512 u differ exactly in the top three
    // tile bits: their butterflies run in registers before the first store
    longlong2 a[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) a[u] = make_longlong2(d2fix(v[u].x, G), d2fix(v[u].y, G));
    bfly_regs<3>(a);
#pragma unroll
    for (int u = 0; u < PER; ++u) sm[st + u * padded<3>(WHT_T)] = a[u];
    __syncthreads();
    // the other blocks of three bits from the top: [TB-6, TB-3), [TB-9, TB-6), ...
    if constexpr (L >= 6) { wht_block_c128<TB, TB - 6, 3>(sm); __syncthreads(); }
    if constexpr (L >= 9) { wht_block_c128<TB, TB - 9, 3>(sm); __syncthreads(); }
    if constexpr (L >= 12) { wht_block_c128<TB, TB - 12, 3>(sm); __syncthreads(); }
    if constexpr (L % 3 == 2) { wht_block_c128<TB, TB - L, 2>(sm); __syncthreads(); }
    if constexpr (L % 3 == 1) { wht_block_c128<TB, TB - L, 1>(sm); __syncthreads(); }
    const int F = 1075 - G + L / 2;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      longlong2 z = sm[st + u * padded<3>(WHT_T)];
      if (L & 1) {
        z.x = __mul64hi(z.x, rsqrt2) << 1;
        z.y = __mul64hi(z.y, rsqrt2) << 1;
      }
      s[c <= 9 ? g0 + u * gstep : wht_global((uint64_t)(tid + u * WHT_T), T, lo, k, c)] =
          make_double2(fix2d(z.x, F), fix2d(z.y, F));
    }
    __syncthreads();  // the tile is read before the next one is staged
  }
}

template <int TB, int B0, int RB>
__device__ __forceinline__ void wht_block_c64(float2* sm) {
  constexpr int NR = 1 << RB;
  for (int p = threadIdx.x; p < ((1 << TB) >> RB); p += WHT_T) {
    const int base = padded<4>(ins_bits<B0, RB>(p));
    float2 a[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) a[j] = sm[base + padded<4>(j << B0)];
#pragma unroll
    for (int lv = 0; lv < RB; ++lv)
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        if ((i >> lv) & 1) continue;
        const int j = i | (1 << lv);
        const float2 x = a[i], y = a[j];
        a[i] = make_float2(x.x + y.x, x.y + y.y);
        a[j] = make_float2(x.x - y.x, x.y - y.y);
      }
#pragma unroll
    for (int j = 0; j < NR; ++j) sm[base + padded<4>(j << B0)] = a[j];
  }
}

template <int L>
__global__ void __launch_bounds__(WHT_T, 2) k_wht_c64_top(float2* __restrict__ s, uint64_t ntiles, int lo, int k, int c,
                                                           float scale) {
  constexpr int TB = 13, NE = 1 << TB, PER = NE / WHT_T;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int tid = threadIdx.x;
  const uint64_t gstep = c <= 9 ? ((uint64_t)(WHT_T >> c) << lo) : 0;
  const int st = padded<4>(tid);
  for (uint64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
    const uint64_t g0 = wht_global((uint64_t)tid, T, lo, k, c);
    float2 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u)
      v[u] = s[c <= 9 ? g0 + u * gstep : wht_global((uint64_t)(tid + u * WHT_T), T, lo, k, c)];
    // a thread's sixteen elements tid + 512 u differ exactly in the top four
    // tile bits: their butterflies run in registers before the first store
#pragma unroll
    for (int lv = 0; lv < 4; ++lv)
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        if ((i >> lv) & 1) continue;
        const int j = i | (1 << lv);
        const float2 x = v[i], y = v[j];
        v[i] = make_float2(x.x + y.x, x.y + y.y);
        v[j] = make_float2(x.x - y.x, x.y - y.y);
      }
#pragma unroll
    for (int u = 0; u < PER; ++u) sm[st + u * padded<4>(WHT_T)] = v[u];
    __syncthreads();
    // the other blocks of four bits from the top
    if constexpr (L >= 8) { wht_block_c64<TB, TB - 8, 4>(sm); __syncthreads(); }
    if constexpr (L >= 12) { wht_block_c64<TB, TB - 12, 4>(sm); __syncthreads(); }
    if constexpr (L % 4 == 3) { wht_block_c64<TB, TB - L, 3>(sm); __syncthreads(); }
    if constexpr (L % 4 == 2) { wht_block_c64<TB, TB - L, 2>(sm); __syncthreads(); }
    if constexpr (L % 4 == 1) { wht_block_c64<TB, TB - L, 1>(sm); __syncthreads(); }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const float2 z = sm[st + u * padded<4>(WHT_T)];
      s[c <= 9 ? g0 + u * gstep : wht_global((uint64_t)(tid + u * WHT_T), T, lo, k, c)] =
          make_float2(z.x * scale, z.y * scale);
    }
    __syncthreads();
  }
}

template <typename K>
static void wht_top_attr(K kernel, size_t smem) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Launch the whole-group kernel for L = k butterfly bits (L <= TB); false if
// this L has no instantiation.
static bool launch_wht_top_c128(qc_state* s, int L, uint64_t ntiles, int lo, int k, int c, long long rsqrt2) {
  const size_t smem = (size_t)padded<3>(1 << 12) * 16;
  double2* d = reinterpret_cast<double2*>(s->data);
#define QC_WHT_C128(LL)                                                                            \
  case LL: {                                                                                       \
    static bool a = false;                                                                         \
    if (!a) {                                                                                      \
      wht_top_attr(k_wht_c128_top<LL>, smem);                                                      \
      a = true;                                                                                    \
    }                                                                                              \
    const unsigned grid = resident_grid(k_wht_c128_top<LL>, WHT_T, (int64_t)ntiles, 1, smem);      \
    k_wht_c128_top<LL><<<grid, WHT_T, smem, s->stream>>>(d, ntiles, lo, k, c, rsqrt2);             \
    return true;                                                                                   \
  }
  switch (L) {
    QC_WHT_C128(3) QC_WHT_C128(4) QC_WHT_C128(5) QC_WHT_C128(6) QC_WHT_C128(7) QC_WHT_C128(8)
    QC_WHT_C128(9) QC_WHT_C128(10) QC_WHT_C128(12)
    default: return false;
  }
#undef QC_WHT_C128
}

static bool launch_wht_top_c64(qc_state* s, int L, uint64_t ntiles, int lo, int k, int c, float scale) {
  const size_t smem = (size_t)padded<4>(1 << 13) * 8;
  float2* d = reinterpret_cast<float2*>(s->data);
#define QC_WHT_C64(LL)                                                                             \
  case LL: {                                                                                       \
    static bool a = false;                                                                         \
    if (!a) {                                                                                      \
      wht_top_attr(k_wht_c64_top<LL>, smem);                                                       \
      a = true;                                                                                    \
    }                                                                                              \
    const unsigned grid = resident_grid(k_wht_c64_top<LL>, WHT_T, (int64_t)ntiles, 1, smem);       \
    k_wht_c64_top<LL><<<grid, WHT_T, smem, s->stream>>>(d, ntiles, lo, k, c, scale);               \
    return true;                                                                                   \
  }
  switch (L) {
    QC_WHT_C64(4) QC_WHT_C64(5) QC_WHT_C64(6) QC_WHT_C64(7) QC_WHT_C64(8) QC_WHT_C64(9) QC_WHT_C64(10)
    QC_WHT_C64(13)
    default: return false;
  }
#undef QC_WHT_C64
}

// --------------------------------------------------------------- host ----
// floor(2^62.5) = floor(sqrt(2^125)) by integer Newton iteration (exact).
static long long rsqrt2_fixed() {
  static long long c = 0;
  if (!c) {
    const unsigned __int128 N = (unsigned __int128)1 << 125;
    unsigned __int128 x = (unsigned __int128)1 << 63;  // >= sqrt(N)
    for (;;) {
      const unsigned __int128 y = (x + N / x) >> 1;
      if (y >= x) break;
      x = y;
    }
    c = (long long)x;
  }
  return c;
}

// Groups of qubits for the Hadamard passes: the lowest one 2^TB amplitudes
// wide (no contiguous bits needed), the others up to TB - C qubits with at
// least C contiguous low index bits (rows of at least 64 bytes; a group of
// fewer qubits keeps more, up to 128-byte rows and beyond), split evenly
// and into even sizes where the total allows: 30 qubits (complex128) take
// 12 + 10 + 8, 32 qubits (complex64) 13 + 10 + 9.
template <typename R> struct WhtCfg;
template <> struct WhtCfg<double> { static constexpr int TB = 12, C = 2; };
template <> struct WhtCfg<float> { static constexpr int TB = 13, C = 3; };

template <typename R>
static qc_status wht_layer(qc_state* s, uint64_t mask) {
  const int n = s->n, TB = WhtCfg<R>::TB, C = WhtCfg<R>::C;
  struct G {
    int lo, k;
  };
  std::vector<G> groups;
  groups.push_back({0, TB});
  const int rest = n - TB, K = TB - C;  // K even
  if (rest > 0) {
    // balanced sizes, then even ones where the total allows: an even
    // number of butterfly levels scales by an exact power of two, so only
    // an odd total leaves one group with the fixed-point 1/sqrt 2
    const int np = (rest + K - 1) / K;
    std::vector<int> ks(np);
    for (int i = 0, r = rest; i < np; ++i) {
      ks[i] = (r + (np - i) - 1) / (np - i);
      r -= ks[i];
    }
    int odd_seen = -1;
    for (int i = 0; i < np; ++i)
      if (ks[i] & 1) {
        if (odd_seen < 0) {
          odd_seen = i;
        } else {  // two odd sizes (each below K): one up, one down
          ++ks[odd_seen];
          --ks[i];
          odd_seen = -1;
        }
      }
    int lo = TB;
    for (int k : ks) {
      groups.push_back({lo, k});
      lo += k;
    }
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_wht_c128, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_wht_c64, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    attr = true;
  }
  int launches = 0;
  for (const G& g : groups) {
    WhtProg P;
    P.lo = g.lo;
    P.k = g.k;
    P.c = g.lo == 0 ? 0 : std::min(g.lo, TB - g.k);
    P.nb = 0;
    for (int j = 0; j < g.k; ++j)
      if ((mask >> (g.lo + j)) & 1) P.bits[P.nb++] = (int8_t)(P.c + j);
    if (!P.nb) continue;
    P.rsqrt2 = rsqrt2_fixed();
    const uint64_t ntiles = 1ull << (n - g.k - P.c);
    const size_t smem = ((size_t)1 << (g.k + P.c)) * (sizeof(R) * 2 == 16 ? 16 : 8);
    // every qubit of the group butterflied: the compile-time kernels
    if (P.nb == g.k && g.k + P.c == TB) {
      const bool done = sizeof(R) == 8 ? launch_wht_top_c128(s, g.k, ntiles, g.lo, g.k, P.c, P.rsqrt2)
                                       : launch_wht_top_c64(s, g.k, ntiles, g.lo, g.k, P.c,
                                                            (float)std::exp2(-0.5 * P.nb));
      if (done) {
        ++launches;
        continue;
      }
    }
    if constexpr (sizeof(R) == 8) {
      const unsigned grid = resident_grid(k_wht_c128, WHT_T, (int64_t)ntiles, 1, smem);
      k_wht_c128<<<grid, WHT_T, smem, s->stream>>>(reinterpret_cast<double2*>(s->data), ntiles, P);
    } else {
      const float scale = (float)std::exp2(-0.5 * P.nb);
      const unsigned grid = resident_grid(k_wht_c64, WHT_T, (int64_t)ntiles, 1, smem);
      k_wht_c64<<<grid, WHT_T, smem, s->stream>>>(reinterpret_cast<float2*>(s->data), ntiles, P, scale);
    }
    ++launches;
  }
  s->sum_valid = false;
  return check_launch("Hadamard layer (Walsh-Hadamard tiles)", launches);
}

int hadamard_layer_min_qubits(qc_dtype dt) { return dt == QC_C128 ? WhtCfg<double>::TB : WhtCfg<float>::TB; }

// A layer of Hadamards on the qubits of `mask`, for states of at least
// hadamard_layer_min_qubits(dt) qubits.
qc_status launch_hadamard_layer(qc_state* s, uint64_t mask) {
  return s->dt == QC_C128 ? wht_layer<double>(s, mask) : wht_layer<float>(s, mask);
}

}  // namespace qc
