// Fused shared-memory tile passes.
//
// One-qubit operators on distinct pairs are independent (sec. 3, after
// Eq. resmat1), and operators on different qubits commute, so every gate
// acting on a contiguous group of qubits [lo, lo+k) can be applied in one
// pass: a CTA stages a tile -- all 2^k values of the group bits, times the
// 2^c lowest index bits kept contiguous for 128-byte rows -- in shared
// memory, applies the group's gates there, and writes the tile back.
// HALL (Eq. HALL) and layers of one-qubit operators take ceil(n / k)-ish
// passes instead of n.
//
// The QFT circuit of Appendix A processes qubits from the most significant
// down: Hadamard on t, then CPHASEK(t, t') for every lower t' with phase
// e^{2 pi i / 2^{t-t'+1}}.  For a group [lo, hi] the phases with t' inside
// the group are applied right after the group's Hadamard on t (a diagonal
// "ladder"); those with t' < lo commute with the rest of the group's gates
// and are applied at the end of the pass as one twiddle factor
//   exp(2 pi i * L * f / 2^{hi+1}),  L = index bits below lo,
//   f = the group bits in reversed order,
// read from two tables of 2^n-th roots of unity.  The final SWAPs are one
// in-place blocked bit-reversal pass.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace qc {

enum TileOpKind { TOP_U2 = 0, TOP_QFTLEVEL = 1 };
#define QC_TILE_MAXOPS 36

template <typename R> struct TileProg {
  int nops;
  int lo, k, c;   // group [lo, lo+k), c low contiguous bits (c <= lo)
  int n;
  int twiddle;    // apply the QFT cross phase with the bits below lo
  int nl;         // twiddle table split: low table has 2^nl entries
  int8_t kind[QC_TILE_MAXOPS];
  int8_t q[QC_TILE_MAXOPS];   // group-relative qubit
  int8_t mk[QC_TILE_MAXOPS];  // MatKind of a TOP_U2 operator
  Mat2<R> U[QC_TILE_MAXOPS];
};

template <typename R>
__device__ __forceinline__ uint64_t tile_global(uint64_t e, uint64_t T, int lo, int k, int c) {
  const uint64_t cm = (1ull << c) - 1ull;
  const uint64_t tmid = T & ((1ull << (lo - c)) - 1ull);
  const uint64_t thi = T >> (lo - c);
  return (e & cm) | (tmid << c) | ((e >> c) << lo) | (thi << (lo + k));
}

template <typename R, int KIND>
__device__ __forceinline__ void tile_u2(Cx<R>* sm, int E, int b, const Mat2<R>& U) {
  for (int p = threadIdx.x; p < (E >> 1); p += blockDim.x) {
    const int e0 = (int)insert0((uint64_t)p, b), e1 = e0 | (1 << b);
    Cx<R> a0 = sm[e0], a1 = sm[e1];
    apply2<R, KIND>(U, a0, a1);
    sm[e0] = a0;
    sm[e1] = a1;
  }
}

// Root of unity Omega^r, Omega = e^{2 pi i / 2^n}, from the two tables.
template <typename R>
__device__ __forceinline__ Cx<R> omega(const typename CT<R>::V2* __restrict__ tlo,
                                       const typename CT<R>::V2* __restrict__ thi, uint64_t r, int nl) {
  const auto a = tlo[r & ((1ull << nl) - 1ull)];
  const auto b = thi[r >> nl];
  return cmul(cmake<R>(a.x, a.y), cmake<R>(b.x, b.y));
}

template <typename R>
__global__ void __launch_bounds__(512) k_tile(typename CT<R>::V2* __restrict__ s, uint64_t ntiles,
                                              const TileProg<R> P, const typename CT<R>::V2* __restrict__ tlo,
                                              const typename CT<R>::V2* __restrict__ thi) {
  using V2 = typename CT<R>::V2;
  extern __shared__ __align__(16) unsigned char smraw[];
  Cx<R>* sm = reinterpret_cast<Cx<R>*>(smraw);
  const int lo = P.lo, k = P.k, c = P.c;
  const int E = 1 << (k + c);
  for (uint64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
    // load: 16-byte vectors; for complex64 two neighbouring elements (c >= 1
    // or a fully contiguous tile, so e and e+1 are neighbours in memory)
    if (sizeof(R) == 8) {
      for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const V2 v = s[tile_global<R>(e, T, lo, k, c)];
        sm[e] = cmake<R>(v.x, v.y);
      }
    } else {
      for (int e = 2 * threadIdx.x; e < E; e += 2 * blockDim.x) {
        const float4 v = *reinterpret_cast<const float4*>(s + tile_global<R>(e, T, lo, k, c));
        sm[e] = cmake<R>(v.x, v.y);
        sm[e + 1] = cmake<R>(v.z, v.w);
      }
    }
    __syncthreads();
    for (int o = 0; o < P.nops; ++o) {
      const int b = c + P.q[o];
      if (P.kind[o] == TOP_U2) {
        switch (P.mk[o]) {
          case MK_GENERAL: tile_u2<R, MK_GENERAL>(sm, E, b, P.U[o]); break;
          case MK_REAL: tile_u2<R, MK_REAL>(sm, E, b, P.U[o]); break;
          case MK_DIAG: tile_u2<R, MK_DIAG>(sm, E, b, P.U[o]); break;
          case MK_PHASE1: tile_u2<R, MK_PHASE1>(sm, E, b, P.U[o]); break;
          case MK_ANTI: tile_u2<R, MK_ANTI>(sm, E, b, P.U[o]); break;
          case MK_SWAPX: tile_u2<R, MK_SWAPX>(sm, E, b, P.U[o]); break;
          case MK_HAD: tile_u2<R, MK_HAD>(sm, E, b, P.U[o]); break;
          default: break;
        }
      } else {
        // Hadamard on group qubit j, then the ladder phase
        // e^{2 pi i x / 2^{j+1}} on the bit-1 half, x = group bits below j.
        const int j = P.q[o];
        const R h = (R)0.70710678118654752440;
        for (int p = threadIdx.x; p < (E >> 1); p += blockDim.x) {
          const int e0 = (int)insert0((uint64_t)p, b), e1 = e0 | (1 << b);
          const Cx<R> a0 = sm[e0], a1 = sm[e1];
          const R qr = h * a1.re, qi = h * a1.im;
          Cx<R> b1 = cmake<R>(fma(h, a0.re, -qr), fma(h, a0.im, -qi));
          sm[e0] = cmake<R>(fma(h, a0.re, qr), fma(h, a0.im, qi));
          const uint64_t x = (uint64_t)((e0 >> c) & ((1 << j) - 1));
          if (x) b1 = cmul(omega<R>(tlo, thi, x << (P.n - j - 1), P.nl), b1);
          sm[e1] = b1;
        }
      }
      __syncthreads();
    }
    // store (with the QFT cross twiddle when requested)
    const int hi = lo + k - 1;
    if (sizeof(R) == 8) {
      for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const uint64_t g = tile_global<R>(e, T, lo, k, c);
        Cx<R> z = sm[e];
        if (P.twiddle) {
          const uint64_t L = g & ((1ull << lo) - 1ull);
          const uint64_t f = __brevll((unsigned long long)(e >> c)) >> (64 - k);
          const uint64_t r = L * f;  // < 2^{hi+1}
          if (r) z = cmul(omega<R>(tlo, thi, r << (P.n - hi - 1), P.nl), z);
        }
        s[g] = CT<R>::make(z.re, z.im);
      }
    } else {
      for (int e = 2 * threadIdx.x; e < E; e += 2 * blockDim.x) {
        const uint64_t g = tile_global<R>(e, T, lo, k, c);
        Cx<R> z0 = sm[e], z1 = sm[e + 1];
        if (P.twiddle) {
          const uint64_t L = g & ((1ull << lo) - 1ull);
          const uint64_t f0 = __brevll((unsigned long long)(e >> c)) >> (64 - k);
          const uint64_t f1 = __brevll((unsigned long long)((e + 1) >> c)) >> (64 - k);
          const uint64_t r0 = L * f0, r1 = (L + ((c > 0) ? 1 : 0)) * f1;
          if (r0) z0 = cmul(omega<R>(tlo, thi, r0 << (P.n - hi - 1), P.nl), z0);
          if (r1) z1 = cmul(omega<R>(tlo, thi, r1 << (P.n - hi - 1), P.nl), z1);
        }
        *reinterpret_cast<float4*>(s + g) = make_float4(z0.re, z0.im, z1.re, z1.im);
      }
    }
    __syncthreads();
  }
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
// the tile holds 2^{k+c} amplitudes (64 KiB).
template <typename R> struct TileCfg;
template <> struct TileCfg<double> { static constexpr int C = 3, K = 9; };
template <> struct TileCfg<float> { static constexpr int C = 4, K = 9; };

struct Group {
  int lo, k;
};

// Groups covering qubits [0, n): the lowest group holds up to C + K qubits
// (no separate contiguous bits needed), the others up to K.
template <typename R>
static std::vector<Group> plan_groups(int n) {
  const int C = TileCfg<R>::C, K = TileCfg<R>::K;
  std::vector<Group> g;
  const int g0 = std::min(n, C + K);
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
static qc_status run_tile(qc_state* s, TileProg<R>& P, const typename CT<R>::V2* tlo,
                          const typename CT<R>::V2* thi) {
  using V2 = typename CT<R>::V2;
  if (P.nops == 0 && !P.twiddle) return QC_OK;
  P.n = s->n;
  const int tb = P.k + P.c;
  const uint64_t ntiles = 1ull << (s->n - tb);
  const size_t smem = sizeof(Cx<R>) << tb;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_tile<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  const int threads = 512;
  const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)sm_count() * 3);
  k_tile<R><<<grid, threads, smem, s->stream>>>(reinterpret_cast<V2*>(s->data), ntiles, P, tlo, thi);
  return check_launch("tile pass");
}

template <typename R>
static void prog_init(TileProg<R>& P, const Group& g, int n) {
  const int C = TileCfg<R>::C;
  P.nops = 0;
  P.lo = g.lo;
  P.k = g.k;
  P.c = std::min(C, g.lo);
  P.n = n;
  P.twiddle = 0;
  P.nl = 0;
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
      P.kind[P.nops] = TOP_U2;
      P.q[P.nops] = (int8_t)j;
      P.mk[P.nops] = (int8_t)mk;
      P.U[P.nops] = mat_from_host<R>(U + 8 * q);
      ++P.nops;
    }
    qc_status st = run_tile<R>(s, P, nullptr, nullptr);
    if (st) return st;
  }
  return QC_OK;
}

qc_status launch_layer(qc_state* s, const double* U, uint64_t mask) {
  s->sum_valid = false;
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
// In-place reversal of all n index bits.  Index = (h, m, l) with h, l of b
// bits: rev(h, m, l) = (rev l, rev m, rev h).  The block for middle value m
// (with m <= rev m) exchanges the 2^b x 2^b tiles of m and rev m through
// shared memory (rows of 2^b contiguous amplitudes, padded against bank
// conflicts).
template <typename R>
__global__ void __launch_bounds__(256) k_bitrev(typename CT<R>::V2* __restrict__ s, int n, int b) {
  using V2 = typename CT<R>::V2;
  const int W = 1 << b, WP = W + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  V2* A = reinterpret_cast<V2*>(smraw);
  V2* B = A + W * WP;
  const int nm = n - 2 * b;
  const uint64_t M = 1ull << nm;
  for (uint64_t m = blockIdx.x; m < M; m += gridDim.x) {
    const uint64_t mr = nm ? (__brevll((unsigned long long)m) >> (64 - nm)) : 0ull;
    if (mr < m) continue;
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
      const int h = e >> b, l = e & (W - 1);
      A[h * WP + l] = s[((uint64_t)h << (n - b)) | (m << b) | (uint64_t)l];
      if (mr != m) B[h * WP + l] = s[((uint64_t)h << (n - b)) | (mr << b) | (uint64_t)l];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
      const int h = e >> b, l = e & (W - 1);
      const int rl = (int)(__brev((unsigned)l) >> (32 - b)), rh = (int)(__brev((unsigned)h) >> (32 - b));
      // element (h, m, l) of the output is the input at rev(h, m, l)
      if (mr != m) {
        s[((uint64_t)h << (n - b)) | (m << b) | (uint64_t)l] = B[rl * WP + rh];
        s[((uint64_t)h << (n - b)) | (mr << b) | (uint64_t)l] = A[rl * WP + rh];
      } else {
        s[((uint64_t)h << (n - b)) | (m << b) | (uint64_t)l] = A[rl * WP + rh];
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
static qc_status bitrev_impl(qc_state* s) {
  using V2 = typename CT<R>::V2;
  V2* d = reinterpret_cast<V2*>(s->data);
  const int n = s->n;
  const int b = 5;
  if (n < 2 * b) {
    k_bitrev_small<R><<<1, 256, sizeof(V2) << n, s->stream>>>(d, n);
    return check_launch("bitrev small");
  }
  const size_t smem = 2 * (size_t)(1 << b) * ((1 << b) + 1) * sizeof(V2);
  const uint64_t M = 1ull << (n - 2 * b);
  const unsigned grid = (unsigned)std::min<uint64_t>(M, (uint64_t)sm_count() * 8);
  k_bitrev<R><<<grid, 256, smem, s->stream>>>(d, n, b);
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
  std::vector<Group> groups = plan_groups<R>(n);
  for (int gi = (int)groups.size() - 1; gi >= 0 && !st; --gi) {
    const Group& g = groups[gi];
    TileProg<R> P;
    prog_init(P, g, n);
    P.nl = nl;
    for (int j = g.k - 1; j >= 0; --j) {
      P.kind[P.nops] = TOP_QFTLEVEL;
      P.q[P.nops] = (int8_t)j;
      P.mk[P.nops] = 0;
      ++P.nops;
    }
    P.twiddle = g.lo > 0;
    st = run_tile<R>(s, P, tlo, thi);
  }
  if (!st) st = bitrev_impl<R>(s);
  cudaFreeAsync(tab, s->stream);
  return st;
}

qc_status launch_qft(qc_state* s) {
  s->sum_valid = false;
  return s->dt == QC_C128 ? qft_impl<double>(s) : qft_impl<float>(s);
}

}  // namespace qc
