// The paper's noise intrusions and the ensemble density matrix (sec. 6.1-6.3).
//
// * qc_wigner_d: the Wigner rotation D^j(alpha, beta, gamma) for j = 1/2
//   (D2, a one-qubit intrusion) and j = 3/2 (D4, a two-qubit one), rows and
//   columns ordered m = j .. -j, D_{m'm} = e^{-i m' alpha} d^j_{m'm}(beta)
//   e^{-i m gamma}; host arithmetic, applied with qc_apply_1q / qc_apply_2q.
// * qc_density_matrix: <n|rho|n'> = sum_a P_a C_a(n) C_a(n')^* over a batch
//   of B states ("multiverses"), written out for small n.
// * qc_mixed_spectrum: the eigenvalues of rho without forming it.  rho has
//   rank <= B, and its nonzero eigenvalues are those of the B x B Gram
//   matrix G_ab = sqrt(P_a P_b) <psi_a|psi_b>, which one streaming pass over
//   the batch builds; one CTA reduces G to tridiagonal form (Householder)
//   and finds its eigenvalues by bisection.  Trace,
//   purity Tr rho^2 and the entropy -sum l ln l follow.
//
// Inner products run in double-float on the FP32 pipe (GB300's FP64 rate is
// ~1/70 of FP32); the eigenvalue solver works in FP64 on a matrix of at
// most 64 x 64.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace qc {

// ------------------------------------------------ amplitudes as ff pairs --
// A non-finite amplitude becomes a NaN pair (the double-float split would
// turn it into a finite value), so that it reaches the Gram matrix.
__device__ __forceinline__ ffc load_ffc(const double2* p, uint64_t i) {
  const double2 v = p[i];
  if (!isfinite(v.x) || !isfinite(v.y)) return ffc_make(ff_make(NAN, 0.f), ff_make(NAN, 0.f));
  return ffc_make(ff_from_d(v.x), ff_from_d(v.y));
}
__device__ __forceinline__ ffc load_ffc(const float2* p, uint64_t i) {
  const float2 v = p[i];
  return ffc_make(ff_make(v.x, 0.f), ff_make(v.y, 0.f));
}
template <typename V2> __device__ __forceinline__ V2 ffc_to_v2(const ffc& z);
template <> __device__ __forceinline__ double2 ffc_to_v2<double2>(const ffc& z) {
  return make_double2(ff_to_d(z.re), ff_to_d(z.im));
}
template <> __device__ __forceinline__ float2 ffc_to_v2<float2>(const ffc& z) {
  return make_float2(z.re.hi + z.re.lo, z.im.hi + z.im.lo);
}
__device__ __forceinline__ double2 conj_v(double2 v) { return make_double2(v.x, -v.y); }
__device__ __forceinline__ float2 conj_v(float2 v) { return make_float2(v.x, -v.y); }

// rho is Hermitian: only tiles on and above the diagonal are formed, and an
// off-diagonal tile's conjugate transpose goes through shared memory (Tm) to
// the mirrored tile in coalesced rows.
template <typename V2>
__device__ __forceinline__ void rho_mirror(V2 (*Tm)[33], V2* __restrict__ rho, uint64_t N, uint64_t r0, uint64_t c0) {
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int rr = e >> 5, cc = e & 31;
    if (c0 + rr < N && r0 + cc < N) rho[(c0 + rr) * N + r0 + cc] = Tm[rr][cc];
  }
}

// acc += a * conj(b)
__device__ __forceinline__ void mac_conj_b(ffc& acc, const ffc& a, const ffc& b) {
  acc.re = ff_add(acc.re, ff_dot2p(a.re, b.re, a.im, b.im));
  acc.im = ff_add(acc.im, ff_dot2m(a.im, b.re, a.re, b.im));
}

// ------------------------------------------------------------- rho -------
#define RHO_TILE 32
#define RHO_KC 16

// One CTA: a 32 x 32 tile of rho (rows r0.., columns c0..); each of the 256
// threads owns 2 x 2 entries.  The weights P_a scale the row operands.
template <typename V2>
__global__ void __launch_bounds__(256) k_rho(const V2* __restrict__ psi, uint64_t N, int B,
                                             const double* __restrict__ P, V2* __restrict__ rho) {
  static_assert(RHO_TILE == 32, "the mirror tile is 32 x 32");
  if (blockIdx.y > blockIdx.x) return;  // the mirror of a tile above the diagonal
  const bool mirror = blockIdx.y != blockIdx.x;
  __shared__ ffc Ar[RHO_KC][RHO_TILE], Ac[RHO_KC][RHO_TILE];
  __shared__ V2 Tm[RHO_TILE][RHO_TILE + 1];
  const uint64_t r0 = (uint64_t)blockIdx.y * RHO_TILE, c0 = (uint64_t)blockIdx.x * RHO_TILE;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if constexpr (std::is_same<V2, float2>::value) {
    // complex64: plain FP32 (B terms per entry, the dtype's own precision)
    __shared__ float2 Fr[RHO_KC][RHO_TILE], Fc[RHO_KC][RHO_TILE];
    float2 f[2][2] = {{{0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}}};
    for (int a0 = 0; a0 < B; a0 += RHO_KC) {
      for (int e = threadIdx.x; e < RHO_KC * RHO_TILE; e += blockDim.x) {
        const int k = e / RHO_TILE, x = e % RHO_TILE, a = a0 + k;
        float2 vr = make_float2(0.f, 0.f), vc = vr;
        if (a < B) {
          const float w = (float)P[a];
          if (r0 + x < N) {
            vr = psi[(uint64_t)a * N + r0 + x];
            vr.x *= w;
            vr.y *= w;
          }
          if (c0 + x < N) vc = psi[(uint64_t)a * N + c0 + x];
        }
        Fr[k][x] = vr;
        Fc[k][x] = vc;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < RHO_KC; ++k) {
        const float2 r[2] = {Fr[k][2 * ty], Fr[k][2 * ty + 1]}, c[2] = {Fc[k][2 * tx], Fc[k][2 * tx + 1]};
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j) {  // r conj(c)
            f[i][j].x = fmaf(r[i].x, c[j].x, fmaf(r[i].y, c[j].y, f[i][j].x));
            f[i][j].y = fmaf(r[i].y, c[j].x, fmaf(-r[i].x, c[j].y, f[i][j].y));
          }
      }
      __syncthreads();
    }
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        const uint64_t r = r0 + 2 * ty + i, c = c0 + 2 * tx + j;
        if (r < N && c < N) rho[r * N + c] = f[i][j];
        Tm[2 * tx + j][2 * ty + i] = conj_v(f[i][j]);
      }
    if (mirror) rho_mirror<V2>(Tm, rho, N, r0, c0);
  } else {
  ffc acc[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) acc[i][j] = ffc_make(ff_make(0.f, 0.f), ff_make(0.f, 0.f));
  for (int a0 = 0; a0 < B; a0 += RHO_KC) {
    for (int e = threadIdx.x; e < RHO_KC * RHO_TILE; e += blockDim.x) {
      const int k = e / RHO_TILE, x = e % RHO_TILE;
      const int a = a0 + k;
      ffc vr = ffc_make(ff_make(0.f, 0.f), ff_make(0.f, 0.f)), vc = vr;
      if (a < B) {
        const ff w = ff_from_d(P[a]);
        if (r0 + x < N) {
          vr = load_ffc(psi, (uint64_t)a * N + r0 + x);
          vr = ffc_make(ff_mul(vr.re, w), ff_mul(vr.im, w));
        }
        if (c0 + x < N) vc = load_ffc(psi, (uint64_t)a * N + c0 + x);
      }
      Ar[k][x] = vr;
      Ac[k][x] = vc;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < RHO_KC; ++k) {
      const ffc ra = Ar[k][2 * ty], rb = Ar[k][2 * ty + 1], ca = Ac[k][2 * tx], cb = Ac[k][2 * tx + 1];
      mac_conj_b(acc[0][0], ra, ca);
      mac_conj_b(acc[0][1], ra, cb);
      mac_conj_b(acc[1][0], rb, ca);
      mac_conj_b(acc[1][1], rb, cb);
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const uint64_t r = r0 + 2 * ty + i, c = c0 + 2 * tx + j;
      const V2 v = ffc_to_v2<V2>(acc[i][j]);
      if (r < N && c < N) rho[r * N + c] = v;
      Tm[2 * tx + j][2 * ty + i] = conj_v(v);
    }
  if (mirror) rho_mirror<V2>(Tm, rho, N, r0, c0);
  }
}

// ------------------------------------------------------------ Gram -------
#define GRAM_K 32

// Partial Gram sums over one slice of the amplitude axis per CTA:
// part[blk][a][b] = sum_n conj(C_a(n)) C_b(n) (float pairs: re hi, re lo,
// im hi, im lo).  Thread t owns the 4 x 4 block a = 4 (t/16).., b = 4 (t%16)..
template <typename V2>
__global__ void __launch_bounds__(256) k_gram(const V2* __restrict__ psi, uint64_t N, int B, uint64_t per_blk,
                                              float4* __restrict__ part) {
  __shared__ ffc X[QC_SPECTRUM_MAX_UNIVERSES][GRAM_K];
  const int ta = (threadIdx.x >> 4) * 4, tb = (threadIdx.x & 15) * 4;
  ffc acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = ffc_make(ff_make(0.f, 0.f), ff_make(0.f, 0.f));
  const uint64_t lo = (uint64_t)blockIdx.x * per_blk, hi = min(N, lo + per_blk);
  for (uint64_t k0 = lo; k0 < hi; k0 += GRAM_K) {
    for (int e = threadIdx.x; e < B * GRAM_K; e += blockDim.x) {
      const int a = e / GRAM_K, x = e % GRAM_K;
      X[a][x] = (k0 + x < hi) ? load_ffc(psi, (uint64_t)a * N + k0 + x)
                              : ffc_make(ff_make(0.f, 0.f), ff_make(0.f, 0.f));
    }
    __syncthreads();
    if (std::is_same<V2, float2>::value && ta < B && tb < B) {
      // complex64: exact-enough FP32 sums over the 32 amplitudes of a tile,
      // added into the float pairs once per tile
      float2 f[4][4];
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) f[i][j] = make_float2(0.f, 0.f);
      for (int x = 0; x < GRAM_K; ++x) {
        float2 va[4], vb[4];
        for (int i = 0; i < 4; ++i) {
          va[i] = (ta + i < B) ? make_float2(X[ta + i][x].re.hi, X[ta + i][x].im.hi) : make_float2(0.f, 0.f);
          vb[i] = (tb + i < B) ? make_float2(X[tb + i][x].re.hi, X[tb + i][x].im.hi) : make_float2(0.f, 0.f);
        }
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) {  // conj(C_a) C_b
            f[i][j].x = fmaf(va[i].x, vb[j].x, fmaf(va[i].y, vb[j].y, f[i][j].x));
            f[i][j].y = fmaf(va[i].x, vb[j].y, fmaf(-va[i].y, vb[j].x, f[i][j].y));
          }
      }
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          acc[i][j].re = ff_add(acc[i][j].re, ff_make(f[i][j].x, 0.f));
          acc[i][j].im = ff_add(acc[i][j].im, ff_make(f[i][j].y, 0.f));
        }
    } else if (ta < B && tb < B) {
      for (int x = 0; x < GRAM_K; ++x) {
        ffc va[4], vb[4];
        for (int i = 0; i < 4; ++i) {
          va[i] = (ta + i < B) ? X[ta + i][x] : ffc_make(ff_make(0.f, 0.f), ff_make(0.f, 0.f));
          vb[i] = (tb + i < B) ? X[tb + i][x] : ffc_make(ff_make(0.f, 0.f), ff_make(0.f, 0.f));
        }
        // conj(C_a) C_b = C_b conj(C_a)
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) mac_conj_b(acc[i][j], vb[j], va[i]);
      }
    }
    __syncthreads();
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      const int a = ta + i, b = tb + j;
      if (a < B && b < B)
        part[((uint64_t)blockIdx.x * B + a) * B + b] =
            make_float4(acc[i][j].re.hi, acc[i][j].re.lo, acc[i][j].im.hi, acc[i][j].im.lo);
    }
}

// G[a][b] = sqrt(P_a P_b) * sum over blocks (in block order), one thread per
// entry.  G is made exactly Hermitian: the entries with a > b are the
// conjugates of their mirrors and the diagonal is real (the two triangles'
// separately rounded sums differ by ~1e-14; the solver assumes a Hermitian G).
__global__ void k_gram_final(const float4* __restrict__ part, int nblk, int B, const double* __restrict__ sqrtP,
                             double2* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * B) return;
  const int a = e / B, b = e % B;
  const int u = min(a, b) * B + max(a, b);  // the upper-triangle entry
  ff re = ff_make(0.f, 0.f), im = ff_make(0.f, 0.f);
  for (int k = 0; k < nblk; ++k) {
    const float4 v = part[(uint64_t)k * B * B + u];
    re = ff_add(re, ff_make(v.x, v.y));
    im = ff_add(im, ff_make(v.z, v.w));
  }
  if (!isfinite(re.hi) || !isfinite(im.hi)) {  // kept non-finite (the join would not)
    G[e] = make_double2(NAN, NAN);
    return;
  }
  const double w = sqrtP[a] * sqrtP[b];
  const double gi = (a == b) ? 0.0 : ff_to_d(im) * w;
  G[e] = make_double2(ff_to_d(re) * w, a > b ? -gi : gi);
}

// ------------------------------------------------------- eigenvalues ----
// Eigenvalues of the Hermitian B x B matrix G (one CTA, FP64, B <= 64):
//  1. Householder reduction to a real symmetric tridiagonal matrix.  Step k
//     reflects x = A[k+1.., k] onto alpha e_1 with alpha = -(x_0/|x_0|) |x|
//     (no cancellation in v = x - alpha e_1), through u = v / |v|:
//     p = A22 u, K = u^H p, q = p - K u, A22 -= 2 (u q^H + q u^H).  The
//     off-diagonal entries' phases are removed by a diagonal unitary
//     similarity, so T has diagonal Re A_kk and off-diagonal |x|.
//  2. Each eigenvalue by bisection on Sturm counts of T (one thread each;
//     the number of negative pivots of T - x I is the number of
//     eigenvalues below x), from the Gershgorin interval down to a width
//     of 2^-52 of its magnitude.
// About n^3 complex multiply-adds once, where the cyclic Jacobi method it
// replaces took that per sweep on one SM's FP64 pipe (64 x 64: 15 ms with
// Jacobi's ~10 sweeps).
// Out: ev[0..B) descending; stats = trace, sum l^2, -sum l ln l (l > 1e-14);
// status[0] = 0, or 1 if T has a non-finite entry.
#define EIG_SMEM(B) ((size_t)(B) * ((B) + 1) * sizeof(double2))

__device__ __forceinline__ double eig_block_sum(double x, double* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();  // red is free
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// number of eigenvalues of T (diagonal d, squared off-diagonal e2) below x
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int B, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int i = 1; i < B; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

__global__ void __launch_bounds__(256) k_eigh(const double2* __restrict__ G, int B, double* __restrict__ ev,
                                              double* __restrict__ stats, int* __restrict__ status) {
  extern __shared__ double2 A[];  // B x (B + 1), padded rows
  __shared__ double2 u[QC_SPECTRUM_MAX_UNIVERSES], pq[QC_SPECTRUM_MAX_UNIVERSES];
  __shared__ double d[QC_SPECTRUM_MAX_UNIVERSES], e2[QC_SPECTRUM_MAX_UNIVERSES];
  __shared__ double red[8];
  __shared__ double lam[QC_SPECTRUM_MAX_UNIVERSES];
  const int tid = threadIdx.x, T = blockDim.x, W = B + 1;
  for (int e = tid; e < B * B; e += T) A[(e / B) * W + e % B] = G[e];
  __syncthreads();
  for (int k = 0; k + 2 < B; ++k) {
    const int m = B - 1 - k, o = k + 1;  // x = A[o + i][k], i < m
    double2 x = make_double2(0.0, 0.0);
    if (tid < m) x = A[(o + tid) * W + k];
    const double sigma = eig_block_sum(x.x * x.x + x.y * x.y, red);
    const double2 x0 = A[o * W + k];
    const double nx = sqrt(sigma), a0 = sqrt(x0.x * x0.x + x0.y * x0.y);
    if (tid == 0) {
      d[k] = A[k * W + k].x;
      e2[k] = sigma;
    }
    if (!(nx > 0.0)) {  // nothing below the diagonal (or non-finite: caught at the end)
      __syncthreads();
      continue;
    }
    // phase of x0 (1 for x0 = 0); v = x - alpha e_1, |v|^2 = 2 |x| (|x| + |x0|)
    const double2 ph = a0 > 0.0 ? make_double2(x0.x / a0, x0.y / a0) : make_double2(1.0, 0.0);
    const double inv = 1.0 / sqrt(2.0 * nx * (nx + a0));
    if (tid < m) {
      const double2 xv = tid == 0 ? make_double2(x0.x + ph.x * nx, x0.y + ph.y * nx) : x;
      u[tid] = make_double2(xv.x * inv, xv.y * inv);
    }
    __syncthreads();
    // p = A22 u: four threads per row
    {
      const int r = tid >> 2, part = tid & 3;
      double pr = 0.0, pi = 0.0;
      if (r < m)
        for (int c = part; c < m; c += 4) {
          const double2 a = A[(o + r) * W + o + c], uv = u[c];
          pr = fma(a.x, uv.x, fma(-a.y, uv.y, pr));
          pi = fma(a.x, uv.y, fma(a.y, uv.x, pi));
        }
      pr += __shfl_xor_sync(0xffffffffu, pr, 1);
      pi += __shfl_xor_sync(0xffffffffu, pi, 1);
      pr += __shfl_xor_sync(0xffffffffu, pr, 2);
      pi += __shfl_xor_sync(0xffffffffu, pi, 2);
      if (r < m && part == 0) pq[r] = make_double2(pr, pi);
    }
    __syncthreads();
    // K = u^H p (real for Hermitian A22), then q = p - K u
    double kk = 0.0;
    if (tid < m) kk = u[tid].x * pq[tid].x + u[tid].y * pq[tid].y;
    const double K = eig_block_sum(kk, red);
    if (tid < m) pq[tid] = make_double2(pq[tid].x - K * u[tid].x, pq[tid].y - K * u[tid].y);
    __syncthreads();
    // A22 -= 2 (u q^H + q u^H)
    for (int e = tid; e < m * m; e += T) {
      const int r = e / m, c = e % m;
      const double2 ur = u[r], uc = u[c], qr = pq[r], qc = pq[c];
      double2 a = A[(o + r) * W + o + c];
      a.x -= 2.0 * (ur.x * qc.x + ur.y * qc.y + qr.x * uc.x + qr.y * uc.y);
      a.y -= 2.0 * (ur.y * qc.x - ur.x * qc.y + qr.y * uc.x - qr.x * uc.y);
      A[(o + r) * W + o + c] = a;
    }
    __syncthreads();
  }
  if (tid == 0) {
    const int k0 = B >= 2 ? B - 2 : 0;
    for (int k = k0; k < B; ++k) d[k] = A[k * W + k].x;
    if (B >= 2) {
      const double2 c = A[(B - 1) * W + B - 2];
      e2[B - 2] = c.x * c.x + c.y * c.y;
    }
  }
  __syncthreads();
  // Gershgorin interval and the pivot floor
  double lo = 0.0, hi = 0.0, emax = 0.0;
  bool finite = true;
  for (int i = 0; i < B; ++i) {
    const double el = i > 0 ? sqrt(e2[i - 1]) : 0.0, er = i + 1 < B ? sqrt(e2[i]) : 0.0;
    lo = i ? fmin(lo, d[i] - el - er) : d[i] - el - er;
    hi = i ? fmax(hi, d[i] + el + er) : d[i] + el + er;
    if (i + 1 < B) emax = fmax(emax, e2[i]);
    finite = finite && isfinite(d[i]) && (i + 1 >= B || isfinite(e2[i]));
  }
  const double span = fmax(fabs(lo), fabs(hi));
  lo -= 2.2e-16 * span + 1e-300;
  hi += 2.2e-16 * span + 1e-300;
  const double pivmin = fmax(2.2e-308, 2.2e-308 * emax);
  if (finite && tid < B) {  // the tid-th smallest eigenvalue
    double a = lo, b = hi;
    for (int it = 0; it < 200 && b - a > 2.2e-16 * fmax(fabs(a), fabs(b)) + 1e-19 * span + 1e-300; ++it) {
      const double mid = 0.5 * (a + b);
      if (sturm_count(d, e2, B, mid, pivmin) > tid) b = mid;
      else a = mid;
    }
    lam[tid] = 0.5 * (a + b);
  }
  __syncthreads();
  if (tid == 0) {
    double tr = 0.0, p2 = 0.0, sl = 0.0;
    for (int i = 0; i < B; ++i) {
      const double l = finite ? lam[B - 1 - i] : NAN;
      ev[i] = l;
      tr += l;
      p2 += l * l;
      if (l > 1e-14) sl -= l * log(l);
    }
    stats[0] = tr;
    stats[1] = p2;
    stats[2] = sl;
    status[0] = finite ? 0 : 1;
  }
}

}  // namespace qc

using namespace qc;

// ------------------------------------------------------------- host ------
QC_API qc_status qc_wigner_d(int twoj, double alpha, double beta, double gamma, double* D_out) {
  clear_error();
  if (!D_out || (twoj != 1 && twoj != 3) || !std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(gamma)) {
    set_error("qc_wigner_d: twoj must be 1 or 3, angles finite, output non-NULL");
    return QC_EINVAL;
  }
  const double c = cos(0.5 * beta), s = sin(0.5 * beta);
  const int dim = twoj + 1;
  double d[16];
  if (twoj == 1) {  // d^{1/2}(beta), m = +1/2, -1/2
    const double t[4] = {c, -s, s, c};
    for (int i = 0; i < 4; ++i) d[i] = t[i];
  } else {  // d^{3/2}(beta), m = 3/2, 1/2, -1/2, -3/2
    const double r3 = sqrt(3.0);
    const double t[16] = {c * c * c,       -r3 * c * c * s,           r3 * c * s * s,            -s * s * s,
                          r3 * c * c * s,  c * (c * c - 2.0 * s * s), -s * (2.0 * c * c - s * s), r3 * c * s * s,
                          r3 * c * s * s,  s * (2.0 * c * c - s * s), c * (c * c - 2.0 * s * s), -r3 * c * c * s,
                          s * s * s,       r3 * c * s * s,            r3 * c * c * s,            c * c * c};
    for (int i = 0; i < 16; ++i) d[i] = t[i];
  }
  for (int r = 0; r < dim; ++r)
    for (int col = 0; col < dim; ++col) {
      const double mp = 0.5 * (twoj - 2 * r), m = 0.5 * (twoj - 2 * col);
      const double ph = -(mp * alpha + m * gamma);  // e^{-i m' alpha} e^{-i m gamma}
      D_out[2 * (r * dim + col)] = d[r * dim + col] * cos(ph);
      D_out[2 * (r * dim + col) + 1] = d[r * dim + col] * sin(ph);
    }
  return QC_OK;
}

static qc_status check_batch(const void* psi, int n, qc_dtype dt, int B, const double* P, int max_n, int max_b) {
  if (!psi || !P || n < 1 || n > max_n || B < 1 || B > max_b || (dt != QC_C128 && dt != QC_C64)) {
    set_error("bad batch: psi/P NULL, n = %d (1..%d), B = %d (1..%d) or dtype %d", n, max_n, B, max_b, (int)dt);
    return QC_EINVAL;
  }
  for (int a = 0; a < B; ++a)
    if (!(P[a] >= 0.0) || !std::isfinite(P[a])) {
      set_error("weight P[%d] = %g is not a finite non-negative number", a, P[a]);
      return QC_EINVAL;
    }
  return QC_OK;
}

QC_API qc_status qc_density_matrix(const void* psi_dev, int n, qc_dtype dt, int B, const double* P_host,
                                   void* rho_dev, void* stream) {
  clear_error();
  qc_status st = check_batch(psi_dev, n, dt, B, P_host, QC_DM_MAX_QUBITS, 1 << 30);
  if (st) return st;
  if (!rho_dev) {
    set_error("rho_dev is NULL");
    return QC_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t N = 1ull << n;
  double* P = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&P, sizeof(double) * B, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P, P_host, sizeof(double) * B, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    if (P) cudaFreeAsync(P, s);
    return cuda_fail(e, "density matrix weights");
  }
  if (dt == QC_C64 && B <= 64) {  // tensor cores (rho_tc.cu)
    cudaFreeAsync(P, s);
    return rho_tc_c64(reinterpret_cast<const float2*>(psi_dev), n, B, P_host, reinterpret_cast<float2*>(rho_dev), s);
  }
  const unsigned nt = (unsigned)((N + RHO_TILE - 1) / RHO_TILE);
  const dim3 grid(nt, nt);
  if (dt == QC_C128)
    k_rho<double2><<<grid, 256, 0, s>>>(reinterpret_cast<const double2*>(psi_dev), N, B, P,
                                         reinterpret_cast<double2*>(rho_dev));
  else
    k_rho<float2><<<grid, 256, 0, s>>>(reinterpret_cast<const float2*>(psi_dev), N, B, P,
                                        reinterpret_cast<float2*>(rho_dev));
  st = check_launch("density matrix", 1);
  cudaFreeAsync(P, s);
  return st;
}

QC_API qc_status qc_mixed_spectrum(const void* psi_dev, int n, qc_dtype dt, int B, const double* P_host,
                                   double* evals_host, double* stats_host, void* stream) {
  clear_error();
  qc_status st = check_batch(psi_dev, n, dt, B, P_host, 34, QC_SPECTRUM_MAX_UNIVERSES);
  if (st) return st;
  if (!evals_host || !stats_host) {
    set_error("NULL output");
    return QC_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t N = 1ull << n;
  // slices of the amplitude axis: a resident grid, each slice a multiple of GRAM_K
  const int nblk = (int)std::min<uint64_t>((N + GRAM_K - 1) / GRAM_K, (uint64_t)sm_count() * 2);
  uint64_t per = (N + nblk - 1) / nblk;
  per = (per + GRAM_K - 1) / GRAM_K * GRAM_K;
  const size_t part_b = sizeof(float4) * (size_t)nblk * B * B;
  const size_t g_b = sizeof(double2) * B * B;
  const size_t small_b = sizeof(double) * (2 * B + 3) + sizeof(int) * 2;
  char* buf = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&buf, part_b + g_b + small_b + 64, s);
  if (e != cudaSuccess) return cuda_fail(e, "spectrum workspace");
  float4* part = reinterpret_cast<float4*>(buf);
  double2* G = reinterpret_cast<double2*>(buf + part_b);
  double* sqrtP = reinterpret_cast<double*>(buf + part_b + g_b);
  double* ev = sqrtP + B;
  double* stats = ev + B;
  int* status = reinterpret_cast<int*>(stats + 3);
  std::vector<double> sq(B);
  for (int a = 0; a < B; ++a) sq[a] = sqrt(P_host[a]);
  e = cudaMemcpyAsync(sqrtP, sq.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(buf, s);
    return cuda_fail(e, "spectrum weights");
  }
  if (dt == QC_C128)
    k_gram<double2><<<nblk, 256, 0, s>>>(reinterpret_cast<const double2*>(psi_dev), N, B, per, part);
  else
    k_gram<float2><<<nblk, 256, 0, s>>>(reinterpret_cast<const float2*>(psi_dev), N, B, per, part);
  k_gram_final<<<(B * B + 255) / 256, 256, 0, s>>>(part, nblk, B, sqrtP, G);
  static bool eig_attr = false;  // the opt-in above 48 KiB, once per process
  if (!eig_attr) {
    cudaFuncSetAttribute(k_eigh, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)EIG_SMEM(QC_SPECTRUM_MAX_UNIVERSES));
    eig_attr = true;
  }
  k_eigh<<<1, 256, EIG_SMEM(B), s>>>(G, B, ev, stats, status);
  st = check_launch("mixed spectrum", 3);
  if (!st) {
    e = cudaMemcpyAsync(evals_host, ev, sizeof(double) * B, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stats_host, stats, sizeof(double) * 3, cudaMemcpyDeviceToHost, s);
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "spectrum readback");
    else if (bad) {
      set_error("mixed spectrum: the Gram matrix has a non-finite entry");
      st = QC_ECUDA;
    }
  }
  cudaFreeAsync(buf, s);
  return st;
}
