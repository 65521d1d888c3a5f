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
//   the batch builds; a one-CTA Jacobi solver diagonalises G.  Trace,
//   purity Tr rho^2 and the entropy -sum l ln l follow.
//
// Inner products run in double-float on the FP32 pipe (GB300's FP64 rate is
// ~1/70 of FP32); the Jacobi solver works in FP64 on a matrix of at most
// 64 x 64.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace qc {

// ------------------------------------------------ amplitudes as ff pairs --
__device__ __forceinline__ ffc load_ffc(const double2* p, uint64_t i) {
  const double2 v = p[i];
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
// separately rounded sums differ by ~1e-14, which Jacobi cannot rotate away).
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
  const double w = sqrtP[a] * sqrtP[b];
  const double gi = (a == b) ? 0.0 : ff_to_d(im) * w;
  G[e] = make_double2(ff_to_d(re) * w, a > b ? -gi : gi);
}

// ----------------------------------------------------------- Jacobi ------
// Eigenvalues of the Hermitian B x B matrix G (one CTA, FP64, B <= 64):
// cyclic Jacobi with a round-robin ordering, so the B'/2 rotations of one
// round touch disjoint rows and columns.  Rotation (p, q): with
// c = A_pq = |c| e^{i phi}, the phase e^{-i phi} on q makes the pair real
// and the classical rotation tan(2 theta) = 2|c| / (A_qq - A_pp) zeroes it.
// Out: ev[0..B) descending; stats = trace, sum l^2, -sum l ln l (l > 1e-14);
// status[0] = sweeps used (a capped, bounded loop).
#define JAC_MAX_SWEEPS 40
// The matrix lives in dynamic shared memory, B' x (B'+1) entries (B' = B
// rounded up to even, the extra row and column zero).
#define JAC_SMEM(Bp) ((size_t)(Bp) * ((Bp) + 1) * sizeof(double2))
__global__ void __launch_bounds__(256) k_jacobi(const double2* __restrict__ G, int B, double* __restrict__ ev,
                                                double* __restrict__ stats, int* __restrict__ status) {
  extern __shared__ double2 Ash[];
  __shared__ double prm[QC_SPECTRUM_MAX_UNIVERSES / 2][4];  // cs, sn, e re, e im
  __shared__ int pq[QC_SPECTRUM_MAX_UNIVERSES / 2][2];
  __shared__ double red[256];
  __shared__ int done;
  const int Bp = B + (B & 1);
  const int tid = threadIdx.x, T = blockDim.x;
  for (int e = tid; e < Bp * Bp; e += T) {
    const int r = e / Bp, c = e % Bp;
    Ash[(r) * (Bp + 1) + (c)] = (r < B && c < B) ? G[r * B + c] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < JAC_MAX_SWEEPS; ++sweep) {
    // off-diagonal and total Frobenius mass
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < Bp * Bp; e += T) {
      const double2 v = Ash[(e / Bp) * (Bp + 1) + (e % Bp)];
      const double m2 = v.x * v.x + v.y * v.y;
      tot += m2;
      if (e / Bp != e % Bp) off += m2;
    }
    red[tid] = off;
    __syncthreads();
    if (tid == 0) {
      double o = 0.0;
      for (int i = 0; i < T; ++i) o += red[i];
      red[0] = o;
    }
    __syncthreads();
    const double offs = red[0];
    __syncthreads();
    red[tid] = tot;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < T; ++i) t += red[i];
      done = !(offs > 1e-28 * t);  // off-diagonal mass at the FP64 floor; also ends on a zero or NaN matrix
    }
    __syncthreads();
    if (done) break;
    for (int r = 0; r < Bp - 1; ++r) {
      if (tid < Bp / 2) {
        const int i = tid;
        int p = (i == 0) ? 0 : 1 + (r + i - 1) % (Bp - 1);
        int q = 1 + (r + Bp - 2 - i) % (Bp - 1);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        pq[i][0] = p;
        pq[i][1] = q;
        const double2 c = Ash[(p) * (Bp + 1) + (q)];
        const double d = sqrt(c.x * c.x + c.y * c.y);
        if (d == 0.0) {
          prm[i][0] = 1.0;
          prm[i][1] = 0.0;
          prm[i][2] = 1.0;
          prm[i][3] = 0.0;
        } else {
          const double th = (Ash[(q) * (Bp + 1) + (q)].x - Ash[(p) * (Bp + 1) + (p)].x) / (2.0 * d);
          const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
          const double cs = 1.0 / sqrt(1.0 + t * t);
          prm[i][0] = cs;
          prm[i][1] = t * cs;
          prm[i][2] = c.x / d;
          prm[i][3] = c.y / d;
        }
      }
      __syncthreads();
      // columns: A[:,p] = cs A[:,p] - sn e* A[:,q];  A[:,q] = sn A[:,p] + cs e* A[:,q]
      for (int w = tid; w < (Bp / 2) * Bp; w += T) {
        const int i = w / Bp, k = w % Bp;
        const int p = pq[i][0], q = pq[i][1];
        const double cs = prm[i][0], sn = prm[i][1], er = prm[i][2], ei = -prm[i][3];
        const double2 ap = Ash[(k) * (Bp + 1) + (p)], aq = Ash[(k) * (Bp + 1) + (q)];
        const double eqr = er * aq.x - ei * aq.y, eqi = er * aq.y + ei * aq.x;  // e* A[k][q]
        Ash[(k) * (Bp + 1) + (p)] = make_double2(cs * ap.x - sn * eqr, cs * ap.y - sn * eqi);
        Ash[(k) * (Bp + 1) + (q)] = make_double2(sn * ap.x + cs * eqr, sn * ap.y + cs * eqi);
      }
      __syncthreads();
      // rows: A[p,:] = cs A[p,:] - sn e A[q,:];  A[q,:] = sn A[p,:] + cs e A[q,:]
      for (int w = tid; w < (Bp / 2) * Bp; w += T) {
        const int i = w / Bp, k = w % Bp;
        const int p = pq[i][0], q = pq[i][1];
        const double cs = prm[i][0], sn = prm[i][1], er = prm[i][2], ei = prm[i][3];
        const double2 ap = Ash[(p) * (Bp + 1) + (k)], aq = Ash[(q) * (Bp + 1) + (k)];
        const double eqr = er * aq.x - ei * aq.y, eqi = er * aq.y + ei * aq.x;  // e A[q][k]
        Ash[(p) * (Bp + 1) + (k)] = make_double2(cs * ap.x - sn * eqr, cs * ap.y - sn * eqi);
        Ash[(q) * (Bp + 1) + (k)] = make_double2(sn * ap.x + cs * eqr, sn * ap.y + cs * eqi);
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    double l[QC_SPECTRUM_MAX_UNIVERSES + 1];
    for (int i = 0; i < Bp; ++i) l[i] = Ash[(i) * (Bp + 1) + (i)].x;
    for (int i = 1; i < Bp; ++i) {  // insertion sort, descending
      const double v = l[i];
      int j = i - 1;
      while (j >= 0 && l[j] < v) {
        l[j + 1] = l[j];
        --j;
      }
      l[j + 1] = v;
    }
    double tr = 0.0, p2 = 0.0, s = 0.0;
    for (int i = 0; i < B; ++i) {
      ev[i] = l[i];
      tr += l[i];
      p2 += l[i] * l[i];
      if (l[i] > 1e-14) s -= l[i] * log(l[i]);
    }
    stats[0] = tr;
    stats[1] = p2;
    stats[2] = s;
    status[0] = sweep;
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
  const int Bp = B + (B & 1);
  static bool jac_attr = false;  // the opt-in above 48 KiB, once per process
  if (!jac_attr) {
    cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)JAC_SMEM(QC_SPECTRUM_MAX_UNIVERSES));
    jac_attr = true;
  }
  k_jacobi<<<1, 256, JAC_SMEM(Bp), s>>>(G, B, ev, stats, status);
  st = check_launch("mixed spectrum", 3);
  if (!st) {
    e = cudaMemcpyAsync(evals_host, ev, sizeof(double) * B, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stats_host, stats, sizeof(double) * 3, cudaMemcpyDeviceToHost, s);
    int sweeps = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sweeps, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "spectrum readback");
    else if (sweeps >= JAC_MAX_SWEEPS) {
      set_error("Jacobi did not converge in %d sweeps", JAC_MAX_SWEEPS);
      st = QC_ECUDA;
    }
  }
  cudaFreeAsync(buf, s);
  return st;
}
