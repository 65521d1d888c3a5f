// Batched noisy Grover trajectories -- the "multiverse" of sec. 6.2-6.3:
// many independent replicas of the algorithm, each with its own random
// disturbances -- as one persistent launch.
//
// Launch shape: thread-block clusters of G CTAs; each cluster takes the
// next instance from an atomic work queue (instances sorted by cost,
// largest first) and runs it to the end with its state in a per-cluster
// slot of global memory (the slots together are sized to stay in L2).  CTA
// c of the cluster owns 1/G of the amplitudes.  Per-iteration scalars (the
// amplitude sum S, the squared norm Q, the marked amplitude) are exchanged
// through distributed shared memory, synchronised by the hardware cluster
// barrier (no spin waits).  G and the CTA size are picked by a built-in
// autotuner from timed trial runs.
//
// Noise (per-gate Pauli errors): every gate location draws Philox4x32-10
// with counter (instance, stage, qubit, 'NOIS').  Errors after the H gates
// of a HALL commute with the other H gates, so one noisy iteration is
//   E4 . HALL . E3 . Inv . E2 . HALL . E1 . Oracle
//     = E4 E3' . D . E2' E1 . Oracle,   D = HALL . Inv . HALL = 2|s><s| - I,
// with P' = HALL P HALL (X <-> Z, Y -> -Y).  With Pauli strings
// A = E4 E3' and B = E2' E1 one iteration is a single pass
//   out[j] = A-phase(j) * (2 m - B-phase * s * (O psi)[j ^ xA ^ xB]),
// where m is the mean of B O psi-hat and s = 1/sqrt(Q) renormalises the
// state every iteration (complex64 arithmetic, FP64 reductions).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace qc {

#define TAG_NOISE 0x4E4F4953u
#define TAG_MEAS 0x4D454153u
#define TAG_READ 0x52454144u

struct TrajInst {
  int n, iters;
  uint64_t marked;
  int id;
  int pad;
};

struct TrajParams {
  const TrajInst* inst;
  int n_inst;
  float2* slots;
  uint64_t slot_amps;
  uint64_t seed;
  uint32_t thr_gate, thr_ro;
  double p_ro;
  unsigned* queue;
  int* status;
  double* p_success;
  double* p_readout;
  uint64_t* outcome;
  uint32_t* n_errors;
};

// Pauli string i^a X^x Z^z.
struct Pauli {
  uint64_t x, z;
  int a;
};

__device__ __forceinline__ Pauli pmul(const Pauli& p, const Pauli& q) {  // p . q
  Pauli r;
  r.x = p.x ^ q.x;
  r.z = p.z ^ q.z;
  r.a = (p.a + q.a + 2 * (__popcll(p.z & q.x) & 1)) & 3;
  return r;
}
__device__ __forceinline__ Pauli hconj(const Pauli& p) {  // HALL p HALL
  Pauli r;
  r.x = p.z;
  r.z = p.x;
  r.a = (p.a + 2 * (__popcll(p.x & p.z) & 1)) & 3;
  return r;
}

// (re, im) * i^a
__device__ __forceinline__ void ipow(int a, float& re, float& im) {
  const float r = re, i = im;
  if (a == 1) { re = -i; im = r; }
  else if (a == 2) { re = -r; im = -i; }
  else if (a == 3) { re = i; im = -r; }
}

struct Xch {
  int inst;
  int pad;
  double v[2][8];  // double-buffered partials: S re, S im, Q, cm re, cm im, aux0, aux1, aux2
  unsigned long long w[2];
};

__device__ __forceinline__ void ff_add(float& s, float& c, float p) {
  const float t = s + p;
  const float bp = t - s;
  c += (s - (t - bp)) + (p - bp);
  s = t;
}

struct Sums {  // per-thread float-pair accumulators
  float sr, cr, si, ci, q, cq;
  __device__ void zero() { sr = cr = si = ci = q = cq = 0.f; }
  __device__ void add(float re, float im) {
    ff_add(sr, cr, re);
    ff_add(si, ci, im);
    const float p = re * re;
    ff_add(q, cq, p);
    cq += fmaf(re, re, -p);
    const float p2 = im * im;
    ff_add(q, cq, p2);
    cq += fmaf(im, im, -p2);
  }
};

__device__ __forceinline__ double bsum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;  // every thread gets the same value
}

// Block sum of float pairs (h + l) on the FP32 pipe: two-sum reduction across
// the warp, one FP64 add per warp, the warp totals added in FP64 by thread 0.
// The result is valid in thread 0 only (the FP64 pipe of GB300 is too
// narrow to let every thread take part).
__device__ __forceinline__ double bsum_ff(float h, float l, double* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
    float s, e;
    two_sum(h, h2, s, e);
    e = e + (l + l2);
    two_sum(s, e, h, l);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)h + (double)l;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;
}

// The three float-pair sums of a pass (S re, S im, Q) and the marked
// amplitude (nonzero in one thread only) in one block reduction; results in
// thread 0: out[0..4] = S re, S im, Q, cm re, cm im.  The caller guarantees a
// block barrier between thread 0's last read of `sh` and this call.
__device__ __forceinline__ void bsum_pass(const float h[3], const float l[3], float cr, float ci, double* sh,
                                          double out[5]) {
  float H[3] = {h[0], h[1], h[2]}, L[3] = {l[0], l[1], l[2]};
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const float h2 = __shfl_xor_sync(0xffffffffu, H[v], o), l2 = __shfl_xor_sync(0xffffffffu, L[v], o);
      float s, e;
      two_sum(H[v], h2, s, e);
      e = e + (L[v] + l2);
      two_sum(s, e, H[v], L[v]);
    }
    cr += __shfl_xor_sync(0xffffffffu, cr, o);  // one nonzero term: exact
    ci += __shfl_xor_sync(0xffffffffu, ci, o);
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    for (int v = 0; v < 3; ++v) sh[v * 32 + w] = (double)H[v] + (double)L[v];
    sh[96 + w] = (double)cr;
    sh[128 + w] = (double)ci;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int v = 0; v < 5; ++v) {
      double t = 0.0;
      for (int i = 0; i < nw; ++i) t += sh[v * 32 + i];
      out[v] = t;
    }
}

// Sum of `nv` doubles over the cluster's ranks, read in parallel by warp 0
// (lane r reads rank r); the result is valid in thread 0.
template <int NV>
__device__ __forceinline__ void cluster_gather(cg::cluster_group& cluster, const Xch& xch, int buf, int first,
                                               double out[NV]) {
  if (threadIdx.x >= 32) return;
  const int G = (int)cluster.num_blocks();
  double v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  if ((int)threadIdx.x < G) {
    const Xch* x = cluster.map_shared_rank(&xch, (int)threadIdx.x);
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = x->v[buf][first + i];
  }
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = v[i];
}

__device__ __forceinline__ unsigned long long bsum_u64(unsigned long long v, unsigned long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long t = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;
}

// Pauli string of the errors drawn at `stage` (warp 0; lane q = qubit q).
__device__ __forceinline__ Pauli stage_errors(const TrajParams& P, int inst_id, int stage, int n, int lane,
                                              int* nerr) {
  unsigned xb = 0, zb = 0, yb = 0, eb = 0;
  if (lane < n) {
    uint32_t r[4];
    philox4x32_10((uint32_t)inst_id, (uint32_t)stage, (uint32_t)lane, TAG_NOISE, (uint32_t)P.seed,
                  (uint32_t)(P.seed >> 32), r);
    if (r[0] < P.thr_gate) {
      const int t = (int)(((uint64_t)r[1] * 3ull) >> 32);  // 0 X, 1 Y, 2 Z
      eb = 1;
      xb = (t == 0 || t == 1);
      zb = (t == 1 || t == 2);
      yb = (t == 1);
    }
  }
  Pauli p;
  p.x = __ballot_sync(0xffffffffu, xb);
  p.z = __ballot_sync(0xffffffffu, zb);
  p.a = __popc(__ballot_sync(0xffffffffu, yb)) & 3;  // Y = i X Z
  *nerr += __popc(__ballot_sync(0xffffffffu, eb));
  return p;
}

// One stage's Pauli string, drawn by one warp into slot `slot`.
__device__ __forceinline__ void draw_stage(const TrajParams& P, int inst_id, int stage, int n, int lane, Pauli* e,
                                           int* ne, int slot) {
  int c = 0;
  const Pauli p = stage_errors(P, inst_id, stage, n, lane, &c);
  if (lane == 0) {
    e[slot] = p;
    ne[slot] = c;
  }
}

// Thread 0's per-iteration scalars from W = sum of B's Z-signed O psi:
// the mean m = i^aB s W / N, broadcast as 2 m (re, im) and s = 1/sqrt(Q).
__device__ __forceinline__ void grover_scalars(double wr, double wi, double Q, int a, uint64_t N, float* sc) {
  const double s = 1.0 / sqrt(Q);
  double mr = wr, mi = wi;
  if (a == 1) { mr = -wi; mi = wr; }
  else if (a == 2) { mr = -wr; mi = -wi; }
  else if (a == 3) { mr = wi; mi = -wr; }
  const double scale = s / (double)N;
  sc[0] = (float)(2.0 * mr * scale);
  sc[1] = (float)(2.0 * mi * scale);
  sc[2] = (float)s;
}

// An iteration without errors (A = B = 1): out = 2 m - s psi, except at the
// marked index, where the oracle's sign flip gives 2 m + s psi.  Amplitudes
// move as 16-byte pairs, four pairs in flight per thread; the sums of each
// group of eight amplitudes are formed in plain FP32 (their rounding errors
// are independent and average out) and added into the float-pair
// accumulators once per group.
__device__ __forceinline__ void clean_pass(float2* psi, uint64_t lo, uint64_t hi, uint64_t m, float t2r, float t2i,
                                           float sf, int tid, int T, Sums& acc, float& cmr, float& cmi) {
  float4* p4 = reinterpret_cast<float4*>(psi);
  const uint32_t vlo = (uint32_t)(lo >> 1), vhi = (uint32_t)(hi >> 1), vm = (uint32_t)(m >> 1);
  const float nsf = -sf;
  const bool modd = (m & 1) != 0;
  auto one = [&](uint32_t v, const float4& u, float& bsr, float& bsi, float& bq) -> float4 {
    float4 o;
    o.x = fmaf(nsf, u.x, t2r);
    o.y = fmaf(nsf, u.y, t2i);
    o.z = fmaf(nsf, u.z, t2r);
    o.w = fmaf(nsf, u.w, t2i);
    if (v == vm) {
      if (modd) {
        o.z = fmaf(sf, u.z, t2r);
        o.w = fmaf(sf, u.w, t2i);
        cmr = o.z;
        cmi = o.w;
      } else {
        o.x = fmaf(sf, u.x, t2r);
        o.y = fmaf(sf, u.y, t2i);
        cmr = o.x;
        cmi = o.y;
      }
    }
    bsr += o.x + o.z;
    bsi += o.y + o.w;
    bq = fmaf(o.x, o.x, bq);
    bq = fmaf(o.y, o.y, bq);
    bq = fmaf(o.z, o.z, bq);
    bq = fmaf(o.w, o.w, bq);
    return o;
  };
  const uint32_t uT = (uint32_t)T;
  uint32_t v = vlo + (uint32_t)tid;
  for (; v + 3u * uT < vhi; v += 4u * uT) {
    const float4 u0 = p4[v], u1 = p4[v + uT], u2 = p4[v + 2u * uT], u3 = p4[v + 3u * uT];
    float bsr = 0.f, bsi = 0.f, bq = 0.f;
    p4[v] = one(v, u0, bsr, bsi, bq);
    p4[v + uT] = one(v + uT, u1, bsr, bsi, bq);
    p4[v + 2u * uT] = one(v + 2u * uT, u2, bsr, bsi, bq);
    p4[v + 3u * uT] = one(v + 3u * uT, u3, bsr, bsi, bq);
    ff_add(acc.sr, acc.cr, bsr);
    ff_add(acc.si, acc.ci, bsi);
    ff_add(acc.q, acc.cq, bq);
  }
  for (; v < vhi; v += uT) {
    const float4 u0 = p4[v];
    float bsr = 0.f, bsi = 0.f, bq = 0.f;
    p4[v] = one(v, u0, bsr, bsi, bq);
    ff_add(acc.sr, acc.cr, bsr);
    ff_add(acc.si, acc.ci, bsi);
    ff_add(acc.q, acc.cq, bq);
  }
}

__global__ void __launch_bounds__(512, 2) k_traj(TrajParams P) {
  cg::cluster_group cluster = cg::this_cluster();
  const int G = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int cid = blockIdx.x / G;
  __shared__ Xch xch;
  __shared__ double shd[160];  // five 32-entry rows for bsum_pass
  __shared__ unsigned long long shu[32];
  __shared__ Pauli pA, pB;
  __shared__ Pauli sh_e[4];  // the four stages of the next iteration
  __shared__ int sh_ne[4];
  __shared__ int sh_err;
  __shared__ double wtab[QC_TRAJ_MAX_QUBITS + 1];
  __shared__ unsigned long long sh_target;
  __shared__ float sh_sc[3];
  float2* psi = P.slots + (uint64_t)cid * P.slot_amps;
  const int tid = threadIdx.x, T = blockDim.x;
  for (;;) {
    if (rank == 0 && tid == 0) xch.inst = (int)atomicAdd(P.queue, 1u);
    cluster.sync();
    const int k = cluster.map_shared_rank(&xch, 0)->inst;
    cluster.sync();  // rank 0's shared memory is read before any CTA may exit
    if (k >= P.n_inst) break;
    const TrajInst I = P.inst[k];
    const int n = I.n;
    const uint64_t N = 1ull << n;
    const uint64_t per = N / (uint64_t)G, lo = (uint64_t)rank * per, hi = lo + per;
    const uint64_t m = I.marked;
    if (tid == 0) sh_err = 0;
    __syncthreads();
    int buf = 0;
    // ---- stage 0: E0 HALL |0..0> = E0 |s>: psi[j] = i^a (-1)^{|(j^x)&z|} 2^{-n/2}
    if (tid < 32) {
      int ne = 0;
      const Pauli e0 = stage_errors(P, I.id, 0, n, tid, &ne);
      if (tid == 0) {
        pA = e0;
        sh_err += ne;
      }
    }
    __syncthreads();
    {
      const Pauli e0 = pA;
      const float a0 = (float)(1.0 / sqrt(ldexp(1.0, n)));
      Sums acc;
      acc.zero();
      float cmr = 0.f, cmi = 0.f;
      for (uint64_t j = lo + tid; j < hi; j += T) {
        float re = (__popcll((j ^ e0.x) & e0.z) & 1) ? -a0 : a0, im = 0.f;
        ipow(e0.a, re, im);
        psi[j] = make_float2(re, im);
        acc.add(re, im);
        if (j == m) {
          cmr = re;
          cmi = im;
        }
      }
      const float hh[3] = {acc.sr, acc.si, acc.q}, ll[3] = {acc.cr, acc.ci, acc.cq};
      double red[5];
      bsum_pass(hh, ll, cmr, cmi, shd, red);
      if (tid == 0)
        for (int v = 0; v < 5; ++v) xch.v[buf][v] = red[v];
    }
    // the error draws of iteration 0 (stages 1..4, one per warp)
    if (I.iters > 0 && tid < 128) draw_stage(P, I.id, 1 + (tid >> 5), n, tid & 31, sh_e, sh_ne, tid >> 5);
    __threadfence();
    cluster.sync();
    // the per-iteration FP64 scalars live in thread 0 only (GB300's FP64 pipe
    // is too narrow for every thread to repeat them); the others receive the
    // three floats they need through shared memory
    double S[2] = {0, 0}, Q = 0, cm[2] = {0, 0};
    {
      double g5[5];
      cluster_gather<5>(cluster, xch, buf, 0, g5);
      if (tid == 0) {
        S[0] = g5[0]; S[1] = g5[1]; Q = g5[2]; cm[0] = g5[3]; cm[1] = g5[4];
      }
    }
    for (int it = 0; it < I.iters; ++it) {
      buf ^= 1;
      // three block barriers and one cluster barrier per iteration: the
      // scalars below, the block reduction and the cluster exchange
      if (tid == 0) {
        const Pauli B = pmul(hconj(sh_e[1]), sh_e[0]), A = pmul(sh_e[3], hconj(sh_e[2]));
        pB = B;
        pA = A;
        sh_err += sh_ne[0] + sh_ne[1] + sh_ne[2] + sh_ne[3];
        // sum of O psi: S with the marked amplitude's sign flipped
        if (!B.z) grover_scalars(S[0] - 2.0 * cm[0], S[1] - 2.0 * cm[1], Q, B.a, N, sh_sc);
      }
      __syncthreads();
      const Pauli A = pA, B = pB;
      if (B.z) {
        // sum of O psi, signed by Z^zB: one extra reading pass
        Sums acc;
        acc.zero();
        for (uint64_t j = lo + tid; j < hi; j += T) {
          float2 v = psi[j];
          if (__popcll(j & B.z) & 1) { v.x = -v.x; v.y = -v.y; }
          acc.add(v.x, v.y);
        }
        const double w0 = bsum_ff(acc.sr, acc.cr, shd);
        const double w1 = bsum_ff(acc.si, acc.ci, shd);
        if (tid == 0) {
          xch.v[buf][5] = w0;
          xch.v[buf][6] = w1;
        }
        __threadfence();
        cluster.sync();
        double g2[2];
        cluster_gather<2>(cluster, xch, buf, 5, g2);
        if (tid == 0) {
          const double sg = (__popcll(m & B.z) & 1) ? -1.0 : 1.0;
          grover_scalars(g2[0] - 2.0 * sg * cm[0], g2[1] - 2.0 * sg * cm[1], Q, B.a, N, sh_sc);
        }
        // publishes sh_sc; every CTA has read the W slots before they are reused
        cluster.sync();
      }
      const float t2r = sh_sc[0], t2i = sh_sc[1], sf = sh_sc[2];
      const uint64_t X = A.x ^ B.x;
      Sums acc;
      acc.zero();
      float cmr = 0.f, cmi = 0.f;
      if (((A.x | A.z | B.x | B.z) == 0) && ((A.a | B.a) == 0)) {
        clean_pass(psi, lo, hi, m, t2r, t2i, sf, tid, T, acc, cmr, cmi);
      } else {
        // out[j] from src = j ^ X
        auto out_of = [&](uint64_t j, float2 u) -> float2 {
          const uint64_t src = j ^ X;
          float re = u.x * sf, im = u.y * sf;
          if (src == m) { re = -re; im = -im; }                 // oracle
          if (__popcll(src & B.z) & 1) { re = -re; im = -im; }  // B's Z part
          ipow(B.a, re, im);
          re = t2r - re;                                        // D
          im = t2i - im;
          if (__popcll((j ^ A.x) & A.z) & 1) { re = -re; im = -im; }
          ipow(A.a, re, im);
          return make_float2(re, im);
        };
        if (X == 0) {
          for (uint64_t j = lo + tid; j < hi; j += T) {
            const float2 o = out_of(j, psi[j]);
            psi[j] = o;
            acc.add(o.x, o.y);
            if (j == m) { cmr = o.x; cmi = o.y; }
          }
        } else {
          const int hb = 63 - __clzll((long long)X);
          const uint64_t plo = lo / 2, phi = hi / 2;  // pair indices owned by this CTA
          for (uint64_t p = plo + tid; p < phi; p += T) {
            const uint64_t j = insert0(p, hb), jx = j ^ X;
            const float2 u = psi[j], v = psi[jx];
            const float2 oj = out_of(j, v), ojx = out_of(jx, u);
            psi[j] = oj;
            psi[jx] = ojx;
            acc.add(oj.x, oj.y);
            acc.add(ojx.x, ojx.y);
            if (j == m) { cmr = oj.x; cmi = oj.y; }
            if (jx == m) { cmr = ojx.x; cmi = ojx.y; }
          }
        }
      }
      // the next iteration's error draws (thread 0 read sh_e before the
      // barrier above), published by the reduction's barrier
      if (it + 1 < I.iters && tid < 128) draw_stage(P, I.id, 5 + 4 * it + (tid >> 5), n, tid & 31, sh_e, sh_ne, tid >> 5);
      {
        const float hh[3] = {acc.sr, acc.si, acc.q}, ll[3] = {acc.cr, acc.ci, acc.cq};
        double red[5];
        bsum_pass(hh, ll, cmr, cmi, shd, red);
        if (tid == 0) for (int v = 0; v < 5; ++v) xch.v[buf][v] = red[v];
      }
      __threadfence();
      cluster.sync();
      {
        double g5[5];
        cluster_gather<5>(cluster, xch, buf, 0, g5);
        if (tid == 0) { S[0] = g5[0]; S[1] = g5[1]; Q = g5[2]; cm[0] = g5[3]; cm[1] = g5[4]; }
      }
    }
    // ---- read-out: success probabilities and one seeded measurement
    buf ^= 1;
    if (tid <= n) {
      wtab[tid] = pow(P.p_ro, (double)tid) * pow(1.0 - P.p_ro, (double)(n - tid));
    }
    __syncthreads();
    double ro = 0.0;
    unsigned long long wt = 0;
    for (uint64_t j = lo + tid; j < hi; j += T) {
      const float2 v = psi[j];
      const double pj = __dadd_rn(__dmul_rn((double)v.x, (double)v.x), __dmul_rn((double)v.y, (double)v.y));
      ro = fma(pj, wtab[__popcll(j ^ m)], ro);
      wt += __double2ull_rz(pj * 4611686018427387904.0);
    }
    const double rop = bsum(ro, shd);
    const unsigned long long wtot = bsum_u64(wt, shu);
    if (tid == 0) {
      xch.v[buf][5] = rop;
      xch.w[buf] = wtot;
    }
    __threadfence();
    cluster.sync();
    double rosum = 0.0;
    unsigned long long off = 0, total = 0;
    for (int r = 0; r < G; ++r) {
      const Xch* x = cluster.map_shared_rank(&xch, r);
      rosum += x->v[buf][5];
      if (r < rank) off += x->w[buf];
      total += x->w[buf];
    }
    uint32_t rr[4];
    philox4x32_10((uint32_t)I.id, 0xFFFFFFFFu, 0u, TAG_MEAS, (uint32_t)P.seed, (uint32_t)(P.seed >> 32), rr);
    const unsigned long long target = __umul64hi(((unsigned long long)rr[0] << 32) | rr[1], total);
    // the CTA whose weight range holds the target finds the outcome
    if (total > 0 && target >= off && target < off + wtot) {
      // contiguous chunk per thread, block-level exclusive scan of chunk sums
      const uint64_t chunk = (per + T - 1) / T;
      const uint64_t c_lo = lo + (uint64_t)tid * chunk, c_hi = min(hi, c_lo + chunk);
      unsigned long long mine = 0;
      for (uint64_t j = c_lo; j < c_hi; ++j) {
        const float2 v = psi[j];
        const double pj = __dadd_rn(__dmul_rn((double)v.x, (double)v.x), __dmul_rn((double)v.y, (double)v.y));
        mine += __double2ull_rz(pj * 4611686018427387904.0);
      }
      // inclusive scan over threads (simple two-level through shared memory)
      unsigned long long x = mine;
      const int lane = tid & 31, wid = tid >> 5;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      __syncthreads();
      if (lane == 31) shu[wid] = x;
      __syncthreads();
      unsigned long long wo = 0;
      for (int w = 0; w < wid; ++w) wo += shu[w];
      const unsigned long long incl = off + wo + x, excl = incl - mine;
      if (target >= excl && target < incl) {
        unsigned long long run = excl;
        uint64_t j = c_lo;
        for (; j < c_hi; ++j) {
          const float2 v = psi[j];
          const double pj = __dadd_rn(__dmul_rn((double)v.x, (double)v.x), __dmul_rn((double)v.y, (double)v.y));
          run += __double2ull_rz(pj * 4611686018427387904.0);
          if (run > target) break;
        }
        sh_target = j;
      }
      __syncthreads();
      if (tid < 32) {
        uint64_t outc = sh_target;
        unsigned flip = 0;
        if (tid < n) {
          uint32_t q[4];
          philox4x32_10((uint32_t)I.id, 0xFFFFFFFFu, (uint32_t)tid, TAG_READ, (uint32_t)P.seed,
                        (uint32_t)(P.seed >> 32), q);
          flip = q[0] < P.thr_ro;
        }
        const unsigned fm = __ballot_sync(0xffffffffu, flip);
        if (tid == 0) {
          outc ^= (uint64_t)fm;
          P.outcome[I.id] = outc;
        }
      }
    }
    if (rank == 0 && tid == 0) {
      P.p_success[I.id] = (cm[0] * cm[0] + cm[1] * cm[1]) / Q;
      P.p_readout[I.id] = rosum / Q;
      P.n_errors[I.id] = (uint32_t)sh_err;
    }
    cluster.sync();  // slot, exchange buffers and xch.inst are free again
  }
}

}  // namespace qc

using namespace qc;

// The plan launches on a private non-blocking stream (graphs cannot be
// captured on the legacy default stream) joined to the caller's stream by
// events in both directions.
struct qc_traj_plan {
  cudaStream_t user;
  cudaStream_t stream;
  cudaEvent_t ev_in, ev_out;
  int n_inst;
  TrajInst* d_inst;
  float2* slots;
  unsigned* queue;
  int* status;
  uint64_t slot_amps;
  TrajParams params;
  int G, T, grid;
  cudaGraphExec_t gexec;
  qc_traj_out last_out;
  bool have_graph;
};

static qc_status traj_launch(qc_traj_plan* p, int G, int T, int grid, const TrajParams& prm) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(T);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = p->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = G;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_traj, prm);
  if (e != cudaSuccess) return cuda_fail(e, "trajectory launch");
  return QC_OK;
}

// Largest number of co-resident clusters for (G, T); 0 if not launchable.
static int traj_max_clusters(int G, int T) {
  cudaFuncSetAttribute(k_traj, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G * 64);
  cfg.blockDim = dim3(T);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = G;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, k_traj, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

QC_API qc_status qc_traj_plan_create(const qc_traj_desc* d, void* stream, int autotune, qc_traj_plan** out) {
  clear_error();
  if (!d || !out || d->n_inst < 1 || !d->nq || !d->marked || !d->iters) {
    set_error("bad trajectory descriptor");
    return QC_EINVAL;
  }
  *out = nullptr;
  if (!(d->p_readout >= 0.0 && d->p_readout <= 1.0)) {
    set_error("p_readout outside [0, 1]");
    return QC_EINVAL;
  }
  int nmin = 64, nmax = 0;
  std::vector<TrajInst> h(d->n_inst);
  for (int i = 0; i < d->n_inst; ++i) {
    const int n = d->nq[i];
    if (n < 1 || n > QC_TRAJ_MAX_QUBITS || d->iters[i] < 0 || d->marked[i] >= (1ull << n)) {
      set_error("instance %d: n = %d, iters = %d or marked item out of range", i, n, d->iters[i]);
      return QC_EINVAL;
    }
    h[i] = TrajInst{n, d->iters[i], d->marked[i], i, 0};
    nmin = std::min(nmin, n);
    nmax = std::max(nmax, n);
  }
  std::stable_sort(h.begin(), h.end(), [](const TrajInst& a, const TrajInst& b) {
    return ldexp((double)a.iters + 1.0, a.n) > ldexp((double)b.iters + 1.0, b.n);
  });
  qc_traj_plan* p = new qc_traj_plan();
  p->user = (cudaStream_t)stream;
  p->n_inst = d->n_inst;
  p->slot_amps = 1ull << nmax;
  p->have_graph = false;
  cudaError_t e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "trajectory plan stream");
  }
  // the plan's setup work follows whatever the caller queued before
  e = cudaEventRecord(p->ev_in, p->user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->ev_in, 0);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_inst, sizeof(TrajInst) * h.size());
  if (e == cudaSuccess) e = cudaMemcpy(p->d_inst, h.data(), sizeof(TrajInst) * h.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&p->queue, sizeof(unsigned) + sizeof(int));
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "trajectory plan");
  }
  p->status = reinterpret_cast<int*>(p->queue + 1);
  // candidate shapes: G CTAs per instance (G <= 2^{nmin-1}), T threads
  std::vector<int> Gs, Ts = {256, 512};
  for (int G = 1; G <= 16; G *= 2)
    if ((uint64_t)G * 2 <= (1ull << nmin) && (G >= 4 || nmax <= 14)) Gs.push_back(G);
  struct Cand {
    int G, T, grid;
  };
  std::vector<Cand> cands;
  for (int G : Gs)
    for (int T : Ts) {
      const int nc = traj_max_clusters(G, T);
      if (nc > 0) cands.push_back({G, T, nc * G});
    }
  if (cands.empty()) {
    cudaFree(p->d_inst);
    cudaFree(p->queue);
    delete p;
    set_error("no launchable cluster shape");
    return QC_ECUDA;
  }
  // slots for the largest grid among candidates
  int maxc = 0;
  for (auto& c : cands) maxc = std::max(maxc, c.grid / c.G);
  e = cudaMalloc(&p->slots, sizeof(float2) * p->slot_amps * (size_t)maxc);
  if (e != cudaSuccess) {
    cudaFree(p->d_inst);
    cudaFree(p->queue);
    delete p;
    return cuda_fail(e, "trajectory slots");
  }
  TrajParams base = {};
  base.inst = p->d_inst;
  base.n_inst = d->n_inst;
  base.slots = p->slots;
  base.slot_amps = p->slot_amps;
  base.seed = d->seed;
  base.thr_gate = d->thr_gate;
  base.thr_ro = d->thr_readout;
  base.p_ro = d->p_readout;
  base.queue = p->queue;
  base.status = p->status;
  p->params = base;
  // default: the largest cluster with 512 threads
  Cand best = cands.back();
  for (auto& c : cands)
    if (c.T == 512 && c.G >= best.G) best = c;
  if (autotune && cands.size() > 1) {
    // time each shape on an evenly spaced sample of the cost-sorted list
    const int stride = std::max(1, d->n_inst / 32);
    std::vector<TrajInst> samp;
    for (int i = 0; i < d->n_inst; i += stride) {
      TrajInst t = h[i];
      t.id = (int)samp.size();
      samp.push_back(t);
    }
    TrajInst* ds = nullptr;
    double* dout = nullptr;
    const size_t ns = samp.size();
    e = cudaMalloc(&ds, sizeof(TrajInst) * ns);
    if (e == cudaSuccess) e = cudaMemcpy(ds, samp.data(), sizeof(TrajInst) * ns, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&dout, ns * 32);
    if (e != cudaSuccess) {
      cudaFree(ds);
      cudaFree(p->d_inst);
      cudaFree(p->queue);
      cudaFree(p->slots);
      delete p;
      return cuda_fail(e, "autotune workspace");
    }
    TrajParams sp = base;
    sp.inst = ds;
    sp.n_inst = (int)ns;
    sp.p_success = dout;
    sp.p_readout = dout + ns;
    sp.outcome = reinterpret_cast<uint64_t*>(dout + 2 * ns);
    sp.n_errors = reinterpret_cast<uint32_t*>(dout + 3 * ns);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (auto& c : cands) {
      float ms_min = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {  // first run warms up, both are timed
        cudaMemsetAsync(p->queue, 0, sizeof(unsigned), p->stream);
        cudaEventRecord(e0, p->stream);
        if (traj_launch(p, c.G, c.T, c.grid, sp)) break;
        cudaEventRecord(e1, p->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_min = std::min(ms_min, ms);
      }
      if (cudaGetLastError() != cudaSuccess) continue;
      if (ms_min < best_ms) {
        best_ms = ms_min;
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(p->stream);
    cudaFree(ds);
    cudaFree(dout);
  }
  p->G = best.G;
  p->T = best.T;
  p->grid = best.grid;
  // later work on the caller's stream sees the uploaded descriptors
  e = cudaEventRecord(p->ev_out, p->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->user, p->ev_out, 0);
  if (e != cudaSuccess) {
    qc_traj_plan_free(p);
    return cuda_fail(e, "trajectory plan join");
  }
  *out = p;
  return check_launch("trajectory plan", autotune ? 2 * (int)cands.size() : 0);
}

QC_API qc_status qc_traj_plan_run(qc_traj_plan* p, const qc_traj_out* o) {
  clear_error();
  if (!p || !o || !o->p_success || !o->p_readout || !o->outcome || !o->n_errors) {
    set_error("bad plan or output pointers");
    return QC_EINVAL;
  }
  const bool same = p->have_graph && o->p_success == p->last_out.p_success && o->p_readout == p->last_out.p_readout &&
                    o->outcome == p->last_out.outcome && o->n_errors == p->last_out.n_errors;
  if (!same) {
    if (p->have_graph) {
      cudaGraphExecDestroy(p->gexec);
      p->have_graph = false;
    }
    TrajParams prm = p->params;
    prm.p_success = o->p_success;
    prm.p_readout = o->p_readout;
    prm.outcome = o->outcome;
    prm.n_errors = o->n_errors;
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    cudaMemsetAsync(p->queue, 0, sizeof(unsigned) + sizeof(int), p->stream);
    qc_status st = traj_launch(p, p->G, p->T, p->grid, prm);
    e = cudaStreamEndCapture(p->stream, &g);
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
    e = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    p->have_graph = true;
    p->last_out = *o;
  }
  // order: caller's stream -> plan stream (graph) -> caller's stream
  cudaError_t e = cudaEventRecord(p->ev_in, p->user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->ev_in, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(p->gexec, p->stream);
  if (e == cudaSuccess) e = cudaEventRecord(p->ev_out, p->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->user, p->ev_out, 0);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return check_launch("trajectory run", 1);
}

QC_API qc_status qc_traj_plan_info(const qc_traj_plan* p, int* G, int* T, int* grid) {
  clear_error();
  if (!p) {
    set_error("plan is NULL");
    return QC_EINVAL;
  }
  if (G) *G = p->G;
  if (T) *T = p->T;
  if (grid) *grid = p->grid;
  return QC_OK;
}

QC_API qc_status qc_traj_plan_free(qc_traj_plan* p) {
  clear_error();
  if (!p) return QC_OK;
  cudaStreamSynchronize(p->stream);
  if (p->have_graph) cudaGraphExecDestroy(p->gexec);
  cudaFree(p->d_inst);
  cudaFree(p->queue);
  cudaFree(p->slots);
  cudaEventDestroy(p->ev_in);
  cudaEventDestroy(p->ev_out);
  cudaStreamDestroy(p->stream);
  delete p;
  return QC_OK;
}
