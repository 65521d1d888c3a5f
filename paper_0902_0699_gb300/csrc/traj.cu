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
//
// At the error rates of interest most iterations draw no error, and such an
// iteration moves every unmarked amplitude by one common affine map (see
// Track below).  The draws of 256 iterations are made up front, in
// parallel; error-free iterations then only update FP64 scalars in thread
// 0, and the state is read and written only by iterations with errors (and
// once at the end), which apply the pending map on the fly.
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
  // optional: instance i's final state goes to states + state_off[i]
  // (amplitudes; ~0 skips the instance)
  float2* states;
  const uint64_t* state_off;
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

// Partial sums exchanged between the CTAs of a cluster, as float pairs
// (hi, lo), double-buffered: S re, S im, Q, cm re, cm im, W re, W im, aux.
struct Xch {
  int inst;
  int pad;
  float2 v[2][8];
  unsigned long long w[2];
};

// One float-pair accumulation step s + c += p (Knuth two-sum, error kept).
__device__ __forceinline__ void ff_add(float& s, float& c, float p) {
  const float t = s + p;
  const float bp = t - s;
  c += (s - (t - bp)) + (p - bp);
  s = t;
}

// Float-pair sum across a warp (every lane gets the total).
__device__ __forceinline__ void warp_ff_sum(float& h, float& l) {
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
    float s, e;
    two_sum(h, h2, s, e);
    e = e + (l + l2);
    two_sum(s, e, h, l);
  }
}

// Block sums of NV float pairs, all on the FP32 pipe (a single thread's FP64
// chain is slow on GB300): warp sums, then warp 0 sums the warp totals.  The
// results are valid in thread 0.  The caller guarantees a block barrier
// between thread 0's last read of `sh` (NV * 32 entries) and this call.
template <int NV>
__device__ __forceinline__ void block_ff_sum(float h[NV], float l[NV], float2* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    warp_ff_sum(h[v], l[v]);
    if (lane == 0) sh[v * 32 + w] = make_float2(h[v], l[v]);
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float2 x = lane < nw ? sh[v * 32 + lane] : make_float2(0.f, 0.f);
      h[v] = x.x;
      l[v] = x.y;
      warp_ff_sum(h[v], l[v]);
    }
  }
}

// Sum over the cluster's ranks of NV exchanged float pairs, read in parallel
// by warp 0 (lane r reads rank r); the result is valid in thread 0.
template <int NV>
__device__ __forceinline__ void cluster_gather(cg::cluster_group& cluster, const Xch& xch, int buf, int first,
                                               ff out[NV]) {
  if (threadIdx.x >= 32) return;
  const int G = (int)cluster.num_blocks();
  float h[NV], l[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) h[i] = l[i] = 0.f;
  if ((int)threadIdx.x < G) {
    const Xch* x = cluster.map_shared_rank(&xch, (int)threadIdx.x);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float2 y = x->v[buf][first + i];
      h[i] = y.x;
      l[i] = y.y;
    }
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    warp_ff_sum(h[i], l[i]);
    out[i] = ff_make(h[i], l[i]);
  }
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

// Thread 0's per-iteration scalars from W = sum of B's Z-signed O psi:
// the mean m = i^aB s W / N, broadcast as 2 m (re, im) and s = 1/sqrt(Q),
// in FP32 (the kernel's arithmetic precision; the same s scales both terms).
__device__ __forceinline__ void grover_scalars(ff wr, ff wi, ff Q, int a, int n, float* sc) {
  const float s = 1.f / sqrtf(Q.hi + Q.lo);
  float mr = wr.hi + wr.lo, mi = wi.hi + wi.lo;
  const float r0 = mr, i0 = mi;
  if (a == 1) { mr = -i0; mi = r0; }
  else if (a == 2) { mr = -r0; mi = -i0; }
  else if (a == 3) { mr = i0; mi = -r0; }
  const float scale = ldexpf(s, 1 - n);  // 2 s / N
  sc[0] = mr * scale;
  sc[1] = mi * scale;
  sc[2] = s;
}

// Runs of error-free iterations.  Without errors (A = B = 1) an iteration is
// the unitary map
//   psi_j -> g - psi_j (j != m),   c -> g + c,   g = 2 W / N,  W = S - 2 c,
// one common affine map for every unmarked amplitude; the new sum is S' = W
// and the squared norm Q is unchanged.  So such an iteration needs no pass
// over the state: thread 0 updates (S, c) and composes the map
//   virtual psi_j = a + b stored_j   (j != m; b = +-1; the marked one is c)
// in double-float.  The next iteration that draws an error (or the end of the run)
// applies the map while it reads the state, and renormalises.
struct Track {
  // double-float: a single thread's FP64 chain is slow on GB300, and these
  // updates run once per iteration
  ff S[2], c[2], a[2], Q;
  float b;
  bool mapped;  // the map is not the identity
  // From the last pass: Tz = sum_j (-1)^{|j&tz|} stored_j for the next
  // noisy iteration's Z mask tz (0: not taken) and the stored value at m.
  ff Tz[2], cst[2];
  uint32_t tz;
  __device__ void anchor(const ff g[7], uint32_t z) {  // after a pass with reductions
    S[0] = g[0];
    S[1] = g[1];
    Q = g[2];
    c[0] = cst[0] = g[3];
    c[1] = cst[1] = g[4];
    Tz[0] = g[5];
    Tz[1] = g[6];
    tz = z;
    a[0] = a[1] = ff_make(0.f, 0.f);
    b = 1.f;
    mapped = false;
  }
  // W = sum_j (-1)^{|j&z|} (O psi)_j for z = tz != 0 without reading the
  // state: with psi_j = a + b stored_j (j != m), psi_m = c, s = (-1)^{|m&z|}
  // and sum_j (-1)^{|j&z|} = 0,  W = b (Tz - s cst) - s (a + c).
  __device__ ff Wz(int i, bool s_neg) const {
    ff t = s_neg ? ff_add(Tz[i], cst[i]) : ff_sub(Tz[i], cst[i]);
    if (b < 0.f) t = ff_neg(t);
    const ff u = ff_add(a[i], c[i]);
    return s_neg ? ff_add(t, u) : ff_sub(t, u);
  }
  // k = 2/N, a power of two, so scaling by it is exact
  __device__ void clean_step(float k) {
    for (int i = 0; i < 2; ++i) {
      const ff w = W(i);
      const ff g = ff_make(k * w.hi, k * w.lo);
      a[i] = ff_sub(g, a[i]);
      c[i] = ff_add(g, c[i]);
      S[i] = w;
    }
    b = -b;
    mapped = true;
  }
  // W = S - 2 c, the sum of O psi
  __device__ ff W(int i) const { return ff_sub(S[i], ff_make(2.f * c[i].hi, 2.f * c[i].lo)); }
  // the pending map and the marked amplitude, as floats
  __device__ void to_args(float& ar, float& ai, float& bb, float& cr, float& ci) const {
    ar = a[0].hi + a[0].lo;
    ai = a[1].hi + a[1].lo;
    bb = b;
    cr = c[0].hi + c[0].lo;
    ci = c[1].hi + c[1].lo;
  }
};

// Per-thread sums of a pass: float pairs for S (re, im) and Q, fed by
// groups of a few outputs summed in plain FP32 (their rounding errors are
// independent and average out).
struct Acc {
  float sr, cr, si, ci, q, cq, gr, gi, gq;
  float tr, tcr, ti, tci, gtr, gti;  // sum of (-1)^{|j&tz|} o_j (when tz != 0)
  __device__ void zero() { sr = cr = si = ci = q = cq = gr = gi = gq = tr = tcr = ti = tci = gtr = gti = 0.f; }
  __device__ void add(float2 o) {
    gr += o.x;
    gi += o.y;
    gq = fmaf(o.x, o.x, fmaf(o.y, o.y, gq));
  }
  __device__ void add_t(float2 o, bool neg) {
    gtr += neg ? -o.x : o.x;
    gti += neg ? -o.y : o.y;
  }
  __device__ void flush() {
    ff_add(sr, cr, gr);
    ff_add(si, ci, gi);
    ff_add(q, cq, gq);
    ff_add(tr, tcr, gtr);
    ff_add(ti, tci, gti);
    gr = gi = gq = gtr = gti = 0.f;
  }
};

// The uniform data of one pass, from shared memory.
struct PassArgs {
  float ar, ai, b, cr, ci;  // pending map and the virtual marked amplitude
  float t2r, t2i, sf;       // 2 m and s of a noisy iteration
  uint32_t m, X, ax, az, bz;
  uint32_t tz;  // Z mask of the next noisy iteration's signed sum (0: none)
  int aa, ba;
};

__device__ __forceinline__ float2 virt(uint32_t j, float2 u, const PassArgs& q) {
  if (j == q.m) return make_float2(q.cr, q.ci);
  return make_float2(fmaf(q.b, u.x, q.ar), fmaf(q.b, u.y, q.ai));
}

// out[j] of a noisy iteration from the virtual amplitude u at src = j ^ X
__device__ __forceinline__ float2 noisy_out(uint32_t j, float2 u, const PassArgs& q) {
  const uint32_t src = j ^ q.X;
  float re = u.x * q.sf, im = u.y * q.sf;
  if ((src == q.m) != (bool)(__popc(src & q.bz) & 1)) {  // oracle, B's Z part
    re = -re;
    im = -im;
  }
  ipow(q.ba, re, im);
  re = q.t2r - re;  // D
  im = q.t2i - im;
  if (__popc((j ^ q.ax) & q.az) & 1) {
    re = -re;
    im = -im;
  }
  ipow(q.aa, re, im);
  return make_float2(re, im);
}

// A pass that maps every 16-byte vector v (amplitudes 2v, 2v+1) of [lo, hi)
// to f(v, stored vector); sums of the outputs and the output at m.  UNR
// vectors are loaded before any is stored, to keep loads in flight (the
// passes are bound by L2 latency).
template <int UNR, class F>
__device__ __forceinline__ void vec_pass(float4* p4, uint32_t lo, uint32_t hi, uint32_t m, int tid, int T, F f,
                                         Acc& acc, float& cmr, float& cmi, uint32_t tz = 0u) {
  const uint32_t vm = m >> 1, vhi = hi >> 1, uT = (uint32_t)T;
  auto one = [&](uint32_t v, const float4& u) {
    const float4 o = f(v, u);
    p4[v] = o;
    acc.add(make_float2(o.x, o.y));
    acc.add(make_float2(o.z, o.w));
    if (tz) {
      const bool s0 = __popc((2 * v) & tz) & 1;
      acc.add_t(make_float2(o.x, o.y), s0);
      acc.add_t(make_float2(o.z, o.w), s0 != (bool)(tz & 1u));
    }
    if (v == vm) {
      cmr = (m & 1) ? o.z : o.x;
      cmi = (m & 1) ? o.w : o.y;
    }
  };
  uint32_t v = (lo >> 1) + (uint32_t)tid;
  for (; v + (UNR - 1) * uT < vhi; v += UNR * uT) {
    float4 u[UNR];
#pragma unroll
    for (int i = 0; i < UNR; ++i) u[i] = p4[v + i * uT];
#pragma unroll
    for (int i = 0; i < UNR; ++i) {
      one(v + i * uT, u[i]);
      if (i % 4 == 3) acc.flush();
    }
  }
  for (; v < vhi; v += uT) {
    one(v, p4[v]);
    acc.flush();
  }
}

// A noisy iteration whose amplitudes move between vectors (X >> 1 != 0):
// vector pairs (v, v ^ (X >> 1)), each visited once.
__device__ __forceinline__ void pair_pass(float4* p4, uint32_t lo, uint32_t hi, int tid, int T, const PassArgs& q,
                                          Acc& acc, float& cmr, float& cmi) {
  const uint32_t Xv = q.X >> 1, vm = q.m >> 1;
  const int hb = 31 - __clz(Xv);
  const bool sw = q.X & 1u;
  auto two = [&](uint32_t v, uint32_t vx, const float4& u, const float4& w) {
    const float2 a0 = virt(2 * v, make_float2(u.x, u.y), q), a1 = virt(2 * v + 1, make_float2(u.z, u.w), q);
    const float2 b0 = virt(2 * vx, make_float2(w.x, w.y), q), b1 = virt(2 * vx + 1, make_float2(w.z, w.w), q);
    const float2 o0 = noisy_out(2 * v, sw ? b1 : b0, q), o1 = noisy_out(2 * v + 1, sw ? b0 : b1, q);
    const float2 o2 = noisy_out(2 * vx, sw ? a1 : a0, q), o3 = noisy_out(2 * vx + 1, sw ? a0 : a1, q);
    p4[v] = make_float4(o0.x, o0.y, o1.x, o1.y);
    p4[vx] = make_float4(o2.x, o2.y, o3.x, o3.y);
    acc.add(o0);
    acc.add(o1);
    acc.add(o2);
    acc.add(o3);
    if (q.tz) {
      const bool s0 = __popc((2 * v) & q.tz) & 1, s2 = __popc((2 * vx) & q.tz) & 1, odd = q.tz & 1u;
      acc.add_t(o0, s0);
      acc.add_t(o1, s0 != odd);
      acc.add_t(o2, s2);
      acc.add_t(o3, s2 != odd);
    }
    acc.flush();
    if (v == vm) {
      cmr = (q.m & 1) ? o1.x : o0.x;
      cmi = (q.m & 1) ? o1.y : o0.y;
    }
    if (vx == vm) {
      cmr = (q.m & 1) ? o3.x : o2.x;
      cmi = (q.m & 1) ? o3.y : o2.y;
    }
  };
  auto vec_of = [&](uint32_t p) { return ((p >> hb) << (hb + 1)) | (p & ((1u << hb) - 1u)); };
  const uint32_t phi = hi >> 2, uT = (uint32_t)T;
  uint32_t p = (lo >> 2) + (uint32_t)tid;
  for (; p + uT < phi; p += 2u * uT) {  // two vector pairs in flight
    const uint32_t v0 = vec_of(p), v1 = vec_of(p + uT);
    const float4 u0 = p4[v0], w0 = p4[v0 ^ Xv], u1 = p4[v1], w1 = p4[v1 ^ Xv];
    two(v0, v0 ^ Xv, u0, w0);
    two(v1, v1 ^ Xv, u1, w1);
  }
  if (p < phi) {
    const uint32_t v0 = vec_of(p);
    two(v0, v0 ^ Xv, p4[v0], p4[v0 ^ Xv]);
  }
}

// trunc(x^2 2^62) from the fields of a float (integer operations, exact):
// x = mm 2^(e - 150), so x^2 2^62 = mm^2 2^(2e - 238); |x| < 2.
__device__ __forceinline__ unsigned long long sqw(float x) {
  const uint32_t bits = __float_as_uint(x) & 0x7fffffffu;
  const int e = (int)(bits >> 23);
  if (e == 0) return 0ull;  // zero or subnormal: below one unit
  const unsigned long long mm = (bits & 0x7fffffu) | 0x800000u;
  const unsigned long long sq = mm * mm;
  const int sh = 2 * e - 238;
  if (sh >= 0) return sq << (sh < 16 ? sh : 16);
  return sh <= -64 ? 0ull : sq >> (-sh);
}

// Read-out weight of amplitude v: trunc(re^2 2^62) + trunc(im^2 2^62).
__device__ __forceinline__ unsigned long long ro_weight(float2 v) { return sqw(v.x) + sqw(v.y); }

// Iterations per table of error draws (shared memory: 12 KiB).  The
// dirty-iteration bitmask is written by threads 0..TCH-1, so a CTA has at
// least TCH threads (the plan's shapes use 256 or 512).
#define TCH 256

// MINB = resident CTAs per SM the register budget is sized for (the plan's
// autotuner picks): 2 caps registers at 64 (some spills), 1 leaves them free.
template <int MINB>
__global__ void __launch_bounds__(512, MINB) k_traj(TrajParams P) {
  cg::cluster_group cluster = cg::this_cluster();
  const int G = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int cid = blockIdx.x / G;
  __shared__ Xch xch;
  __shared__ float2 shf[7 * 32];  // block_ff_sum rows
  __shared__ unsigned long long shu[32];
  __shared__ Pauli pA;
  __shared__ int sh_err;
  __shared__ int sh_flag;
  __shared__ int sh_read;  // this noisy iteration needs the reading pass for W
  __shared__ float wtab[QC_TRAJ_MAX_QUBITS + 1];
  __shared__ unsigned long long sh_target;
  __shared__ PassArgs sh_q;
  // error draws of TCH iterations: X and Z masks and Y count per stage
  __shared__ uint32_t ex[TCH][4], ez[TCH][4];
  __shared__ int ey[TCH][4];
  __shared__ uint32_t dirty[TCH / 32];
  float2* psi = P.slots + (uint64_t)cid * P.slot_amps;
  float4* p4 = reinterpret_cast<float4*>(psi);
  const int tid = threadIdx.x, T = blockDim.x;
  for (;;) {
    if (rank == 0 && tid == 0) xch.inst = (int)atomicAdd(P.queue, 1u);
    cluster.sync();
    const int k = cluster.map_shared_rank(&xch, 0)->inst;
    cluster.sync();  // rank 0's shared memory is read before any CTA may exit
    if (k >= P.n_inst) break;
    const TrajInst I = P.inst[k];
    const int n = I.n;
    const uint32_t N = 1u << n;
    const uint32_t per = N / (uint32_t)G, lo = (uint32_t)rank * per, hi = lo + per;  // per >= 2
    const uint32_t m = (uint32_t)I.marked;
    if (tid == 0) sh_err = 0;
    __syncthreads();
    int buf = 0;
    // one block reduction of a pass's sums, exchanged over the cluster; the
    // totals re-anchor thread 0's scalars
    Track tr;
    auto reduce_anchor = [&](Acc& acc, float cmr, float cmi, uint32_t tz) {
      float h[7] = {acc.sr, acc.si, acc.q, cmr, cmi, acc.tr, acc.ti};
      float l[7] = {acc.cr, acc.ci, acc.cq, 0.f, 0.f, acc.tcr, acc.tci};
      block_ff_sum<7>(h, l, shf);
      if (tid == 0)
        for (int v = 0; v < 7; ++v) xch.v[buf][v] = make_float2(h[v], l[v]);
      __threadfence();
      cluster.sync();
      ff g7[7];
      cluster_gather<7>(cluster, xch, buf, 0, g7);
      if (tid == 0) tr.anchor(g7, tz);
    };
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
      const uint32_t x0 = (uint32_t)e0.x, z0 = (uint32_t)e0.z;
      const int a0p = e0.a;
      const float a0 = (float)(1.0 / sqrt(ldexp(1.0, n)));
      Acc acc;
      acc.zero();
      float cmr = 0.f, cmi = 0.f;
      auto amp = [&](uint32_t j) {
        float re = (__popc((j ^ x0) & z0) & 1) ? -a0 : a0, im = 0.f;
        ipow(a0p, re, im);
        return make_float2(re, im);
      };
      vec_pass<(MINB == 1 ? 8 : 4)>(p4, lo, hi, m, tid, T,
               [&](uint32_t v, const float4&) {
                 const float2 o0 = amp(2 * v), o1 = amp(2 * v + 1);
                 return make_float4(o0.x, o0.y, o1.x, o1.y);
               },
               acc, cmr, cmi);
      reduce_anchor(acc, cmr, cmi, 0u);
    }
    const float two_over_n = ldexpf(1.f, 1 - n);
    for (int base = 0; base < I.iters; base += TCH) {
      const int cnt = min(TCH, I.iters - base);
      // ---- the error draws of iterations base .. base+cnt-1, all at once
      for (int i = tid; i < TCH * 4; i += T) {
        (&ex[0][0])[i] = 0u;
        (&ez[0][0])[i] = 0u;
        (&ey[0][0])[i] = 0;
      }
      __syncthreads();
      if (P.thr_gate) {
        const int per_it = 4 * n, F = cnt * per_it;
        int hits = 0;
        for (int f = tid; f < F; f += T) {
          const int li = f / per_it, r = f - li * per_it, sg = r / n, q = r - sg * n;
          uint32_t x[4];
          philox4x32_10((uint32_t)I.id, (uint32_t)(1 + 4 * (base + li) + sg), (uint32_t)q, TAG_NOISE,
                        (uint32_t)P.seed, (uint32_t)(P.seed >> 32), x);
          if (x[0] < P.thr_gate) {
            const int t = (int)(((uint64_t)x[1] * 3ull) >> 32);  // 0 X, 1 Y, 2 Z
            if (t <= 1) atomicOr(&ex[li][sg], 1u << q);
            if (t >= 1) atomicOr(&ez[li][sg], 1u << q);
            if (t == 1) atomicAdd(&ey[li][sg], 1);
            ++hits;
          }
        }
        if (hits) atomicAdd(&sh_err, hits);
      }
      __syncthreads();
      if (tid < TCH) {
        const bool any = (ex[tid][0] | ex[tid][1] | ex[tid][2] | ex[tid][3] | ez[tid][0] | ez[tid][1] | ez[tid][2] |
                          ez[tid][3]) != 0u;
        const unsigned bal = __ballot_sync(0xffffffffu, any);
        if ((tid & 31) == 0) dirty[tid >> 5] = bal;
      }
      __syncthreads();
      for (int li = 0; li < cnt; ++li) {
        if (!((dirty[li >> 5] >> (li & 31)) & 1u)) {
          if (tid == 0) tr.clean_step(two_over_n);  // no pass, no barrier
          continue;
        }
        // ---- an iteration with errors: one pass over the state
        buf ^= 1;
        if (tid == 0) {
          Pauli e[4];
          for (int sg = 0; sg < 4; ++sg) e[sg] = Pauli{ex[li][sg], ez[li][sg], ey[li][sg] & 3};
          const Pauli B = pmul(hconj(e[1]), e[0]), A = pmul(e[3], hconj(e[2]));
          PassArgs q;
          tr.to_args(q.ar, q.ai, q.b, q.cr, q.ci);
          q.m = m;
          q.X = (uint32_t)(A.x ^ B.x);
          q.ax = (uint32_t)A.x;
          q.az = (uint32_t)A.z;
          q.bz = (uint32_t)B.z;
          q.aa = A.a;
          q.ba = B.a;
          // the next noisy iteration of this chunk: when its B has a Z part,
          // this pass also sums its outputs signed by that part, so the
          // next one needs no extra reading pass
          q.tz = 0u;
          for (int w = (li + 1) >> 5; w < TCH / 32; ++w) {
            uint32_t bits = dirty[w];
            if (w == ((li + 1) >> 5)) bits &= ~0u << ((li + 1) & 31);
            if (bits) {
              const int l2 = 32 * w + __ffs((int)bits) - 1;  // < cnt: later bits are never set
              const Pauli f0{ex[l2][0], ez[l2][0], ey[l2][0] & 3}, f1{ex[l2][1], ez[l2][1], ey[l2][1] & 3};
              q.tz = (uint32_t)pmul(hconj(f1), f0).z;
              break;
            }
          }
          const bool have_w = B.z && tr.tz == (uint32_t)B.z;  // taken by the previous pass
          sh_read = B.z && !have_w;
          if (!sh_read) {  // W = the sum of B's Z-signed O psi
            const bool sn = __popc(m & (uint32_t)B.z) & 1;
            float sc[3];
            if (B.z) grover_scalars(tr.Wz(0, sn), tr.Wz(1, sn), tr.Q, B.a, n, sc);
            else grover_scalars(tr.W(0), tr.W(1), tr.Q, B.a, n, sc);  // S with the marked amplitude's sign flipped
            q.t2r = sc[0];
            q.t2i = sc[1];
            q.sf = sc[2];
          }
          sh_q = q;
        }
        __syncthreads();
        if (sh_read) {
          // sum of O psi, signed by Z^zB: one extra reading pass
          const PassArgs q = sh_q;
          float hr = 0.f, lr = 0.f, hi_ = 0.f, li_ = 0.f;
          auto signed_sum = [&](uint32_t v, const float4& u, float& sr, float& si) {
            const float2 a0 = virt(2 * v, make_float2(u.x, u.y), q), a1 = virt(2 * v + 1, make_float2(u.z, u.w), q);
            const bool s0 = __popc((2 * v) & q.bz) & 1, s1 = s0 != (bool)(q.bz & 1u);
            sr += (s0 ? -a0.x : a0.x) + (s1 ? -a1.x : a1.x);
            si += (s0 ? -a0.y : a0.y) + (s1 ? -a1.y : a1.y);
          };
          const uint32_t vhi = hi >> 1, uT = (uint32_t)T;
          uint32_t v = (lo >> 1) + (uint32_t)tid;
          for (; v + 3u * uT < vhi; v += 4u * uT) {
            const float4 u0 = p4[v], u1 = p4[v + uT], u2 = p4[v + 2u * uT], u3 = p4[v + 3u * uT];
            float sr = 0.f, si = 0.f;
            signed_sum(v, u0, sr, si);
            signed_sum(v + uT, u1, sr, si);
            signed_sum(v + 2u * uT, u2, sr, si);
            signed_sum(v + 3u * uT, u3, sr, si);
            ff_add(hr, lr, sr);
            ff_add(hi_, li_, si);
          }
          for (; v < vhi; v += uT) {
            float sr = 0.f, si = 0.f;
            signed_sum(v, p4[v], sr, si);
            ff_add(hr, lr, sr);
            ff_add(hi_, li_, si);
          }
          float h2[2] = {hr, hi_}, l2[2] = {lr, li_};
          block_ff_sum<2>(h2, l2, shf);
          if (tid == 0) {
            xch.v[buf][5] = make_float2(h2[0], l2[0]);
            xch.v[buf][6] = make_float2(h2[1], l2[1]);
          }
          __threadfence();
          cluster.sync();
          ff g2[2];
          cluster_gather<2>(cluster, xch, buf, 5, g2);
          if (tid == 0) {
            // W = (signed sum of psi) - 2 sign(m) c
            const bool neg = __popc(m & q.bz) & 1;
            ff w[2];
            for (int i = 0; i < 2; ++i) {
              const ff c2 = ff_make(2.f * tr.c[i].hi, 2.f * tr.c[i].lo);
              w[i] = neg ? ff_add(g2[i], c2) : ff_sub(g2[i], c2);
            }
            float sc[3];
            grover_scalars(w[0], w[1], tr.Q, q.ba, n, sc);
            sh_q.t2r = sc[0];
            sh_q.t2i = sc[1];
            sh_q.sf = sc[2];
          }
          // publishes sh_q; every CTA has read the W slots before they are reused
          cluster.sync();
        }
        const PassArgs q = sh_q;
        Acc acc;
        acc.zero();
        float cmr = 0.f, cmi = 0.f;
        if ((q.X >> 1) == 0) {
          const bool sw = q.X & 1u;
          vec_pass<(MINB == 1 ? 8 : 4)>(p4, lo, hi, m, tid, T,
                   [&](uint32_t v, const float4& u) {
                     const float2 a0 = virt(2 * v, make_float2(u.x, u.y), q);
                     const float2 a1 = virt(2 * v + 1, make_float2(u.z, u.w), q);
                     const float2 o0 = noisy_out(2 * v, sw ? a1 : a0, q), o1 = noisy_out(2 * v + 1, sw ? a0 : a1, q);
                     return make_float4(o0.x, o0.y, o1.x, o1.y);
                   },
                   acc, cmr, cmi, q.tz);
        } else {
          pair_pass(p4, lo, hi, tid, T, q, acc, cmr, cmi);
        }
        reduce_anchor(acc, cmr, cmi, q.tz);
      }
      __syncthreads();  // the tables are read before the next chunk clears them
    }
    // ---- a pending map is applied once, with the sums of the result
    if (tid == 0) {
      sh_flag = tr.mapped;
      PassArgs q;
      tr.to_args(q.ar, q.ai, q.b, q.cr, q.ci);
      q.m = m;
      sh_q = q;
    }
    __syncthreads();
    if (sh_flag) {
      buf ^= 1;
      const PassArgs q = sh_q;
      Acc acc;
      acc.zero();
      float cmr = 0.f, cmi = 0.f;
      vec_pass<(MINB == 1 ? 8 : 4)>(p4, lo, hi, m, tid, T,
               [&](uint32_t v, const float4& u) {
                 const float2 o0 = virt(2 * v, make_float2(u.x, u.y), q), o1 = virt(2 * v + 1, make_float2(u.z, u.w), q);
                 return make_float4(o0.x, o0.y, o1.x, o1.y);
               },
               acc, cmr, cmi);
      reduce_anchor(acc, cmr, cmi, 0u);
    }
    // ---- read-out: success probabilities and one seeded measurement
    buf ^= 1;
    if (tid <= n) wtab[tid] = (float)(pow(P.p_ro, (double)tid) * pow(1.0 - P.p_ro, (double)(n - tid)));
    __syncthreads();
    float roh = 0.f, rol = 0.f;
    unsigned long long wt = 0;
    const uint64_t soff = P.states ? P.state_off[I.id] : ~0ull;
    float2* sdst = soff != ~0ull ? P.states + soff : nullptr;
    for (uint32_t v = (lo >> 1) + tid; v < (hi >> 1); v += T) {
      const float4 u = p4[v];
      const float2 v0 = make_float2(u.x, u.y), v1 = make_float2(u.z, u.w);
      if (sdst) {  // the state the read-out is drawn from
        sdst[2 * v] = v0;
        sdst[2 * v + 1] = v1;
      }
      const float p0 = fmaf(v0.x, v0.x, v0.y * v0.y), p1 = fmaf(v1.x, v1.x, v1.y * v1.y);
      ff_add(roh, rol, fmaf(p0, wtab[__popc((2 * v) ^ m)], p1 * wtab[__popc((2 * v + 1) ^ m)]));
      wt += ro_weight(v0) + ro_weight(v1);
    }
    float rh[1] = {roh}, rl[1] = {rol};
    block_ff_sum<1>(rh, rl, shf);
    const unsigned long long wtot = bsum_u64(wt, shu);
    if (tid == 0) {
      xch.v[buf][5] = make_float2(rh[0], rl[0]);
      xch.w[buf] = wtot;
    }
    __threadfence();
    cluster.sync();
    double rosum = 0.0;
    unsigned long long off = 0, total = 0;
    for (int r = 0; r < G; ++r) {
      const Xch* x = cluster.map_shared_rank(&xch, r);
      if (tid == 0) rosum += (double)x->v[buf][5].x + (double)x->v[buf][5].y;  // once per instance
      if (r < rank) off += x->w[buf];
      total += x->w[buf];
    }
    uint32_t rr[4];
    philox4x32_10((uint32_t)I.id, 0xFFFFFFFFu, 0u, TAG_MEAS, (uint32_t)P.seed, (uint32_t)(P.seed >> 32), rr);
    const unsigned long long target = __umul64hi(((unsigned long long)rr[0] << 32) | rr[1], total);
    // the CTA whose weight range holds the target finds the outcome
    if (total > 0 && target >= off && target < off + wtot) {
      // contiguous chunk per thread, block-level exclusive scan of chunk sums
      const uint32_t chunk = (per + T - 1) / T;
      const uint32_t c_lo = min(hi, lo + (uint32_t)tid * chunk), c_hi = min(hi, c_lo + chunk);
      unsigned long long mine = 0;
      for (uint32_t j = c_lo; j < c_hi; ++j) mine += ro_weight(psi[j]);
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
        uint32_t j = c_lo;
        for (; j < c_hi; ++j) {
          run += ro_weight(psi[j]);
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
      const double c0 = ff_to_d(tr.c[0]), c1 = ff_to_d(tr.c[1]), Q = ff_to_d(tr.Q);
      P.p_success[I.id] = (c0 * c0 + c1 * c1) / Q;
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
  int G, T, grid, minb;
  cudaGraphExec_t gexec;
  qc_traj_out last_out;
  float2* last_states;
  const uint64_t* last_state_off;
  bool have_graph;
};

typedef void (*TrajKernel)(TrajParams);
static TrajKernel traj_kernel(int minb) { return minb == 1 ? k_traj<1> : k_traj<2>; }

static qc_status traj_launch(qc_traj_plan* p, int G, int T, int grid, int minb, const TrajParams& prm) {
  if (T < TCH || T > 512 || T % 32) {  // the kernel's tables assume TCH <= T <= 512
    set_error("trajectory launch: %d threads per CTA (need %d..512, a multiple of 32)", T, TCH);
    return QC_EINVAL;
  }
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
  cudaError_t e = cudaLaunchKernelEx(&cfg, traj_kernel(minb), prm);
  if (e != cudaSuccess) return cuda_fail(e, "trajectory launch");
  return QC_OK;
}

// Largest number of co-resident clusters for (G, T); 0 if not launchable.
static int traj_max_clusters(int G, int T, int minb) {
  cudaFuncSetAttribute(traj_kernel(minb), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
  if (cudaOccupancyMaxActiveClusters(&nc, traj_kernel(minb), &cfg) != cudaSuccess) {
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
    int G, T, grid, minb;
  };
  std::vector<Cand> cands;
  for (int G : Gs)
    for (int T : Ts) {
      for (int minb = 1; minb <= 2; ++minb) {
        const int nc = traj_max_clusters(G, T, minb);
        if (nc > 0) cands.push_back({G, T, nc * G, minb});
      }
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
    // time each shape on an evenly spaced sample of the cost-sorted list,
    // large enough to fill every candidate's co-resident clusters four times
    // over: the run's time is a throughput, and a sample of a few instances
    // would only measure the latency of the largest ones (which favours wide
    // clusters that leave SMs idle)
    const int want = std::max(32, 4 * maxc);
    const int stride = std::max(1, d->n_inst / want);
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
        if (traj_launch(p, c.G, c.T, c.grid, c.minb, sp)) break;
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
  p->minb = best.minb;
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

static qc_status traj_run(qc_traj_plan* p, const qc_traj_out* o, const uint64_t* state_off, void* states) {
  if (!p || !o || !o->p_success || !o->p_readout || !o->outcome || !o->n_errors || (!state_off) != (!states)) {
    set_error("bad plan or output pointers");
    return QC_EINVAL;
  }
  float2* st = reinterpret_cast<float2*>(states);
  const bool same = p->have_graph && o->p_success == p->last_out.p_success && o->p_readout == p->last_out.p_readout &&
                    o->outcome == p->last_out.outcome && o->n_errors == p->last_out.n_errors &&
                    st == p->last_states && state_off == p->last_state_off;
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
    prm.states = st;
    prm.state_off = state_off;
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    cudaMemsetAsync(p->queue, 0, sizeof(unsigned) + sizeof(int), p->stream);
    qc_status rs = traj_launch(p, p->G, p->T, p->grid, p->minb, prm);
    e = cudaStreamEndCapture(p->stream, &g);
    if (rs) return rs;
    if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
    e = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    p->have_graph = true;
    p->last_out = *o;
    p->last_states = st;
    p->last_state_off = state_off;
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

QC_API qc_status qc_traj_plan_run(qc_traj_plan* p, const qc_traj_out* o) {
  clear_error();
  return traj_run(p, o, nullptr, nullptr);
}

QC_API qc_status qc_traj_plan_run_states(qc_traj_plan* p, const qc_traj_out* o, const uint64_t* state_off_dev,
                                         void* states_dev) {
  clear_error();
  if (!state_off_dev || !states_dev) {
    set_error("qc_traj_plan_run_states: NULL offsets or state buffer");
    return QC_EINVAL;
  }
  return traj_run(p, o, state_off_dev, states_dev);
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
