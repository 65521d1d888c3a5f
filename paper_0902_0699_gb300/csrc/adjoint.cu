// Parameterised circuits on a batch of states and the adjoint gradient of
// E = <psi|H|psi> (not part of the QCMPI paper).
//
// Forward: psi_b = U_G .. U_1 |0..0>, one batched kernel per gate (grid.y is
// the batch element, so each block builds its element's rotation matrix
// once).  Backward: lambda = H psi (one gather pass over the Pauli terms),
// E = Re <psi|lambda>, then for j = G .. 1 a single fused pass per gate
// reads psi_j and lambda_j, accumulates Im <lambda_j|P_j|psi_j> (the
// derivative of U_j = exp(-i theta P_j / 2) gives
// dE/dtheta_j = 2 Re <lambda_j|(-i/2) P_j|psi_j> = Im <lambda_j|P_j|psi_j>)
// and applies U_j^dagger to both.  No intermediate state is stored: psi is
// uncomputed instead of checkpointed.
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

// Rotation matrices exp(-i sgn theta P / 2) for P = X, Y, Z; H.
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

// ------------------------------------------------------------ forward ----
template <typename R>
__global__ void __launch_bounds__(ADJ_T) k_fwd_gate(typename CT<R>::V2* __restrict__ psi, int n, GateDev g,
                                                    const double* __restrict__ theta, int64_t stride, double sgn) {
  using IO = AmpIO<R>;
  const int b = blockIdx.y;
  typename CT<R>::V2* s = psi + ((uint64_t)b << n);
  const double th = (g.kind <= QC_G_RZ) ? sgn * theta[(int64_t)b * stride + g.param] : 0.0;
  const Mat2<R> U = gate_matrix<R>(g.kind, th);
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

template <typename R>
__global__ void k_zero_state_batch(typename CT<R>::V2* __restrict__ psi, int n, int B) {
  const uint64_t N = 1ull << n, tot = N * (uint64_t)B;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (uint64_t)gridDim.x * blockDim.x)
    psi[i] = CT<R>::make((R)((i & (N - 1)) == 0 ? 1 : 0), (R)0);
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
template <> struct Acc<float> {
  double a = 0.0;
  float s = 0.f, c = 0.f;
  int cnt = 0;
  __device__ void put(float p, float e) {
    const float t = s + p;
    const float bp = t - s;
    c += ((s - (t - bp)) + (p - bp)) + e;
    s = t;
    if (++cnt == 32) flush();
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
    cnt = 0;
  }
  __device__ double value() const { return a; }
};

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
// Fused: accumulate Im <lam|P|psi> over the gate's pairs (P the generator
// X / Y / Z of a rotation on q0), then apply U^dagger to psi and lam.
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
  const Mat2<R> U = gate_matrix<R>(g.kind, th);
  const uint64_t np = (g.kind == QC_G_CNOT) ? (1ull << (n - 2)) : (1ull << (n - 1));
  Acc<R> acc;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t i1;
    const uint64_t i0 = gate_pair(g, p, i1);
    Cx<R> p0 = IO::ld(s + i0), p1 = IO::ld(s + i1);
    Cx<R> l0 = IO::ld(l + i0), l1 = IO::ld(l + i1);
    if (rot) {
      // Im(conj(a) b) = a.re b.im - a.im b.re
      if (g.kind == QC_G_RZ) {  // Z: conj(l0) p0 - conj(l1) p1
        acc.add(l0.re, p0.im); acc.sub(l0.im, p0.re);
        acc.sub(l1.re, p1.im); acc.add(l1.im, p1.re);
      } else if (g.kind == QC_G_RX) {  // X: conj(l0) p1 + conj(l1) p0
        acc.add(l0.re, p1.im); acc.sub(l0.im, p1.re);
        acc.add(l1.re, p0.im); acc.sub(l1.im, p0.re);
      } else {  // Y: conj(l0)(-i p1) + conj(l1)(i p0); Im(conj(a)(-i b)) = -Re(conj(a) b)
        acc.sub(l0.re, p1.re); acc.sub(l0.im, p1.im);
        acc.add(l1.re, p0.re); acc.add(l1.im, p0.im);
      }
    }
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

template <typename R>
static unsigned gx_for(int n, int B) {
  const uint64_t pairs = 1ull << (n - 1);
  uint64_t gx = (pairs + ADJ_T - 1) / ADJ_T;
  const uint64_t cap = std::max<uint64_t>(1, (uint64_t)sm_count() * 8 / (uint64_t)B);
  gx = std::min<uint64_t>(gx, std::min<uint64_t>(cap, ADJ_GX_MAX));
  return (unsigned)std::max<uint64_t>(gx, 1);
}

template <typename R>
static qc_status forward_impl(int n, int B, const qc_gate* gates, int n_gates, const double* theta,
                              int64_t stride, void* psi, cudaStream_t st) {
  using V2 = typename CT<R>::V2;
  V2* d = reinterpret_cast<V2*>(psi);
  const uint64_t tot = (uint64_t)B << n;
  k_zero_state_batch<R><<<grid_for(tot, ADJ_T, 8), ADJ_T, 0, st>>>(d, n, B);
  const dim3 grid(gx_for<R>(n, B), B);
  for (int i = 0; i < n_gates; ++i) {
    const GateDev g{gates[i].kind, gates[i].q0, gates[i].q1, gates[i].param};
    k_fwd_gate<R><<<grid, ADJ_T, 0, st>>>(d, n, g, theta, stride, 1.0);
  }
  return check_launch("circuit forward", 1 + n_gates);
}

template <typename R>
static qc_status adjoint_impl(int n, int B, const qc_gate* gates, int n_gates, const double* theta,
                              int64_t stride, const qc_pauli_term* H, int n_terms, void* psi, void* lam,
                              double* energy, double* grad, cudaStream_t st) {
  using V2 = typename CT<R>::V2;
  qc_status s = forward_impl<R>(n, B, gates, n_gates, theta, stride, psi, st);
  if (s) return s;
  V2* dp = reinterpret_cast<V2*>(psi);
  V2* dl = reinterpret_cast<V2*>(lam);
  const unsigned gx = gx_for<R>(n, B);
  const dim3 grid(gx, B);
  // workspace: Hamiltonian terms + partials
  TermsDev* dT = nullptr;
  double* part = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&dT, sizeof(TermsDev), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&part, sizeof(double) * (size_t)gx * B, st);
  if (e != cudaSuccess) {
    if (dT) cudaFreeAsync(dT, st);
    return cuda_fail(e, "adjoint workspace");
  }
  TermsDev* hT = nullptr;
  e = cudaMallocHost((void**)&hT, sizeof(TermsDev));
  if (e != cudaSuccess) {
    cudaFreeAsync(dT, st);
    cudaFreeAsync(part, st);
    return cuda_fail(e, "adjoint terms (host)");
  }
  hT->nt = n_terms;
  for (int k = 0; k < n_terms; ++k) {
    hT->x[k] = H[k].xmask;
    hT->z[k] = H[k].zmask;
    hT->c[k] = H[k].coeff;
  }
  e = cudaMemcpyAsync(dT, hT, sizeof(TermsDev), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)B * stride, st);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(st);
    cudaFreeHost(hT);
    cudaFreeAsync(dT, st);
    cudaFreeAsync(part, st);
    return cuda_fail(e, "adjoint setup");
  }
  k_apply_h<R><<<grid, ADJ_T, 0, st>>>(dp, dl, n, dT);
  k_energy<R><<<grid, ADJ_T, 0, st>>>(dp, dl, n, part);
  k_final_batch<<<B, ADJ_T, 0, st>>>(part, gx, energy, 1, 0);
  int nk = 3;
  for (int i = n_gates - 1; i >= 0; --i) {
    const GateDev g{gates[i].kind, gates[i].q0, gates[i].q1, gates[i].param};
    k_bwd_gate<R><<<grid, ADJ_T, 0, st>>>(dp, dl, n, g, theta, stride, part);
    ++nk;
    if (g.kind <= QC_G_RZ) {
      k_final_batch<<<B, ADJ_T, 0, st>>>(part, gx, grad, stride, g.param);
      ++nk;
    }
  }
  s = check_launch("adjoint backward", nk);
  e = cudaStreamSynchronize(st);  // the pinned term list is freed below
  cudaFreeHost(hT);
  cudaFreeAsync(dT, st);
  cudaFreeAsync(part, st);
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
