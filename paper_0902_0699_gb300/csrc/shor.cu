// The general two-qubit operator (TwoOpA, Eq. resmat2) and the quantum
// steps of Shor's algorithm (sec. 5.2): the state prepared with register 2
// holding x^j mod M (Eq. Shor2), the projective measurement of a register
// (ProjA, Eq. projreg2) and the QFT of register 1 (Appendix A's circuit on a
// sub-range of qubits).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace qc {

// ------------------------------------------------------------ TwoOpA -----
template <typename R> struct Mat4;
template <> struct Mat4<float> {
  Cx<float> v[16];
};
template <> struct Mat4<double> {
  ffc v[16];  // complex128 runs in double-float on the FP32 pipe
};

// Quartet q: bits t1 and t2 of n00 are zero; n01 = n00 + 2^t2,
// n10 = n00 + 2^t1, n11 = both; position 2*q_{t1} + q_{t2} (Eq. twoopB).
template <typename R>
__global__ void __launch_bounds__(256) k_2q(typename CT<R>::V2* __restrict__ s, uint64_t nq, int lo, int hi, int t1,
                                            int t2, Mat4<R> V) {
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += G) {
    const uint64_t n00 = insert0(insert0(q, lo), hi);
    const uint64_t idx[4] = {n00, n00 | (1ull << t2), n00 | (1ull << t1), n00 | (1ull << t1) | (1ull << t2)};
    if constexpr (sizeof(R) == 4) {
      Cx<float> a[4], b[4];
      for (int i = 0; i < 4; ++i) a[i] = AmpIO<float>::ld(s + idx[i]);
      for (int r = 0; r < 4; ++r) {
        Cx<float> acc = cmul(V.v[4 * r], a[0]);
        for (int c = 1; c < 4; ++c) {
          const Cx<float> p = cmul(V.v[4 * r + c], a[c]);
          acc = cmake(acc.re + p.re, acc.im + p.im);
        }
        b[r] = acc;
      }
      for (int i = 0; i < 4; ++i) AmpIO<float>::st(s + idx[i], b[i]);
    } else {
      ffc a[4], b[4];
      for (int i = 0; i < 4; ++i) {
        const double2 v = s[idx[i]];
        a[i] = ffc_from_d(v.x, v.y);
      }
      for (int r = 0; r < 4; ++r) {
        ffc acc = ffc_mul(V.v[4 * r], a[0]);
        for (int c = 1; c < 4; ++c) acc = ffc_add(acc, ffc_mul(V.v[4 * r + c], a[c]));
        b[r] = acc;
      }
      for (int i = 0; i < 4; ++i) s[idx[i]] = make_double2(ff_to_d(b[i].re), ff_to_d(b[i].im));
    }
  }
}

// ------------------------------------------------------ Shor: Eq. Shor2 --
// psi = 2^{-n1/2} sum_j |j>_{n1} |x^j mod M>_{n2}: register 1 is the high
// n1 bits, register 2 the low n2 bits (the paper's qubit order, register 1
// first).  One thread per j; x^j mod M by square-and-multiply (M < 2^32, so
// every product fits in 64 bits).
__device__ __forceinline__ uint64_t powmod(uint64_t x, uint64_t e, uint64_t M) {
  uint64_t r = 1 % M, b = x % M;
  while (e) {
    if (e & 1) r = (r * b) % M;
    b = (b * b) % M;
    e >>= 1;
  }
  return r;
}

template <typename R>
__global__ void k_shor_fill(typename CT<R>::V2* __restrict__ s, uint64_t n1count, int n2, uint64_t x, uint64_t M,
                            R amp) {
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n1count; j += G)
    s[(j << n2) | powmod(x, j, M)] = CT<R>::make(amp, (R)0);
}

// ------------------------------------------------- ProjA, Eq. projreg2 ---
// Probability of bits [lo, lo+w) == value (FP64 partials per block).
template <typename R>
__global__ void __launch_bounds__(256) k_proj_prob(const typename CT<R>::V2* __restrict__ s, uint64_t N, int lo,
                                                   uint64_t wmask, uint64_t value, double* __restrict__ part) {
  __shared__ double sh[32];
  double a = 0.0;
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) {
    if (((i >> lo) & wmask) != value) continue;
    const auto v = s[i];
    a = fma((double)v.x, (double)v.x, a);
    a = fma((double)v.y, (double)v.y, a);
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// Zero the amplitudes outside the outcome, scale the rest by f.
template <typename R>
__global__ void k_proj_apply(typename CT<R>::V2* __restrict__ s, uint64_t N, int lo, uint64_t wmask, uint64_t value,
                             R f) {
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) {
    auto v = s[i];
    if (((i >> lo) & wmask) == value) {
      v.x *= f;
      v.y *= f;
    } else {
      v.x = 0;
      v.y = 0;
    }
    s[i] = v;
  }
}

}  // namespace qc

using namespace qc;

QC_API qc_status qc_apply_2q(qc_state* s, int t1, int t2, const double V[32]) {
  clear_error();
  qc_status st = check_state(s);
  if (!st) st = check_qubit(s, t1, "t1");
  if (!st) st = check_qubit(s, t2, "t2");
  if (st) return st;
  if (t1 == t2) {
    set_error("TwoOpA on one qubit (%d)", t1);
    return QC_EINVAL;
  }
  if (!V) {
    set_error("operator pointer is NULL");
    return QC_EINVAL;
  }
  for (int k = 0; k < 32; ++k)
    if (!std::isfinite(V[k])) {
      set_error("operator entry %d is not finite", k);
      return QC_EINVAL;
    }
  if (s->n < 2) {
    set_error("TwoOpA needs n >= 2");
    return QC_EINVAL;
  }
  const int lo = std::min(t1, t2), hi = std::max(t1, t2);
  const uint64_t nq = (1ull << s->n) >> 2;
  const int T = 256;
  if (s->dt == QC_C128) {
    Mat4<double> M;
    for (int k = 0; k < 16; ++k) M.v[k] = ffc_from_d(V[2 * k], V[2 * k + 1]);
    k_2q<double><<<resident_grid(k_2q<double>, T, nq, T), T, 0, s->stream>>>(
        reinterpret_cast<double2*>(s->data), nq, lo, hi, t1, t2, M);
  } else {
    Mat4<float> M;
    for (int k = 0; k < 16; ++k) M.v[k] = Cx<float>{(float)V[2 * k], (float)V[2 * k + 1]};
    k_2q<float><<<resident_grid(k_2q<float>, T, nq, T), T, 0, s->stream>>>(
        reinterpret_cast<float2*>(s->data), nq, lo, hi, t1, t2, M);
  }
  s->sum_valid = false;
  return check_launch("apply_2q");
}

QC_API qc_status qc_shor_prepare(qc_state* s, int n2, uint64_t x, uint64_t M) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  const int n1 = s->n - n2;
  if (n2 < 1 || n1 < 1 || n1 > 40) {
    set_error("register sizes n1 = %d, n2 = %d invalid for n = %d", n1, n2, s->n);
    return QC_EINVAL;
  }
  if (M < 2 || M >= (1ull << 32) || M > (1ull << n2) || x < 1 || x >= M) {
    set_error("need 2 <= M < 2^32, M <= 2^n2 and 1 <= x < M (M = %llu, x = %llu)", (unsigned long long)M,
              (unsigned long long)x);
    return QC_EINVAL;
  }
  const size_t bytes = ((size_t)1 << s->n) * amp_bytes(s->dt);
  cudaError_t e = cudaMemsetAsync(s->data, 0, bytes, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "shor prepare");
  const uint64_t cnt = 1ull << n1;
  const double a = 1.0 / sqrt(ldexp(1.0, n1));
  if (s->dt == QC_C128)
    k_shor_fill<double><<<grid_for(cnt, 256, 8), 256, 0, s->stream>>>(reinterpret_cast<double2*>(s->data), cnt, n2,
                                                                      x, M, a);
  else
    k_shor_fill<float><<<grid_for(cnt, 256, 8), 256, 0, s->stream>>>(reinterpret_cast<float2*>(s->data), cnt, n2, x,
                                                                     M, (float)a);
  s->sum_valid = false;
  return check_launch("shor prepare");
}

QC_API qc_status qc_project(qc_state* s, int lo, int width, uint64_t value, double* prob_out) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (lo < 0 || width < 1 || lo + width > s->n || (width < 64 && value >= (1ull << width))) {
    set_error("bad register [%d, %d) or value for n = %d", lo, lo + width, s->n);
    return QC_EINVAL;
  }
  const uint64_t N = 1ull << s->n;
  const uint64_t wmask = (width >= 64) ? ~0ull : ((1ull << width) - 1ull);
  double* part = s->scratch + QC_SCR_PARTIALS;
  const unsigned nb = std::min<unsigned>(grid_for(N, 256 * 4, 8), QC_PARTIALS);
  if (s->dt == QC_C128)
    k_proj_prob<double><<<nb, 256, 0, s->stream>>>(reinterpret_cast<const double2*>(s->data), N, lo, wmask, value,
                                                   part);
  else
    k_proj_prob<float><<<nb, 256, 0, s->stream>>>(reinterpret_cast<const float2*>(s->data), N, lo, wmask, value,
                                                  part);
  st = check_launch("project (probability)");
  if (st) return st;
  std::vector<double> h(nb);
  cudaError_t e = cudaMemcpyAsync(h.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "project readback");
  double p = 0.0;
  for (unsigned i = 0; i < nb; ++i) p += h[i];
  if (prob_out) *prob_out = p;
  if (!(p > 0.0)) {
    set_error("outcome has probability zero");
    return QC_EINVAL;
  }
  const double f = 1.0 / sqrt(p);
  if (s->dt == QC_C128)
    k_proj_apply<double><<<grid_for(N, 256, 8), 256, 0, s->stream>>>(reinterpret_cast<double2*>(s->data), N, lo,
                                                                     wmask, value, f);
  else
    k_proj_apply<float><<<grid_for(N, 256, 8), 256, 0, s->stream>>>(reinterpret_cast<float2*>(s->data), N, lo,
                                                                    wmask, value, (float)f);
  s->sum_valid = false;
  return check_launch("project (apply)");
}

// Appendix A's circuit on the register of qubits [lo, lo+width): for the
// register's qubits from the most significant down, a Hadamard, then
// CPHASEK with each lower register qubit; then the pair swaps that restore
// the register's bit order.  Built from the gate kernels.
QC_API qc_status qc_qft_range(qc_state* s, int lo, int width) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (lo < 0 || width < 1 || lo + width > s->n) {
    set_error("bad register [%d, %d) for n = %d", lo, lo + width, s->n);
    return QC_EINVAL;
  }
  const double h = 1.0 / sqrt(2.0);
  const double H[8] = {h, 0, h, 0, h, 0, -h, 0};
  for (int i = width - 1; i >= 0 && !st; --i) {
    st = launch_1q(s, lo + i, H);
    for (int j = i - 1; j >= 0 && !st; --j) {
      const int k = i - j + 1;
      double U[8] = {1, 0, 0, 0, 0, 0, 0, 0};
      if (k == 1) {
        U[6] = -1.0;
      } else if (k == 2) {
        U[7] = 1.0;
      } else {
        double sn, cs;
        sincospi(2.0 / ldexp(1.0, k), &sn, &cs);
        U[6] = cs;
        U[7] = sn;
      }
      st = launch_ctrl(s, lo + i, lo + j, U);
    }
  }
  for (int i = 0; i < width / 2 && !st; ++i) st = launch_swap(s, lo + i, lo + width - 1 - i);
  return st;
}
