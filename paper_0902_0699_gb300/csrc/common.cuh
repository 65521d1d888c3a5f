// Internal definitions shared by the CUDA translation units of the gate
// engine: the state handle, error reporting, launch sizing, complex helpers
// and index arithmetic.  Nothing here is exported.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/qc.h"
#include "ff.cuh"

#define QC_API extern "C" __attribute__((visibility("default")))

// Device scratch kept per state: running sums, means and block partials.
// Layout (doubles): [0,2) running amplitude sum, [2,4) Grover mean m,
// [4,8) misc scalars, [8, 8+2*QC_MAX_MARKED) saved marked amplitudes,
// then QC_PARTIALS doubles of reduction partials.
#define QC_SCR_SUM 0
#define QC_SCR_MEAN 2
#define QC_SCR_MISC 4
#define QC_SCR_MARKED 8
#define QC_SCR_PARTIALS (8 + 2 * QC_MAX_MARKED)
#define QC_PARTIALS 16384
#define QC_SCRATCH_DOUBLES (QC_SCR_PARTIALS + QC_PARTIALS)

struct qc_state {
  void* data;
  int n;
  qc_dtype dt;
  cudaStream_t stream;
  bool owns;
  bool sum_valid;  // scratch[QC_SCR_SUM] holds sum_i C_i of the current data
  int device;
  double* scratch;  // device, QC_SCRATCH_DOUBLES
  void* marked_dev;  // device copy of the last Grover marked list (lazy)
  std::vector<uint64_t> marked_host;  // what marked_dev holds
  bool grover_partial_ready;  // qc_grover_partial saved the marked amplitudes and P_r
};

// ------------------------------------------------------------ errors -----
namespace qc {

void set_error(const char* fmt, ...);
void clear_error();
qc_status cuda_fail(cudaError_t e, const char* what);
// Checks the last launch and adds `nkernels` (the kernels launched since
// the previous check) to the process-wide launch counter; returns QC_OK or
// QC_ECUDA (with message).
qc_status check_launch(const char* what, int nkernels = 1);

int sm_count();  // SMs of the current device (cached per device)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Grid for a grid-stride kernel over `items` work items of `per_block`
// items each, capped at `waves` x SMs blocks.
inline unsigned grid_for(int64_t items, int per_block, int waves) {
  int64_t b = ceil_div(items, per_block);
  int64_t cap = (int64_t)sm_count() * waves;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// Blocks of `kernel` that fit on one SM at once (cached per kernel).
int resident_blocks(const void* kernel, int threads, size_t smem);

// Grid for a grid-stride kernel: no more blocks than are resident at once
// (a second partial wave would leave most SMs idle at the end).
template <typename K>
inline unsigned resident_grid(K kernel, int threads, int64_t items, int per_block, size_t smem = 0) {
  int64_t b = ceil_div(items, per_block);
  const int64_t cap = (int64_t)sm_count() * resident_blocks((const void*)kernel, threads, smem);
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// ------------------------------------------------------ index helpers ----
// Insert a 0 bit at position `pos` of p: bits below pos stay, bits from pos
// up move one place up.
__host__ __device__ __forceinline__ uint64_t insert0(uint64_t p, int pos) {
  const uint64_t lo = p & ((1ull << pos) - 1ull);
  return ((p >> pos) << (pos + 1)) | lo;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply-xor round on the 4-word counter, key advanced by the Weyl
// constants between rounds.
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                       uint32_t k0, uint32_t k1, uint32_t out[4]) {
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// ------------------------------------------------------ complex types ----
template <typename R> struct CT;
template <> struct CT<double> {
  using V2 = double2;
  __host__ __device__ static V2 make(double a, double b) { return make_double2(a, b); }
};
template <> struct CT<float> {
  using V2 = float2;
  __host__ __device__ static V2 make(float a, float b) { return make_float2(a, b); }
};

template <typename R> struct Cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cmake(R a, R b) {
  Cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return cmake<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// a*b + c*d
template <typename R>
__device__ __forceinline__ Cx<R> cmul2(Cx<R> a, Cx<R> b, Cx<R> c, Cx<R> d) {
  R re = a.re * b.re;
  re = fma(-a.im, b.im, re);
  re = fma(c.re, d.re, re);
  re = fma(-c.im, d.im, re);
  R im = a.re * b.im;
  im = fma(a.im, b.re, im);
  im = fma(c.re, d.im, im);
  im = fma(c.im, d.re, im);
  return cmake<R>(re, im);
}

// A 2x2 operator passed by value to kernels.
template <typename R> struct Mat2 {
  Cx<R> m[4];  // U00 U01 U10 U11
};

template <typename R>
inline Mat2<R> mat_from_host(const double* U) {
  Mat2<R> M;
  for (int k = 0; k < 4; ++k) {
    M.m[k].re = (R)U[2 * k];
    M.m[k].im = (R)U[2 * k + 1];
  }
  return M;
}

// Structure of a 2x2 operator, decided on exact values on the host.
enum MatKind {
  MK_GENERAL = 0,
  MK_REAL = 1,     // all entries real
  MK_DIAG = 2,     // U01 = U10 = 0
  MK_PHASE1 = 3,   // diagonal with U00 = 1: only the bit-1 amplitudes change
  MK_ANTI = 4,     // U00 = U11 = 0
  MK_SWAPX = 5,    // U01 = U10 = 1, U00 = U11 = 0 (Pauli X): a pure exchange
  MK_HAD = 6,      // U00 = U01 = U10 = -U11 = h real
  MK_IDENT = 7,    // identity: nothing to do
  MK_PH_NEG = 8,   // diag(1, -1): the bit-1 amplitudes change sign (exact)
  MK_PH_I = 9,     // diag(1, i): (re, im) -> (-im, re) on bit 1 (exact)
  MK_PH_MI = 10    // diag(1, -i): (re, im) -> (im, -re) on bit 1 (exact)
};
MatKind classify(const double* U);

// Exact sign change of a double or float by flipping the sign bit with an
// integer operation (no floating-point instruction is issued).
__device__ __forceinline__ double neg_exact(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}
__device__ __forceinline__ float neg_exact(float x) { return __uint_as_float(__float_as_uint(x) ^ 0x80000000u); }

// Loads / stores of one amplitude.
template <typename R> struct AmpIO;
template <> struct AmpIO<double> {
  __device__ static Cx<double> ld(const double2* p) {
    double2 v = *p;
    return cmake<double>(v.x, v.y);
  }
  __device__ static void st(double2* p, Cx<double> z) { *p = make_double2(z.re, z.im); }
};
template <> struct AmpIO<float> {
  __device__ static Cx<float> ld(const float2* p) {
    float2 v = *p;
    return cmake<float>(v.x, v.y);
  }
  __device__ static void st(float2* p, Cx<float> z) { *p = make_float2(z.re, z.im); }
};

// Apply a structured 2x2 operator to (a0, a1).
template <typename R, int KIND>
__device__ __forceinline__ void apply2(const Mat2<R>& U, Cx<R>& a0, Cx<R>& a1) {
  if (KIND == MK_GENERAL) {
    Cx<R> b0 = cmul2(U.m[0], a0, U.m[1], a1);
    Cx<R> b1 = cmul2(U.m[2], a0, U.m[3], a1);
    a0 = b0;
    a1 = b1;
  } else if (KIND == MK_REAL) {
    const R u00 = U.m[0].re, u01 = U.m[1].re, u10 = U.m[2].re, u11 = U.m[3].re;
    Cx<R> b0 = cmake<R>(fma(u01, a1.re, u00 * a0.re), fma(u01, a1.im, u00 * a0.im));
    Cx<R> b1 = cmake<R>(fma(u11, a1.re, u10 * a0.re), fma(u11, a1.im, u10 * a0.im));
    a0 = b0;
    a1 = b1;
  } else if (KIND == MK_DIAG) {
    a0 = cmul(U.m[0], a0);
    a1 = cmul(U.m[3], a1);
  } else if (KIND == MK_PHASE1) {
    a1 = cmul(U.m[3], a1);
  } else if (KIND == MK_PH_NEG) {
    a1 = cmake<R>(neg_exact(a1.re), neg_exact(a1.im));
  } else if (KIND == MK_PH_I) {
    a1 = cmake<R>(neg_exact(a1.im), a1.re);
  } else if (KIND == MK_PH_MI) {
    a1 = cmake<R>(a1.im, neg_exact(a1.re));
  } else if (KIND == MK_ANTI) {
    Cx<R> b0 = cmul(U.m[1], a1);
    Cx<R> b1 = cmul(U.m[2], a0);
    a0 = b0;
    a1 = b1;
  } else if (KIND == MK_SWAPX) {
    Cx<R> t = a0;
    a0 = a1;
    a1 = t;
  } else if (KIND == MK_HAD) {
    // h*(a0+a1), h*(a0-a1) with one product shared: q = h*a1
    const R h = U.m[0].re;
    const R qr = h * a1.re, qi = h * a1.im;
    Cx<R> b0 = cmake<R>(fma(h, a0.re, qr), fma(h, a0.im, qi));
    Cx<R> b1 = cmake<R>(fma(h, a0.re, -qr), fma(h, a0.im, -qi));
    a0 = b0;
    a1 = b1;
  }
}

// True for the kinds that only touch the bit-1 amplitude of a pair.
__host__ __device__ constexpr bool touches_bit1_only(int k) {
  return k == MK_PHASE1 || k == MK_PH_NEG || k == MK_PH_I || k == MK_PH_MI;
}

// ---------------------------------------- complex128 in double-float -----
// A 2x2 operator split into double-float entries (built on the host).
struct Mat2ff {
  ffc m[4];
};
inline Mat2ff mat2ff_from_host(const double* U) {
  Mat2ff r;
  for (int k = 0; k < 4; ++k) r.m[k] = ffc_from_d(U[2 * k], U[2 * k + 1]);
  return r;
}

// The arithmetic kinds of apply2 in double-float (the exact kinds -- swaps,
// sign flips, identity -- never need it).
template <int KIND>
__device__ __forceinline__ void apply2_ff(const Mat2ff& U, ffc& a0, ffc& a1) {
  if (KIND == MK_GENERAL) {
    // each output component as one four-term dot (one renormalisation)
    const ffc b0 = ffc_make(ff_dot4(U.m[0].re, a0.re, ff_neg(U.m[0].im), a0.im, U.m[1].re, a1.re, ff_neg(U.m[1].im), a1.im),
                            ff_dot4(U.m[0].re, a0.im, U.m[0].im, a0.re, U.m[1].re, a1.im, U.m[1].im, a1.re));
    a1 = ffc_make(ff_dot4(U.m[2].re, a0.re, ff_neg(U.m[2].im), a0.im, U.m[3].re, a1.re, ff_neg(U.m[3].im), a1.im),
                  ff_dot4(U.m[2].re, a0.im, U.m[2].im, a0.re, U.m[3].re, a1.im, U.m[3].im, a1.re));
    a0 = b0;
  } else if (KIND == MK_REAL) {
    const ffc b0 = ffc_make(ff_dot2p(U.m[0].re, a0.re, U.m[1].re, a1.re), ff_dot2p(U.m[0].re, a0.im, U.m[1].re, a1.im));
    a1 = ffc_make(ff_dot2p(U.m[2].re, a0.re, U.m[3].re, a1.re), ff_dot2p(U.m[2].re, a0.im, U.m[3].re, a1.im));
    a0 = b0;
  } else if (KIND == MK_DIAG) {
    a0 = ffc_mul(U.m[0], a0);
    a1 = ffc_mul(U.m[3], a1);
  } else if (KIND == MK_PHASE1) {
    a1 = ffc_mul(U.m[3], a1);
  } else if (KIND == MK_ANTI) {
    const ffc b0 = ffc_mul(U.m[1], a1);
    a1 = ffc_mul(U.m[2], a0);
    a0 = b0;
  } else if (KIND == MK_HAD) {
    const ff h = U.m[0].re;
    const ffc b0 = ffc_scale(ffc_add(a0, a1), h);
    a1 = ffc_scale(ffc_sub(a0, a1), h);
    a0 = b0;
  }
}

// Kinds whose complex128 form runs in double-float.
__host__ __device__ constexpr bool uses_ff(int k) {
  return k == MK_GENERAL || k == MK_REAL || k == MK_DIAG || k == MK_ANTI || k == MK_HAD;
}

// Bytes per amplitude.
inline size_t amp_bytes(qc_dtype dt) { return dt == QC_C128 ? 16 : 8; }

// Validation helpers (set the error message and return QC_EINVAL).
qc_status check_state(const qc_state* s);
qc_status check_qubit(const qc_state* s, int t, const char* name);

// Launchers implemented in the .cu files.
qc_status launch_1q(qc_state* s, int t, const double* U);
qc_status launch_ctrl(qc_state* s, int c, int t, const double* U);
qc_status launch_swap(qc_state* s, int a, int b);
qc_status launch_fill_basis(qc_state* s, uint64_t idx);
qc_status launch_fill_uniform(qc_state* s);
qc_status launch_hall(qc_state* s);
qc_status launch_layer(qc_state* s, const double* U, uint64_t mask);
// Hadamard layers as Walsh-Hadamard tile passes (wht.cu), for n >= the
// returned minimum
int hadamard_layer_min_qubits(qc_dtype dt);
qc_status launch_hadamard_layer(qc_state* s, uint64_t mask);
qc_status launch_qft(qc_state* s);
qc_status launch_grover_step(qc_state* s, const uint64_t* marked, int m);
qc_status launch_grover_run(qc_state* s, const uint64_t* marked, int m, int iters);
qc_status launch_grover_partial(qc_state* s, const uint64_t* marked, int m, double* out_host);
qc_status launch_grover_apply(qc_state* s, const uint64_t* marked, int m, const double* mean);
qc_status launch_sum(qc_state* s);  // refreshes scratch[QC_SCR_SUM]
qc_status reduce_norm(const qc_state* s, double* out_host);
qc_status launch_probs(const qc_state* s, double* out);
qc_status reduce_expect(const qc_state* s, uint64_t x, uint64_t z, double* out_host);
qc_status launch_scale(qc_state* s, double f);
// probs: if not NULL, the Born probabilities are written there by the same
// pass that forms the sampler's block weights.
qc_status launch_sample(const qc_state* s, uint64_t seed, int64_t shots, uint64_t* out, double* probs = nullptr);

// Dense k-qubit blocks (dense.cu): the qubit map of a block, the packed
// device form of its operator, and an asynchronous launch.
#define DENSE_MAX_K 6
struct DenseMap {
  int k;
  int pos[DENSE_MAX_K];             // target qubits, ascending (for inserting zeros)
  uint64_t offs[1 << DENSE_MAX_K];  // offs[l]: bit b of l placed on qubit qubits[b]
};
qc_status dense_map(int n, int k, const int* qubits, DenseMap* M);
bool dense_uses_tc(qc_dtype dt, int k);
size_t dense_op_bytes(qc_dtype dt, int k);
void dense_pack(qc_dtype dt, int k, const double* U, void* host_out);
// spin_limit bounds each of the tensor-core kernel's mbarrier waits (polls);
// no_mma = 1 is the timeout self-test (no MMA is issued, so the first wait
// runs out with nothing asynchronous in flight).
#define QC_TC_SPIN_LIMIT (1u << 20)
// The ensemble density matrix of a complex64 batch (B <= 64) on the tensor
// cores (rho_tc.cu); synchronous.
qc_status rho_tc_c64(const float2* psi, int n, int B, const double* P_host, float2* rho, cudaStream_t s);

qc_status dense_launch(qc_state* s, const DenseMap& M, const void* dev_op, int* status,
                       uint32_t spin_limit = QC_TC_SPIN_LIMIT, int no_mma = 0);

}  // namespace qc
