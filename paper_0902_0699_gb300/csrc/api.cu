// C-ABI entry points: state lifecycle, argument validation and dispatch to
// the kernel launchers.  Every entry point validates before launching and
// reports failures through qc_status plus a thread-local message.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace qc {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

qc_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return e == cudaErrorMemoryAllocation ? QC_ENOMEM : QC_ECUDA;
}

static std::atomic<unsigned long long> g_launches{0};

qc_status check_launch(const char* what, int nkernels) {
  g_launches.fetch_add((unsigned long long)nkernels, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return QC_OK;
}

int sm_count() {
  static std::atomic<int> cache[64];  // zero-initialised; threads may fill a slot concurrently (same value)
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  int c = cache[dev].load(std::memory_order_relaxed);
  if (c == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    c = v > 0 ? v : 1;
    cache[dev].store(c, std::memory_order_relaxed);
  }
  return c;
}

int resident_blocks(const void* kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(kernel, threads, smem, dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  cache[key] = nb;
  return nb;
}

static bool is0(double re, double im) { return re == 0.0 && im == 0.0; }

MatKind classify(const double* U) {
  const double *u00 = U, *u01 = U + 2, *u10 = U + 4, *u11 = U + 6;
  const bool offz = is0(u01[0], u01[1]) && is0(u10[0], u10[1]);
  if (offz) {
    if (u00[0] == 1.0 && u00[1] == 0.0) {
      if (u11[0] == 1.0 && u11[1] == 0.0) return MK_IDENT;
      if (u11[0] == -1.0 && u11[1] == 0.0) return MK_PH_NEG;
      if (u11[0] == 0.0 && u11[1] == 1.0) return MK_PH_I;
      if (u11[0] == 0.0 && u11[1] == -1.0) return MK_PH_MI;
      return MK_PHASE1;
    }
    return MK_DIAG;
  }
  if (is0(u00[0], u00[1]) && is0(u11[0], u11[1])) {
    if (u01[0] == 1.0 && u01[1] == 0.0 && u10[0] == 1.0 && u10[1] == 0.0) return MK_SWAPX;
    return MK_ANTI;
  }
  const bool real = u00[1] == 0.0 && u01[1] == 0.0 && u10[1] == 0.0 && u11[1] == 0.0;
  if (real && u00[0] == u01[0] && u00[0] == u10[0] && u11[0] == -u00[0]) return MK_HAD;
  if (real) return MK_REAL;
  return MK_GENERAL;
}

qc_status check_state(const qc_state* s) {
  if (!s) {
    set_error("state handle is NULL");
    return QC_EINVAL;
  }
  if (!s->data) {
    set_error("state has no buffer");
    return QC_EINVAL;
  }
  return QC_OK;
}

qc_status check_qubit(const qc_state* s, int t, const char* name) {
  if (t < 0 || t >= s->n) {
    set_error("%s = %d out of range [0, %d)", name, t, s->n);
    return QC_EINVAL;
  }
  return QC_OK;
}

static qc_status check_matrix(const double* U) {
  if (!U) {
    set_error("operator pointer is NULL");
    return QC_EINVAL;
  }
  for (int k = 0; k < 8; ++k) {
    if (!std::isfinite(U[k])) {
      set_error("operator entry %d is not finite", k);
      return QC_EINVAL;
    }
  }
  return QC_OK;
}

static qc_status new_state(void* data, int n, qc_dtype dt, void* stream, bool owns,
                           qc_state** out) {
  qc_state* s = new qc_state;
  s->data = data;
  s->n = n;
  s->dt = dt;
  s->stream = (cudaStream_t)stream;
  s->owns = owns;
  s->sum_valid = false;
  cudaGetDevice(&s->device);
  s->scratch = nullptr;
  s->marked_dev = nullptr;
  s->grover_partial_ready = false;
  cudaError_t e = cudaMalloc(&s->scratch, QC_SCRATCH_DOUBLES * sizeof(double));
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "scratch allocation");
  }
  *out = s;
  return QC_OK;
}

static qc_status check_n_dt(int n, qc_dtype dt) {
  if (n < 1 || n > QC_MAX_QUBITS) {
    set_error("n = %d out of range [1, %d]", n, QC_MAX_QUBITS);
    return QC_EINVAL;
  }
  if (dt != QC_C128 && dt != QC_C64) {
    set_error("unknown dtype %d", (int)dt);
    return QC_EINVAL;
  }
  return QC_OK;
}

}  // namespace qc

using namespace qc;

QC_API const char* qc_last_error(void) { return qc::g_err.c_str(); }

QC_API const char* qc_version(void) { return "qcgb300 0.1 (sm_103a)"; }

QC_API unsigned long long qc_kernel_launches(void) { return qc::g_launches.load(); }

QC_API qc_status qc_state_alloc(int n, qc_dtype dt, void* stream, qc_state** out) {
  clear_error();
  if (!out) {
    set_error("out is NULL");
    return QC_EINVAL;
  }
  *out = nullptr;
  qc_status st = check_n_dt(n, dt);
  if (st) return st;
  const size_t bytes = ((size_t)1 << n) * amp_bytes(dt);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "state allocation");
  qc_state* s = nullptr;
  st = new_state(p, n, dt, stream, true, &s);
  if (st) {
    cudaFree(p);
    return st;
  }
  st = launch_fill_basis(s, 0);
  if (st) {
    cudaFree(p);
    cudaFree(s->scratch);
    delete s;
    return st;
  }
  *out = s;
  return QC_OK;
}

QC_API qc_status qc_state_wrap(void* dev_ptr, int n, qc_dtype dt, void* stream, qc_state** out) {
  clear_error();
  if (!out) {
    set_error("out is NULL");
    return QC_EINVAL;
  }
  *out = nullptr;
  qc_status st = check_n_dt(n, dt);
  if (st) return st;
  if (!dev_ptr || ((uintptr_t)dev_ptr & 15u)) {
    set_error("device pointer is NULL or not 16-byte aligned");
    return QC_EINVAL;
  }
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, dev_ptr);
  if (e != cudaSuccess || (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    set_error("pointer is not CUDA device memory");
    return QC_EINVAL;
  }
  return new_state(dev_ptr, n, dt, stream, false, out);
}

QC_API qc_status qc_state_free(qc_state* s) {
  clear_error();
  if (!s) return QC_OK;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->owns && s->data) cudaFree(s->data);
  if (s->scratch) cudaFree(s->scratch);
  if (s->marked_dev) cudaFree(s->marked_dev);
  delete s;
  return QC_OK;
}

QC_API qc_status qc_state_reset(qc_state* s, uint64_t idx) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (idx >= (1ull << s->n)) {
    set_error("basis index %llu >= 2^%d", (unsigned long long)idx, s->n);
    return QC_EINVAL;
  }
  return launch_fill_basis(s, idx);
}

QC_API qc_status qc_state_uniform(qc_state* s) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  return launch_fill_uniform(s);
}

QC_API qc_status qc_state_info(const qc_state* s, void** dev_ptr, int* n, qc_dtype* dt) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (dev_ptr) *dev_ptr = s->data;
  if (n) *n = s->n;
  if (dt) *dt = s->dt;
  return QC_OK;
}

QC_API qc_status qc_state_set_stream(qc_state* s, void* stream) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  s->stream = (cudaStream_t)stream;
  return QC_OK;
}

QC_API qc_status qc_state_invalidate(qc_state* s) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  s->sum_valid = false;
  return QC_OK;
}

QC_API qc_status qc_apply_1q(qc_state* s, int t, const double U[8]) {
  clear_error();
  qc_status st = check_state(s);
  if (!st) st = check_qubit(s, t, "t");
  if (!st) st = check_matrix(U);
  if (st) return st;
  return launch_1q(s, t, U);
}

QC_API qc_status qc_apply_ctrl(qc_state* s, int c, int t, const double U[8]) {
  clear_error();
  qc_status st = check_state(s);
  if (!st) st = check_qubit(s, c, "c");
  if (!st) st = check_qubit(s, t, "t");
  if (!st) st = check_matrix(U);
  if (st) return st;
  if (c == t) {
    set_error("control and target are the same qubit (%d)", c);
    return QC_EINVAL;
  }
  return launch_ctrl(s, c, t, U);
}

QC_API qc_status qc_cnot(qc_state* s, int c, int t) {
  static const double X[8] = {0, 0, 1, 0, 1, 0, 0, 0};
  return qc_apply_ctrl(s, c, t, X);
}

QC_API qc_status qc_cphase(qc_state* s, int c, int t, int k) {
  clear_error();
  if (k < 1 || k > 1023) {
    set_error("k = %d out of range [1, 1023]", k);
    return QC_EINVAL;
  }
  double U[8] = {1, 0, 0, 0, 0, 0, 0, 0};
  if (k == 1) {
    U[6] = -1.0;
    U[7] = 0.0;
  } else if (k == 2) {
    U[6] = 0.0;
    U[7] = 1.0;
  } else {
    double sn, cs;
    sincospi(2.0 / ldexp(1.0, k), &sn, &cs);  // e^{2 pi i / 2^k}
    U[6] = cs;
    U[7] = sn;
  }
  return qc_apply_ctrl(s, c, t, U);
}

QC_API qc_status qc_swap(qc_state* s, int a, int b) {
  clear_error();
  qc_status st = check_state(s);
  if (!st) st = check_qubit(s, a, "a");
  if (!st) st = check_qubit(s, b, "b");
  if (st) return st;
  if (a == b) {
    set_error("swap of a qubit with itself (%d)", a);
    return QC_EINVAL;
  }
  return launch_swap(s, a, b);
}

QC_API qc_status qc_hall(qc_state* s) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  return launch_hall(s);
}

QC_API qc_status qc_apply_1q_layer(qc_state* s, const double* U, uint64_t mask) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (!U) {
    set_error("operator array is NULL");
    return QC_EINVAL;
  }
  if (s->n < 64 && (mask >> s->n)) {
    set_error("qubit mask has bits at or above n = %d", s->n);
    return QC_EINVAL;
  }
  for (int q = 0; q < s->n; ++q)
    if ((mask >> q) & 1) {
      st = check_matrix(U + 8 * q);
      if (st) return st;
    }
  return launch_layer(s, U, mask);
}

static qc_status check_marked(const qc_state* s, const uint64_t* marked, int m, int min_m = 1) {
  if ((m > 0 && !marked) || m < min_m || m > QC_MAX_MARKED) {
    set_error("need %d..%d marked items (got %d, ptr %p)", min_m, QC_MAX_MARKED, m, (const void*)marked);
    return QC_EINVAL;
  }
  const uint64_t N = 1ull << s->n;
  std::vector<uint64_t> v(marked, marked + m);
  for (int i = 0; i < m; ++i)
    if (v[i] >= N) {
      set_error("marked item %llu >= 2^%d", (unsigned long long)v[i], s->n);
      return QC_EINVAL;
    }
  std::sort(v.begin(), v.end());
  for (int i = 1; i < m; ++i)
    if (v[i] == v[i - 1]) {
      set_error("marked item %llu repeated", (unsigned long long)v[i]);
      return QC_EINVAL;
    }
  return QC_OK;
}

QC_API qc_status qc_grover_step(qc_state* s, const uint64_t* marked, int m) {
  clear_error();
  qc_status st = check_state(s);
  if (!st) st = check_marked(s, marked, m);
  if (st) return st;
  if (m >= (1ll << s->n)) {
    set_error("every basis state is marked");
    return QC_EINVAL;
  }
  return launch_grover_step(s, marked, m);
}

QC_API qc_status qc_grover_partial(qc_state* s, const uint64_t* marked, int m, double out[2]) {
  clear_error();
  qc_status st = check_state(s);
  if (!st) st = check_marked(s, marked, m, 0);
  if (st) return st;
  if (!out) {
    set_error("qc_grover_partial: out is NULL");
    return QC_EINVAL;
  }
  return launch_grover_partial(s, marked, m, out);
}

QC_API qc_status qc_grover_apply_mean(qc_state* s, const uint64_t* marked, int m, const double mean[2]) {
  clear_error();
  qc_status st = check_state(s);
  if (!st) st = check_marked(s, marked, m, 0);
  if (st) return st;
  if (!mean || !std::isfinite(mean[0]) || !std::isfinite(mean[1])) {
    set_error("qc_grover_apply_mean: mean is NULL or not finite");
    return QC_EINVAL;
  }
  return launch_grover_apply(s, marked, m, mean);
}

QC_API qc_status qc_grover_run(qc_state* s, const uint64_t* marked, int m, int iters) {
  clear_error();
  qc_status st = check_state(s);
  if (!st) st = check_marked(s, marked, m);
  if (st) return st;
  if (iters < 0) {
    set_error("iters = %d < 0", iters);
    return QC_EINVAL;
  }
  return launch_grover_run(s, marked, m, iters);
}

QC_API qc_status qc_qft(qc_state* s) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  return launch_qft(s);
}

QC_API qc_status qc_norm(const qc_state* s, double* out_host) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (!out_host) {
    set_error("out is NULL");
    return QC_EINVAL;
  }
  return reduce_norm(s, out_host);
}

QC_API qc_status qc_probs(const qc_state* s, double* out_dev) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (!out_dev) {
    set_error("out is NULL");
    return QC_EINVAL;
  }
  return launch_probs(s, out_dev);
}

QC_API qc_status qc_expect_pauli(const qc_state* s, uint64_t x, uint64_t z, double out[2]) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (!out) {
    set_error("out is NULL");
    return QC_EINVAL;
  }
  if (s->n < 64 && ((x | z) >> s->n)) {
    set_error("Pauli masks have bits at or above n = %d", s->n);
    return QC_EINVAL;
  }
  return reduce_expect(s, x, z, out);
}

QC_API qc_status qc_renormalize(qc_state* s, double* norm_out) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  double nrm = 0.0;
  st = reduce_norm(s, &nrm);
  if (st) return st;
  if (norm_out) *norm_out = nrm;
  if (!(nrm > 0.0)) {
    set_error("cannot renormalise a zero state");
    return QC_EINVAL;
  }
  return launch_scale(s, 1.0 / sqrt(nrm));
}

QC_API qc_status qc_probs_sample(const qc_state* s, double* probs_dev, uint64_t seed, int64_t shots,
                                 uint64_t* out_dev) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (!probs_dev || shots < 0 || (shots > 0 && !out_dev)) {
    set_error("NULL probabilities, bad shots (%lld) or NULL output", (long long)shots);
    return QC_EINVAL;
  }
  if (shots == 0) return launch_probs(s, probs_dev);
  return launch_sample(s, seed, shots, out_dev, probs_dev);
}

QC_API qc_status qc_sample(const qc_state* s, uint64_t seed, int64_t shots, uint64_t* out_dev) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (shots < 0 || (shots > 0 && !out_dev)) {
    set_error("bad shots (%lld) or NULL output", (long long)shots);
    return QC_EINVAL;
  }
  if (shots == 0) return QC_OK;
  return launch_sample(s, seed, shots, out_dev);
}
