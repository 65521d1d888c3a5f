// Gate fusion: a circuit (one-qubit U(2), CNOT, CPHASEK, SWAP and
// controlled-U operators, sec. 3-4 and App. A) grouped into dense k-qubit
// blocks, each applied in one pass over the state (qc_apply_dense's
// kernels; complex64 5-qubit blocks on the tensor cores).  This is the
// "fused multi-gate pass" generalised from a layer of one-qubit gates to any
// gates whose qubits fit in the block.
//
// Fusion is greedy and dependency-aware: a block starts empty and scans the
// remaining operators in order; an operator joins the block when none of its
// qubits is touched by an earlier operator left out of this block and the
// block's qubit set stays within kmax; otherwise its qubits become blocked.
// Operators left out keep their order, so the blocks, applied in sequence,
// compose to the circuit exactly (operators on disjoint qubits commute).
// The block operator is composed on the host in FP64, by sparse row updates
// (each operator touches two rows per column, or permutes rows).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "common.cuh"

using namespace qc;

namespace {

typedef std::complex<double> cd;

struct FBlock {
  int k;
  int q[DENSE_MAX_K];
  std::vector<double> U;  // 2 * 4^k doubles, row-major, (re, im)
  DenseMap map;
};

struct Composer {
  std::vector<int> B;  // local bit b <-> qubit B[b]
  std::vector<cd> M;   // dim x dim, row-major
  int dim() const { return 1 << (int)B.size(); }
  int bit(int q) const {
    for (size_t b = 0; b < B.size(); ++b)
      if (B[b] == q) return (int)b;
    return -1;
  }
  void reset() {
    B.clear();
    M.assign(1, cd(1.0, 0.0));
  }
  void add_qubit(int q) {  // M <- I (x) M, the new qubit as the highest local bit
    const int d = dim();
    std::vector<cd> N((size_t)4 * d * d, cd(0.0, 0.0));
    for (int r = 0; r < 2 * d; ++r)
      for (int c = 0; c < 2 * d; ++c)
        if ((r >= d) == (c >= d)) N[(size_t)r * 2 * d + c] = M[(size_t)(r % d) * d + (c % d)];
    M.swap(N);
    B.push_back(q);
  }
  // M <- G M for a one-qubit G on local bit b, restricted to rows whose
  // control bit cb (if >= 0) is set
  void pair_update(int b, const cd G[4], int cb) {
    const int d = dim();
    for (int r0 = 0; r0 < d; ++r0) {
      if ((r0 >> b) & 1) continue;
      if (cb >= 0 && !((r0 >> cb) & 1)) continue;
      const int r1 = r0 | (1 << b);
      for (int c = 0; c < d; ++c) {
        const cd a = M[(size_t)r0 * d + c], e = M[(size_t)r1 * d + c];
        M[(size_t)r0 * d + c] = G[0] * a + G[1] * e;
        M[(size_t)r1 * d + c] = G[2] * a + G[3] * e;
      }
    }
  }
  void swap_rows(int r0, int r1) {
    const int d = dim();
    for (int c = 0; c < d; ++c) std::swap(M[(size_t)r0 * d + c], M[(size_t)r1 * d + c]);
  }
  void scale_row(int r, cd f) {
    const int d = dim();
    for (int c = 0; c < d; ++c) M[(size_t)r * d + c] *= f;
  }
};

uint64_t op_mask(const qc_op& o) {
  uint64_t m = 1ull << o.q0;
  if (o.kind != QC_OP_1Q) m |= 1ull << o.q1;
  return m;
}

cd cphase_factor(int k) {
  if (k == 1) return cd(-1.0, 0.0);
  if (k == 2) return cd(0.0, 1.0);
  const double a = 2.0 * M_PI / std::ldexp(1.0, k);
  return cd(std::cos(a), std::sin(a));
}

void absorb(Composer& C, const qc_op& o) {
  const int b0 = C.bit(o.q0), b1 = o.kind == QC_OP_1Q ? -1 : C.bit(o.q1);
  const int d = C.dim();
  switch (o.kind) {
    case QC_OP_1Q: {
      const cd G[4] = {cd(o.m[0], o.m[1]), cd(o.m[2], o.m[3]), cd(o.m[4], o.m[5]), cd(o.m[6], o.m[7])};
      C.pair_update(b0, G, -1);
      break;
    }
    case QC_OP_CTRL: {
      const cd G[4] = {cd(o.m[0], o.m[1]), cd(o.m[2], o.m[3]), cd(o.m[4], o.m[5]), cd(o.m[6], o.m[7])};
      C.pair_update(b1, G, b0);
      break;
    }
    case QC_OP_CNOT:
      for (int r = 0; r < d; ++r)
        if (((r >> b0) & 1) && !((r >> b1) & 1)) C.swap_rows(r, r | (1 << b1));
      break;
    case QC_OP_CPHASE: {
      const cd f = cphase_factor(o.k);
      for (int r = 0; r < d; ++r)
        if (((r >> b0) & 1) && ((r >> b1) & 1)) C.scale_row(r, f);
      break;
    }
    case QC_OP_SWAP:
      for (int r = 0; r < d; ++r)
        if (((r >> b0) & 1) && !((r >> b1) & 1)) C.swap_rows(r, (r & ~(1 << b0)) | (1 << b1));
      break;
  }
}

}  // namespace

struct qc_fused_plan {
  int n, kmax;
  std::vector<FBlock> blocks;
  struct Dev {
    void* buf = nullptr;
    std::vector<size_t> off;
    int* status = nullptr;
    int device = -1;
  } dev[2];
};

QC_API qc_status qc_fused_plan_create(int n, const qc_op* ops, int n_ops, int kmax, int pad, qc_fused_plan** out) {
  clear_error();
  if (!out || n < 1 || n > 34 || n_ops < 0 || (n_ops > 0 && !ops) || kmax < 2 || kmax > DENSE_MAX_K) {
    set_error("qc_fused_plan_create: bad arguments (n = %d, n_ops = %d, kmax = %d in 2..%d)", n, n_ops, kmax,
              DENSE_MAX_K);
    return QC_EINVAL;
  }
  *out = nullptr;
  for (int i = 0; i < n_ops; ++i) {
    const qc_op& o = ops[i];
    const bool two = o.kind != QC_OP_1Q;
    bool ok = o.kind >= QC_OP_1Q && o.kind <= QC_OP_CTRL && o.q0 >= 0 && o.q0 < n;
    if (two) ok = ok && o.q1 >= 0 && o.q1 < n && o.q1 != o.q0;
    if (o.kind == QC_OP_CPHASE) ok = ok && o.k >= 1 && o.k <= 62;
    if (o.kind == QC_OP_1Q || o.kind == QC_OP_CTRL)
      for (int e = 0; e < 8; ++e) ok = ok && std::isfinite(o.m[e]);
    if (!ok) {
      set_error("qc_fused_plan_create: operator %d (kind %d, qubits %d, %d) is invalid", i, o.kind, o.q0, o.q1);
      return QC_EINVAL;
    }
  }
  qc_fused_plan* p = new qc_fused_plan();
  p->n = n;
  p->kmax = std::min(kmax, n);
  const uint64_t all = (n == 64) ? ~0ull : ((1ull << n) - 1);
  std::vector<int> rem(n_ops), next;
  for (int i = 0; i < n_ops; ++i) rem[i] = i;
  Composer C;
  while (!rem.empty()) {
    C.reset();
    uint64_t blocked = 0, inB = 0;
    next.clear();
    for (size_t idx = 0; idx < rem.size(); ++idx) {
      if (blocked == all) {  // every qubit waits on a left-out operator: the block is complete
        next.insert(next.end(), rem.begin() + idx, rem.end());
        break;
      }
      const qc_op& o = ops[rem[idx]];
      const uint64_t m = op_mask(o);
      if ((m & blocked) || __builtin_popcountll(inB | m) > p->kmax) {
        blocked |= m;
        next.push_back(rem[idx]);
        continue;
      }
      for (uint64_t nm = m & ~inB; nm; nm &= nm - 1) C.add_qubit(__builtin_ctzll(nm));
      inB |= m;
      absorb(C, o);
    }
    if (pad)  // pad to kmax qubits (complex64 5-qubit blocks run on the tensor cores)
      for (int q = 0; q < n && (int)C.B.size() < p->kmax; ++q)
        if (!((inB >> q) & 1)) {
          C.add_qubit(q);
          inB |= 1ull << q;
        }
    FBlock blk;
    blk.k = (int)C.B.size();
    for (int b = 0; b < blk.k; ++b) blk.q[b] = C.B[b];
    const int d = C.dim();
    blk.U.resize((size_t)2 * d * d);
    for (int e = 0; e < d * d; ++e) {
      blk.U[2 * e] = C.M[e].real();
      blk.U[2 * e + 1] = C.M[e].imag();
    }
    if (dense_map(n, blk.k, blk.q, &blk.map)) {
      delete p;
      return QC_EINVAL;
    }
    p->blocks.push_back(std::move(blk));
    rem.swap(next);
  }
  *out = p;
  return QC_OK;
}

QC_API qc_status qc_fused_plan_info(const qc_fused_plan* p, int* n_blocks, int* kmax) {
  clear_error();
  if (!p) {
    set_error("plan is NULL");
    return QC_EINVAL;
  }
  if (n_blocks) *n_blocks = (int)p->blocks.size();
  if (kmax) *kmax = p->kmax;
  return QC_OK;
}

QC_API qc_status qc_fused_plan_block(const qc_fused_plan* p, int i, int* k, int* qubits, double* U) {
  clear_error();
  if (!p || i < 0 || i >= (int)p->blocks.size()) {
    set_error("qc_fused_plan_block: no block %d", i);
    return QC_EINVAL;
  }
  const FBlock& b = p->blocks[i];
  if (k) *k = b.k;
  if (qubits)
    for (int j = 0; j < b.k; ++j) qubits[j] = b.q[j];
  if (U) memcpy(U, b.U.data(), sizeof(double) * b.U.size());
  return QC_OK;
}

QC_API qc_status qc_fused_plan_run(qc_state* s, qc_fused_plan* p) {
  clear_error();
  qc_status st = check_state(s);
  if (st) return st;
  if (!p || p->n != s->n) {
    set_error("qc_fused_plan_run: plan is NULL or built for another qubit count");
    return QC_EINVAL;
  }
  if (p->blocks.empty()) return QC_OK;
  qc_fused_plan::Dev& d = p->dev[s->dt == QC_C64 ? 1 : 0];
  int dev = 0;
  cudaGetDevice(&dev);
  if (!d.buf || d.device != dev) {  // packed operators, uploaded once per dtype and device
    if (d.buf) cudaFree(d.buf);
    d.buf = nullptr;
    d.off.clear();
    size_t total = 0;
    for (const FBlock& b : p->blocks) {
      d.off.push_back(total);
      total += (dense_op_bytes(s->dt, b.k) + 255) / 256 * 256;
    }
    std::vector<unsigned char> host(total + 256, 0);
    for (size_t i = 0; i < p->blocks.size(); ++i)
      dense_pack(s->dt, p->blocks[i].k, p->blocks[i].U.data(), host.data() + d.off[i]);
    cudaError_t e = cudaMalloc(&d.buf, total + 256);
    if (e == cudaSuccess) e = cudaMemcpy(d.buf, host.data(), total + 256, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      if (d.buf) cudaFree(d.buf);
      d.buf = nullptr;
      return cuda_fail(e, "fused plan operators");
    }
    d.status = reinterpret_cast<int*>(reinterpret_cast<char*>(d.buf) + total);
    d.device = dev;
  }
  bool tc = false;
  cudaError_t e = cudaMemsetAsync(d.status, 0, sizeof(int), s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "fused plan status reset");
  for (size_t i = 0; i < p->blocks.size(); ++i) {
    const FBlock& b = p->blocks[i];
    tc |= dense_uses_tc(s->dt, b.k);
    dense_launch(s, b.map, reinterpret_cast<char*>(d.buf) + d.off[i], d.status);
  }
  st = check_launch("fused plan", (int)p->blocks.size());
  if (!st && tc) {
    int h = 0;
    e = cudaMemcpyAsync(&h, d.status, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "fused plan status");
    else if (h) {
      set_error("fused plan: a tensor-core block's mbarrier wait timed out");
      st = QC_ETIMEOUT;
    }
  }
  return st;
}

QC_API qc_status qc_fused_plan_free(qc_fused_plan* p) {
  clear_error();
  if (!p) return QC_OK;
  for (auto& d : p->dev)
    if (d.buf) {
      cudaDeviceSynchronize();
      cudaFree(d.buf);
    }
  delete p;
  return QC_OK;
}
