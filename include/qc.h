/*
 * qc.h -- C ABI of the GB300 state-vector gate engine.
 *
 * The operations are those of the QCMPI paper (Tabakin & Julia-Diaz,
 * arXiv:0902.0699): a 2^n-amplitude complex state vector in "standard order"
 * (sec. 2, Eq. staten / Eq. ampn) acted on by one-qubit operators (sec. 3,
 * Eq. resmat1), two-qubit operators and their CNOT / CPHASE / CPHASEK special
 * cases (sec. 4, Eqs. resmat2, cphasek), the Hadamard on all qubits (HALL,
 * Eq. HALL), Grover's oracle and inversion (sec. 5.1, Eqs. oracle1,
 * inversion), the quantum Fourier transform (Appendix A) and Born-rule
 * measurement (sec. 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Qubit t (0 <= t < n) is bit t of the basis index, counted from the
 *    least significant bit.  The paper labels qubits i_s = 1 .. n_q from the
 *    most significant bit, with stride 2^{n_q - i_s}; so t = n_q - i_s.
 *  - A state buffer holds 2^n amplitudes, interleaved (re, im):
 *    QC_C128 = two doubles (16 bytes) per amplitude, QC_C64 = two floats
 *    (8 bytes).  The buffer is device memory, 256-byte aligned.
 *  - A 2x2 operator is 8 host doubles, row-major, (re, im) interleaved:
 *    U00 U01 U10 U11 with U_ab = <a|U|b>; rows are output amplitudes
 *    (Eq. resmat1).  For QC_C64 the matrix is rounded to float once.
 *  - All gate calls are asynchronous and ordered on the state's stream
 *    (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *    Calls that return a host value synchronise that stream.
 *  - Arguments are validated before anything is launched; invalid ones
 *    return QC_EINVAL and leave the state unchanged.  A CUDA launch or
 *    runtime failure returns QC_ECUDA.  qc_last_error() returns a message
 *    describing the last failure on the calling host thread.
 *  - Device code never traps: a bounded wait that gives up reports
 *    QC_ETIMEOUT through a status word the host reads.
 */
#ifndef QC_H
#define QC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QC_OK = 0,
  QC_EINVAL = 1,   /* bad argument; nothing was launched */
  QC_ENOMEM = 2,   /* a device allocation failed */
  QC_ECUDA = 3,    /* a CUDA call or kernel launch failed */
  QC_ETIMEOUT = 4  /* a device-side bounded wait gave up */
} qc_status;

typedef enum { QC_C128 = 0, QC_C64 = 1 } qc_dtype;

#define QC_MAX_QUBITS 34      /* largest n accepted for a single state */
#define QC_MAX_MARKED 1024    /* largest number of Grover marked items per call */

/* Opaque state handle: a device buffer (owned or borrowed), its size, dtype,
 * stream and a small device scratch area for reductions. */
typedef struct qc_state qc_state;

/* Message for the last failure on this host thread ("" if none).  The
 * pointer stays valid until the next qc_* call on this thread. */
const char* qc_last_error(void);

/* Library version string. */
const char* qc_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * threads, all devices) -- a diagnostic for launch accounting.  A CUDA graph
 * replay counts the kernels it contains. */
unsigned long long qc_kernel_launches(void);

/* ---------------------------------------------------------------- state -- */

/* Allocate a 2^n state on the current device and set it to |0..0> (C_0 = 1,
 * all other amplitudes 0: the starting state of sec. 5.1).  The handle owns
 * the buffer; qc_state_free releases it.  1 <= n <= QC_MAX_QUBITS.
 * Returns QC_ENOMEM if the buffer does not fit. */
qc_status qc_state_alloc(int n, qc_dtype dt, void* stream, qc_state** out);

/* Wrap an existing device buffer of 2^n amplitudes (e.g. a torch tensor's
 * storage) without copying or initialising it.  The buffer must stay alive
 * and 16-byte aligned (256-byte alignment recommended) for the handle's
 * lifetime; qc_state_free does not release it. */
qc_status qc_state_wrap(void* dev_ptr, int n, qc_dtype dt, void* stream, qc_state** out);

/* Release the handle (and the buffer if it owns it).  NULL is accepted. */
qc_status qc_state_free(qc_state* s);

/* Set the state to the computational basis state |basis_index>. */
qc_status qc_state_reset(qc_state* s, uint64_t basis_index);

/* Set every amplitude to 2^{-n/2} (= HALL|0..0>, Eq. HALL applied to the
 * start state), without touching the previous contents. */
qc_status qc_state_uniform(qc_state* s);

/* Device pointer, qubit count, dtype of the handle. */
qc_status qc_state_info(const qc_state* s, void** dev_ptr, int* n, qc_dtype* dt);

/* Change the stream later calls on this handle are ordered on. */
qc_status qc_state_set_stream(qc_state* s, void* stream);

/* Tell the handle its buffer was written outside this library (drops cached
 * reductions such as the running amplitude sum used by qc_grover_step). */
qc_status qc_state_invalidate(qc_state* s);

/* ---------------------------------------------------------------- gates -- */

/* One-qubit operator on qubit t: OneOpA, Eq. resmat1.  For each of the
 * 2^{n-1} pairs n0 (bit t = 0), n1 = n0 + 2^t:
 *   C~_{n0} = U00 C_{n0} + U01 C_{n1},  C~_{n1} = U10 C_{n0} + U11 C_{n1}.
 * Structured U (diagonal, anti-diagonal, real, Hadamard, phase-only) run
 * specialised kernels with the same result up to rounding. */
qc_status qc_apply_1q(qc_state* s, int t, const double U[8]);

/* Controlled U: the 4x4 operator diag(I, U) of Eq. resmat2 with qubit c as
 * control and t as target -- U acts on the t-pair only where bit c = 1.
 * c != t. */
qc_status qc_apply_ctrl(qc_state* s, int c, int t, const double U[8]);

/* CNOT (sec. 4.2): flips bit t where bit c = 1.  A pure permutation: the
 * result is bit-exact.  c != t. */
qc_status qc_cnot(qc_state* s, int c, int t);

/* CPHASEK (Eq. cphasek): multiplies the amplitudes whose bits c and t are
 * both 1 by e^{2 pi i / 2^k}, k >= 1 (k = 1 is CPHASEA = diag(1,1,1,-1);
 * k = 1 and 2 are exact sign / i rotations).  Symmetric in c, t; c != t. */
qc_status qc_cphase(qc_state* s, int c, int t, int k);

/* SWAP of qubits a and b (Appendix A): exchanges bits a and b of every basis
 * index.  A permutation: bit-exact.  a != b. */
qc_status qc_swap(qc_state* s, int a, int b);

/* HALL (Eq. HALL): the Hadamard on every qubit, as fused shared-memory tile
 * passes (several qubits per pass over the state). */
qc_status qc_hall(qc_state* s);

/* A layer of one-qubit operators: U[8*q .. 8*q+7] on qubit q for every q
 * whose bit is set in qubit_mask (operators on distinct qubits commute; the
 * result equals applying them one by one).  U is a host array of 8*n
 * doubles.  Runs as fused shared-memory tile passes. */
qc_status qc_apply_1q_layer(qc_state* s, const double* U, uint64_t qubit_mask);

/* Grover operator G = HALL . Inv . HALL . Oracle (sec. 5.1) on the current
 * state: the oracle negates each marked amplitude (Eq. oracle1), and
 * HALL . Inv . HALL = 2|s><s| - I (Eq. inversion) maps C_i -> 2 m - C_i with
 * m the mean amplitude after the oracle.  `marked` is a host array of
 * n_marked (1 .. QC_MAX_MARKED) distinct indices < 2^n.  One fused
 * read+write pass; the running amplitude sum is kept on the device between
 * calls (recomputed after any other mutation). */
qc_status qc_grover_step(qc_state* s, const uint64_t* marked, int n_marked);

/* Grover search of sec. 5.1: prepare HALL|0..0>, then apply G `iters`
 * times.  For small states (<= 8192 amplitudes for QC_C128, 16384 for
 * QC_C64) the whole run is one kernel with the state in shared memory. */
qc_status qc_grover_run(qc_state* s, const uint64_t* marked, int n_marked, int iters);

/* Grover step of a state split over several devices (sec. 5.1's G; the
 * split is the paper's distribution of amplitudes over processes, sec.
 * 3.1-3.3, with the high index bits choosing the device).  `s` is one
 * shard; `marked` (host, n_marked = 0 .. QC_MAX_MARKED distinct indices <
 * 2^n of the shard) are the marked items that fall in it, in shard-local
 * indices.  qc_grover_partial writes out[2] = S_r - 2 sum_{marked} C (S_r
 * the shard's amplitude sum; synchronises the shard's stream) and saves the
 * marked amplitudes; the caller adds the shards' values (one complex
 * all-reduce) into P and calls qc_grover_apply_mean with the same marked
 * list and mean[2] = P / 2^{n_total}, which applies C -> 2m - C (unmarked),
 * 2m + C (marked) in one read+write pass.  The diffusion 2|s><s| - I does
 * not depend on how qubits are ordered over the shards.  QC_EINVAL if the
 * apply call does not follow a partial call with the same list, with no
 * other mutation between them. */
qc_status qc_grover_partial(qc_state* s, const uint64_t* marked, int n_marked, double out[2]);
qc_status qc_grover_apply_mean(qc_state* s, const uint64_t* marked, int n_marked, const double mean[2]);

/* Quantum Fourier transform (Appendix A): the Hadamard / CPHASEK ladder
 * followed by the qubit-order reversal swaps, i.e.
 *   C~_{n'} = 2^{-n/2} sum_n e^{+2 pi i n n' / 2^n} C_n.
 * Runs as fused tile passes plus one in-place bit-reversal pass.  For
 * complex128 the buffer holds an internal double-float form between those
 * passes, so a CUDA failure in the middle (QC_ECUDA) leaves the state's
 * contents undefined. */
qc_status qc_qft(qc_state* s);

/* General two-qubit operator, TwoOpA (Eq. resmat2, Eq. twoopB): for every
 * quartet n00 (bits t1 and t2 zero), n01 = n00 + 2^t2, n10 = n00 + 2^t1,
 * n11 = n00 + 2^t1 + 2^t2, the four amplitudes in the order
 * (n00, n01, n10, n11) are multiplied by V: 32 host doubles, 4x4 row-major,
 * (re, im) interleaved, V_{ij;kl} = <i j|V|k l> at row 2i+j, column 2k+l, i
 * the value of qubit t1 and j of qubit t2.  t1 != t2; n >= 2.  complex128
 * runs in double-float arithmetic. */
qc_status qc_apply_2q(qc_state* s, int t1, int t2, const double V[32]);

/* Dense k-qubit block: OneOpA / TwoOpA (Eqs. resmat1, resmat2) extended to
 * a 2^k x 2^k operator U on k distinct qubits, 1 <= k <= 6.  Local index l
 * has bit b on qubit qubits[b] (host array); for every assignment g of the
 * other qubits, C[g|offs(l)] <- sum_l' U[l][l'] C[g|offs(l')].  U: host,
 * 2 * 4^k doubles, row-major, (re, im) interleaved.  k = 2 with qubits
 * {t2, t1} is qc_apply_2q(t1, t2).  complex64 with k = 5 runs on the
 * tensor cores: each group of 32 amplitudes and the operator are cut into
 * bf16 fixed-point digits from their largest magnitude (rows whose largest
 * magnitude is below 2^-120 keep 8 significant bits), the leading digit
 * products accumulate exactly in FP32, and the result is rounded once
 * (FP32-class accuracy, no bias); the call synchronises the stream to read
 * a status word and returns QC_ETIMEOUT if a device wait gave up.  Other
 * cases run on CUDA cores (complex128 in double-float). */
qc_status qc_apply_dense(qc_state* s, int k, const int* qubits, const double* U);

/* Self-test of the tensor-core block's timeout path (no paper counterpart).
 * Launches qc_apply_dense's tensor-core kernel on qubits 0..4 of a complex64
 * state (n >= 5) with its MMA issue switched off and each mbarrier wait
 * bounded by spin_limit polls (1 .. 2^20), so the first wait runs out while
 * nothing asynchronous is in flight: the kernel records the timeout in its
 * status word, releases its tensor memory and returns.  The state is not
 * modified.  Returns QC_ETIMEOUT when the path works (anything else is a
 * failure of the path); QC_EINVAL for a bad state or limit. */
qc_status qc_dense_timeout_selftest(qc_state* s, uint32_t spin_limit);

/* ------------------------------------------------------- gate fusion -- */
/* A circuit operator for gate fusion: kind QC_OP_1Q applies m (a U(2),
 * row-major (re, im)) to q0; QC_OP_CNOT flips q1 where q0 is 1; QC_OP_CPHASE
 * multiplies the amplitudes with q0 = q1 = 1 by e^{2 pi i / 2^k}; QC_OP_SWAP
 * exchanges q0 and q1; QC_OP_CTRL applies m to q1 where q0 is 1. */
#define QC_OP_1Q 1
#define QC_OP_CNOT 2
#define QC_OP_CPHASE 3
#define QC_OP_SWAP 4
#define QC_OP_CTRL 5
typedef struct {
  int32_t kind;
  int32_t q0, q1;
  int32_t k;
  double m[8];
} qc_op;

typedef struct qc_fused_plan qc_fused_plan;

/* Groups a circuit of n_ops operators (host array, applied in order) on n
 * qubits into dense blocks of at most kmax (2..6) qubits: the fused
 * multi-gate pass of sec. 3 (independent pair updates) generalised to
 * two-qubit operators.  A block takes every later operator whose qubits fit
 * and that no left-out operator precedes on a shared qubit, so the blocks
 * compose to the circuit exactly.  pad != 0 pads blocks to kmax qubits
 * (complex64 5-qubit blocks run on the tensor cores).  The block operators
 * are composed on the host in FP64. */
qc_status qc_fused_plan_create(int n, const qc_op* ops, int n_ops, int kmax, int pad, qc_fused_plan** out);

/* Number of blocks and the block size limit. */
qc_status qc_fused_plan_info(const qc_fused_plan* p, int* n_blocks, int* kmax);

/* Block i of the plan: its qubit count *k, its qubits (local bit b on
 * qubits[b]; up to 6 ints) and, if U is not NULL, its operator (2 * 4^k
 * doubles, row-major, (re, im)).  Host data only. */
qc_status qc_fused_plan_block(const qc_fused_plan* p, int i, int* k, int* qubits, double* U);

/* Applies the blocks to s (one pass each, qc_apply_dense's kernels).  The
 * packed operators are uploaded on the first run for each dtype (a
 * synchronous copy); a run with tensor-core blocks synchronises the stream
 * once to read its status word (QC_ETIMEOUT if a device wait gave up). */
qc_status qc_fused_plan_run(qc_state* s, qc_fused_plan* p);

qc_status qc_fused_plan_free(qc_fused_plan* p);

/* One term of a Hamiltonian: a one- (k = 1) or two-body (k = 2) operator h
 * on qubits[0..k-1] (local bit b on qubits[b], as for qc_apply_dense),
 * row-major 2^k x 2^k, (re, im) interleaved (the first 2 * 4^k doubles of
 * h are used). */
typedef struct {
  int32_t k;
  int32_t qubits[2];
  double h[32];
} qc_hterm;

/* One first-order step of Hamiltonian evolution (sec. 7, hbar = 1):
 *   psi <- [1 - i dt (H1 + H2)] psi,  H = sum of the n_terms terms,
 * each term acting on the state as it was before the step (a temporary
 * device snapshot of 2^n amplitudes).  h is expected Hermitian; the step is
 * computed as written for any h.  One accumulating pass per term. */
qc_status qc_hamiltonian_step(qc_state* s, double dt, const qc_hterm* terms, int n_terms);

/* Shor's state of Eq. Shor2 (sec. 5.2): with register 1 the high
 * n1 = n - n2 qubits and register 2 the low n2 qubits,
 *   psi = 2^{-n1/2} sum_{j < 2^n1} |j>_1 |x^j mod M>_2,
 * written directly (the paper's modular exponentiation "tacked on" to the
 * register).  Requires 2 <= M < 2^32, M <= 2^n2, 1 <= x < M. */
qc_status qc_shor_prepare(qc_state* s, int n2, uint64_t x, uint64_t M);

/* Projective measurement of the register of qubits [lo, lo+width) with
 * outcome `value` (ProjA, Eq. projreg2, Born rule): *prob_out (host, may be
 * NULL) receives the outcome's probability sum |C|^2 over the matching
 * amplitudes (FP64), the other amplitudes are set to zero and the matching
 * ones divided by sqrt(prob).  QC_EINVAL if the probability is zero.
 * Synchronises the stream. */
qc_status qc_project(qc_state* s, int lo, int width, uint64_t value, double* prob_out);

/* QFT of the register of qubits [lo, lo+width) (Appendix A's circuit
 * applied to register 1 of Shor's algorithm, sec. 5.2 step 5): Hadamard /
 * CPHASEK ladder and the swaps restoring the register's bit order, as gate
 * passes.  On the whole state (lo = 0, width = n) it equals qc_qft. */
qc_status qc_qft_range(qc_state* s, int lo, int width);

/* ----------------------------------------------------------- reductions -- */

/* sum_i |C_i|^2 (the normalisation of sec. 2): FP64 for complex128; for
 * complex64 the exact float squares are summed as float pairs over runs of
 * 32 amplitudes and the runs in FP64.  Synchronises the stream; *out_host
 * receives the value. */
qc_status qc_norm(const qc_state* s, double* out_host);

/* Born-rule probabilities p_i = |C_i|^2 in FP64 (re*re + im*im, rounded
 * separately), written to out_dev (2^n doubles of device memory). */
qc_status qc_probs(const qc_state* s, double* out_dev);

/* <psi|P|psi> for the Pauli string P = i^{|x&z|} X^x Z^z (X on bits of
 * xmask only, Z on zmask only, Y where both are set).  P is Hermitian and
 * the amplitude pairs (j, j^x) are combined, so the value is exactly real:
 * out_host[0..1] = (value, 0).  FP64 accumulation (complex64: exact float
 * products in float-pair runs, the runs in FP64).  Synchronises the
 * stream. */
qc_status qc_expect_pauli(const qc_state* s, uint64_t xmask, uint64_t zmask, double out_host[2]);

/* Scale the state by 1/sqrt(sum |C|^2) (FP64 norm).  *norm_out_host (if not
 * NULL) receives the norm before scaling.  Synchronises the stream. */
qc_status qc_renormalize(qc_state* s, double* norm_out_host);

/* Seeded Born-rule measurement, `shots` outcomes written to out_dev
 * (uint64 device array).  Definition (identical on every device):
 *   w_i = trunc(p_i * 2^62) (p_i as in qc_probs), W_i = w_0 + .. + w_i
 *   (exact 64-bit integers), total = W_{N-1}; shot s draws Philox4x32-10
 *   (Salmon et al., SC'11) with counter (s_lo, s_hi, 0, 0) and key
 *   (seed_lo, seed_hi), r = x0 * 2^32 + x1, target = floor(r * total / 2^64),
 *   outcome = smallest i with W_i > target.
 * Requires every p_i in [0, 2] and 0 < total <= 2^63 (so sum p_i <= 2;
 * QC_EINVAL otherwise) and shots >= 0.  With shots <= 2^n / 2048 each shot
 * rescans the one block of 2048 amplitudes that holds its target, and the
 * temporary device buffer is 8 * (2^n / 2048 + 2) bytes (plus 8 bytes per
 * 4096 blocks for n >= 24, whose block sums are scanned in chunks); with
 * more shots the full W is written as well, 8 * 2^n bytes more (QC_ENOMEM
 * if it does not fit).  Both give the outcomes above.  Synchronises the stream
 * once (to read the total back). */
qc_status qc_sample(const qc_state* s, uint64_t seed, int64_t shots, uint64_t* out_dev);

/* Born-rule probabilities and seeded measurement together (sec. 5.2: the
 * probability of each outcome, then ProjA/Randx draws): probs_dev receives
 * exactly what qc_probs writes and out_dev exactly the outcomes of
 * qc_sample(s, seed, shots, out_dev), but the state is read once for both --
 * the pass that writes p_i also forms the sampler's block weight sums.
 * probs_dev: 2^n doubles of device memory; out_dev: `shots` uint64 of device
 * memory (may be NULL when shots = 0, which only writes the probabilities).
 * Same requirements, temporary buffer and stream synchronisation as
 * qc_sample; on QC_EINVAL from the probability check the probabilities have
 * been written and no outcome has. */
qc_status qc_probs_sample(const qc_state* s, double* probs_dev, uint64_t seed, int64_t shots, uint64_t* out_dev);

/* Seeded measurement for callers that cannot allocate device memory.  The
 * paper has no counterpart; this entry point exists for library users.
 *
 * Who needs it: a host framework that has already claimed the device memory
 * for its own pool (a cudaMalloc here would fail or force it to give memory
 * back), and code on a latency-critical path that cannot take the
 * device-wide synchronisation that cudaMalloc / cudaFree imply.  qc_sample
 * allocates its 8 * 2^n-byte CDF per call and needs a qc_state handle, whose
 * creation allocates scratch too; this variant takes the raw state pointer
 * and calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Result: the same outcomes as qc_sample for the same state, seed and shots
 * (the definition written there), written to out_dev (`shots` uint64 in
 * device memory).  psi_dev holds 2^n amplitudes of dtype dt.
 *
 * Limits and scratch: n must be <= QC_SAMPLE_NOALLOC_MAX_QUBITS (20); larger
 * states return QC_EINVAL with a message.  The scratch is a fixed array of
 * 2^20 + 512 + 32 uint64 (about 8 MiB) in the library's own device memory,
 * held on every GPU that loads the library until the process exits.  The
 * first call on a device looks up that array's device address (once per
 * device, kept for later calls); make that first call before any stream
 * capture begins, and do not call this entry point again on a device after
 * cudaDeviceReset there.  The array keeps the last call's contents (each
 * call resets what must start at zero); calls whose work overlaps on the
 * GPU -- on different streams or threads -- race on it and must be
 * serialised by the caller.
 *
 * Validation: every |C_i|^2 must lie in [0, 2] and
 * 0 < sum_i trunc(p_i 2^62) <= 2^63; otherwise QC_EINVAL.  The check runs on
 * the device, and every call synchronises `stream` once to read its verdict
 * back to the host before it draws the samples. */
#define QC_SAMPLE_NOALLOC_MAX_QUBITS 20
qc_status qc_sample_noalloc(const void* psi_dev, int n, qc_dtype dt, uint64_t seed, int64_t shots,
                            uint64_t* out_dev, void* stream);

/* ---------------------------------------------- batched noisy trajectories
 * Many independent noisy Grover runs ("multiverses", sec. 6.2-6.3) of uneven
 * qubit counts, complex64 with FP64 reductions, in one persistent launch.
 * Noise model: after every gate location a Pauli error may strike: stage 0
 * is the initial HALL (one location per qubit), iteration r has stages
 * 1+4r (after the oracle), 2+4r (after each H of the first HALL), 3+4r
 * (after Inv) and 4+4r (after each H of the second HALL), one location per
 * qubit each.  Location (instance i, stage s, qubit q) draws Philox4x32-10
 * with counter (i, s, q, 0x4E4F4953) and key (seed_lo, seed_hi): an error
 * strikes when x0 < thr_gate, and it is X, Y, Z for floor(x1*3/2^32) = 0, 1,
 * 2.  At the end each instance reports its success probability
 * sum_{marked} |C|^2, the probability that a read-out with independent bit
 * flips (each with probability p_readout) returns the marked item, one
 * seeded measured outcome (counter (i, 0xFFFFFFFF, 0, 0x4D454153), sampled
 * as in qc_sample) with each bit q flipped when the draw (i, 0xFFFFFFFF, q,
 * 0x52454144) has x0 < thr_readout, and the number of Pauli errors. */
typedef struct {
  int32_t n_inst;          /* number of instances, >= 1 */
  const int32_t* nq;       /* host, qubit count per instance, 1 .. QC_TRAJ_MAX_QUBITS */
  const uint64_t* marked;  /* host, marked item per instance (< 2^nq) */
  const int32_t* iters;    /* host, Grover iterations per instance (>= 0) */
  uint64_t seed;
  uint32_t thr_gate;       /* floor(p_gate * 2^32) */
  uint32_t thr_readout;    /* floor(p_readout * 2^32) */
  double p_readout;        /* the read-out flip probability itself */
} qc_traj_desc;

#define QC_TRAJ_MAX_QUBITS 22

typedef struct {
  double* p_success;    /* device, n_inst doubles */
  double* p_readout;    /* device, n_inst doubles */
  uint64_t* outcome;    /* device, n_inst outcomes */
  uint32_t* n_errors;   /* device, n_inst counts */
} qc_traj_out;

typedef struct qc_traj_plan qc_traj_plan;

/* Validate the batch, upload its descriptors, pick the launch shape (CTAs
 * cooperating per instance, shared-memory tile size) with the built-in
 * autotuner and allocate the device workspace.  `autotune` = 0 takes the
 * default shape without timing trial runs. */
qc_status qc_traj_plan_create(const qc_traj_desc* d, void* stream, int autotune, qc_traj_plan** out);

/* Run every instance of the plan: one persistent kernel launch (replayed
 * from a CUDA graph after the first run).  Asynchronous on the plan's
 * stream.  Returns QC_ETIMEOUT (after synchronising) if a device-side
 * bounded wait gave up. */
qc_status qc_traj_plan_run(qc_traj_plan* p, const qc_traj_out* out);

/* qc_traj_plan_run, and also each selected instance's final complex64 state:
 * the 2^nq[i] amplitudes its read-out is drawn from (after its last pass;
 * squared norm Q, the value p_success divides by), written to
 * states_dev + state_off_dev[i] (device array of n_inst amplitude offsets,
 * ~0 = skip the instance; the caller makes the ranges disjoint and large
 * enough).  For replaying an instance's seeded read-out from the very
 * weights the kernel used.  QC_EINVAL if either pointer is NULL. */
qc_status qc_traj_plan_run_states(qc_traj_plan* p, const qc_traj_out* out, const uint64_t* state_off_dev,
                                  void* states_dev);

/* Chosen launch shape: clusters of `ctas_per_inst` CTAs, `threads` threads. */
qc_status qc_traj_plan_info(const qc_traj_plan* p, int* ctas_per_inst, int* threads, int* grid);

qc_status qc_traj_plan_free(qc_traj_plan* p);

/* ----------------------------------------------------- adjoint gradient --
 * Parameterised circuits on a batch of B states (state b at element offset
 * b * 2^n) and the gradient of E = <psi|H|psi> by uncomputation.  Not part
 * of the paper. */
typedef enum {
  QC_G_RX = 0,   /* exp(-i theta X / 2) on q0, theta = theta[param] */
  QC_G_RY = 1,   /* exp(-i theta Y / 2) */
  QC_G_RZ = 2,   /* exp(-i theta Z / 2) */
  QC_G_CNOT = 3, /* control q0, target q1 */
  QC_G_H = 4     /* Hadamard on q0 */
} qc_gate_kind;

typedef struct {
  int32_t kind;   /* qc_gate_kind */
  int32_t q0, q1; /* qubits (q1 only for CNOT) */
  int32_t param;  /* angle index for rotations, else ignored */
} qc_gate;

typedef struct {
  uint64_t xmask, zmask; /* Pauli string as in qc_expect_pauli */
  double coeff;          /* real coefficient */
} qc_pauli_term;

/* psi_b = U_G .. U_1 |0..0> for each batch element b, with angles
 * theta_dev[b * theta_stride + param] (device doubles).  psi_dev holds
 * B * 2^n amplitudes of dtype dt.  Gates are a host array. */
qc_status qc_circuit_forward(int n, qc_dtype dt, int B, const qc_gate* gates, int n_gates,
                             const double* theta_dev, int64_t theta_stride,
                             void* psi_dev, void* stream);

/* Energy E_b = <psi_b|H|psi_b> (device doubles energy_dev[b]) and the
 * gradient dE_b/dtheta (grad_dev[b * theta_stride + param], device doubles;
 * entries of parameters the circuit does not use are set to 0).  Runs the
 * forward pass, then walks the gates backwards applying U^dagger to psi and
 * to lambda = H psi (no intermediate states are stored); for a rotation
 * gate j with Pauli generator P: dE/dtheta_j = Im <lambda_j|P|psi_j>, with
 * FP64 accumulation.  psi_dev and lam_dev are caller-owned workspace of
 * B * 2^n amplitudes each; their contents on return are unspecified.  Two
 * rotations in a row on one qubit run as one pass, and a CNOT ring
 * CNOT(0,1), .., CNOT(n-1,0) as one gather pass (using one more temporary
 * buffer of B * 2^n amplitudes).  H is a host array of Pauli terms with real
 * coefficients. */
qc_status qc_adjoint_grad(int n, qc_dtype dt, int B, const qc_gate* gates, int n_gates,
                          const double* theta_dev, int64_t theta_stride, int n_params,
                          const qc_pauli_term* H, int n_terms,
                          void* psi_dev, void* lam_dev, double* energy_dev, double* grad_dev,
                          void* stream);

/* -------------------------------- noise intrusions and density matrix -- */
/* The paper's noise scenario and ensemble average (sec. 6.1-6.3): a batch of
 * B states ("multiverses", each run with its own unitary intrusions) stored
 * one after another, state a at amplitudes [a 2^n, (a+1) 2^n) of psi_dev
 * (device, dtype dt), with weights P_host[a] >= 0 (host). */
#define QC_DM_MAX_QUBITS 15
#define QC_SPECTRUM_MAX_UNIVERSES 64

/* Wigner rotation D^j(alpha, beta, gamma) for j = twoj/2 in {1/2, 3/2}
 * (the paper's D2 and D4 noise operators; it takes gamma = 0):
 *   D_{m'm} = e^{-i m' alpha} d^j_{m'm}(beta) e^{-i m gamma},
 * rows and columns ordered m = j, j-1, .., -j, written row-major as
 * interleaved (re, im) doubles to D_out (host; 8 doubles for j = 1/2, 32
 * for j = 3/2), ready for qc_apply_1q / qc_apply_2q (m = +1/2 is qubit
 * value 0; the j = 3/2 states m = 3/2 .. -3/2 take the quartet positions
 * 0 .. 3).  Host arithmetic only.  QC_EINVAL for other j or non-finite
 * angles. */
qc_status qc_wigner_d(int twoj, double alpha, double beta, double gamma, double* D_out);

/* The ensemble density matrix (sec. 6.1):
 *   rho[n][n'] = sum_a P_a C_a(n) C_a(n')^*,
 * written row-major to rho_dev (device, 4^n amplitudes of dtype dt, owned by
 * the caller).  1 <= n <= QC_DM_MAX_QUBITS, B >= 1.  complex64 with B <= 64
 * runs on the tensor cores (the real GEMM of 128 x 32 tiles over K = 2B,
 * operands in bf16 digit slices with exact leading sums; FP32-class
 * accuracy) and synchronises the stream to read a status word (QC_ETIMEOUT
 * if a device wait gave up); other cases are stream-ordered on CUDA cores
 * (complex128 inner products in double-float). */
qc_status qc_density_matrix(const void* psi_dev, int n, qc_dtype dt, int B, const double* P_host,
                            void* rho_dev, void* stream);

/* Eigenvalues of the same rho without forming it: its nonzero eigenvalues
 * are those of the B x B Gram matrix G_ab = sqrt(P_a P_b) <psi_a|psi_b>
 * (one streaming pass over the batch), whose eigenvalues one CTA finds in
 * FP64 (Householder reduction to tridiagonal form, then bisection on Sturm
 * counts).  evals_host (B doubles) receives them in descending
 * order (the other 2^n - B eigenvalues of rho are zero); stats_host[0..2] =
 * Tr rho, Tr rho^2 and the entropy -sum l ln l over l > 1e-14 (natural
 * logarithm).  1 <= B <= QC_SPECTRUM_MAX_UNIVERSES, 1 <= n <= 34.
 * Synchronises the stream.  QC_ECUDA if G has a non-finite entry. */
qc_status qc_mixed_spectrum(const void* psi_dev, int n, qc_dtype dt, int B, const double* P_host,
                            double* evals_host, double* stats_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QC_H */
