/*
 * Plain CPU complex128 state-vector oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA library: every routine
 * below restates the definition from the QCMPI paper (Tabakin & Julia-Diaz,
 * arXiv:0902.0699) as a direct loop, in IEEE double precision, compiled with
 * -ffp-contract=off so that every + and * is rounded on its own.
 *
 * Conventions (paper sec. 2, Eq. staten):
 *   the state is psi[2*i] + i*psi[2*i+1] for basis index i = 0 .. 2^n - 1 in
 *   "standard order".  The paper labels qubits from the most significant
 *   (q_1) to the least significant (q_{n_q}); qubit i_s has stride
 *   2^{n_q - i_s} (Eq. pair0/pair1).  This file takes t = n_q - i_s, the
 *   0-based bit position counted from the least significant bit, so the
 *   stride of qubit t is 2^t.
 *
 * A 2x2 operator is passed as 8 doubles: row-major
 *   U00.re U00.im U01.re U01.im U10.re U10.im U11.re U11.im
 * with U_ab = <a|U|b> (Eq. resmat1: rows are the output amplitudes).
 *
 * Parity is pinned in tests/test_oracle_*.py against dense Kronecker-product
 * matrices, closed forms (Grover, QFT basis states), numpy's FFT, the
 * Walsh-Hadamard sign rule and the Random123 known-answer vectors.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } cplx;

static inline cplx cx(double re, double im) { cplx z = {re, im}; return z; }
static inline cplx cadd(cplx a, cplx b) { return cx(a.re + b.re, a.im + b.im); }
static inline cplx cmul(cplx a, cplx b) {
  return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
static inline cplx load(const double* psi, uint64_t i) { return cx(psi[2 * i], psi[2 * i + 1]); }
static inline void store(double* psi, uint64_t i, cplx z) { psi[2 * i] = z.re; psi[2 * i + 1] = z.im; }
static inline cplx mat(const double* U, int r, int c, int dim) {
  return cx(U[2 * (r * dim + c)], U[2 * (r * dim + c) + 1]);
}

/* ---- threading for the timed CPU baseline (results do not depend on it) -- */
void or_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}
int or_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---- one-qubit operator: OneOpA, Eq. resmat1 (sec. 3) -------------------
 * For every n0 whose bit t is 0, its partner is n1 = n0 + 2^t, and
 *   C~_{n0} = O00 C_{n0} + O01 C_{n1},   C~_{n1} = O10 C_{n0} + O11 C_{n1}.
 * The 2^{n-1} pair updates are independent (sec. 3, after Eq. resmat1). */
void or_apply_1q(double* psi, int n, int t, const double* U) {
  const int64_t N = (int64_t)1 << n;
  const int64_t stride = (int64_t)1 << t;
  const cplx u00 = mat(U, 0, 0, 2), u01 = mat(U, 0, 1, 2);
  const cplx u10 = mat(U, 1, 0, 2), u11 = mat(U, 1, 1, 2);
#pragma omp parallel for schedule(static)
  for (int64_t n0 = 0; n0 < N; ++n0) {
    if (n0 & stride) continue; /* n0 must have q_s = 0 (Eq. pair0) */
    const int64_t n1 = n0 + stride; /* Eq. pair1 */
    const cplx c0 = load(psi, n0), c1 = load(psi, n1);
    store(psi, n0, cadd(cmul(u00, c0), cmul(u01, c1)));
    store(psi, n1, cadd(cmul(u10, c0), cmul(u11, c1)));
  }
}

/* ---- general two-qubit operator: TwoOpA, Eqs. twoopB, resmat2 (sec. 4) ---
 * The quartet n00, n01, n10, n11 differs in the bits of qubits s1 (bit t1)
 * and s2 (bit t2); the quartet position is 2*q_{s1} + q_{s2}, so
 * n01 = n00 + 2^{t2}, n10 = n00 + 2^{t1}.  V is 4x4 row-major, 32 doubles,
 * V_{ij;kl} = <i j|V|k l> at row 2i+j, column 2k+l. */
void or_apply_2q(double* psi, int n, int t1, int t2, const double* V) {
  const int64_t N = (int64_t)1 << n;
  const int64_t s1 = (int64_t)1 << t1, s2 = (int64_t)1 << t2;
#pragma omp parallel for schedule(static)
  for (int64_t n00 = 0; n00 < N; ++n00) {
    if ((n00 & s1) || (n00 & s2)) continue;
    const int64_t idx[4] = {n00, n00 + s2, n00 + s1, n00 + s1 + s2};
    cplx in[4], out[4];
    for (int a = 0; a < 4; ++a) in[a] = load(psi, idx[a]);
    for (int r = 0; r < 4; ++r) {
      cplx acc = cmul(mat(V, r, 0, 4), in[0]);
      for (int c = 1; c < 4; ++c) acc = cadd(acc, cmul(mat(V, r, c, 4), in[c]));
      out[r] = acc;
    }
    for (int a = 0; a < 4; ++a) store(psi, idx[a], out[a]);
  }
}

/* ---- controlled-U: the 4x4 operator diag(I, U) of Eq. resmat2 with qubit c
 * as s1 (control) and t as s2.  Quartets with q_c = 0 are untouched; on the
 * q_c = 1 half the t-pair is updated with U exactly as in Eq. resmat1. */
void or_apply_ctrl(double* psi, int n, int c, int t, const double* U) {
  const int64_t N = (int64_t)1 << n;
  const int64_t sc = (int64_t)1 << c, st = (int64_t)1 << t;
  const cplx u00 = mat(U, 0, 0, 2), u01 = mat(U, 0, 1, 2);
  const cplx u10 = mat(U, 1, 0, 2), u11 = mat(U, 1, 1, 2);
#pragma omp parallel for schedule(static)
  for (int64_t n0 = 0; n0 < N; ++n0) {
    if (!(n0 & sc) || (n0 & st)) continue;
    const int64_t n1 = n0 + st;
    const cplx c0 = load(psi, n0), c1 = load(psi, n1);
    store(psi, n0, cadd(cmul(u00, c0), cmul(u01, c1)));
    store(psi, n1, cadd(cmul(u10, c0), cmul(u11, c1)));
  }
}

/* ---- CNOT (sec. 4.2): 00->00, 01->01, 10->11, 11->10 with the first qubit
 * (bit c) as control: the amplitudes with q_c = 1 and q_t = 0 / 1 exchange. */
void or_cnot(double* psi, int n, int c, int t) {
  const int64_t N = (int64_t)1 << n;
  const int64_t sc = (int64_t)1 << c, st = (int64_t)1 << t;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    if (!(i & sc) || (i & st)) continue;
    const cplx a = load(psi, i), b = load(psi, i + st);
    store(psi, i, b);
    store(psi, i + st, a);
  }
}

/* e^{2 pi i / 2^k} (Eq. cphasek).  k = 1 and k = 2 are the exact values -1 and
 * i; otherwise cos/sin of 2 pi / 2^k from libm. */
static cplx cphase_factor(int k) {
  if (k == 1) return cx(-1.0, 0.0);
  if (k == 2) return cx(0.0, 1.0);
  const double ang = 2.0 * 3.14159265358979323846 / ldexp(1.0, k);
  return cx(cos(ang), sin(ang));
}
void or_cphase_factor(int k, double* out) {
  cplx z = cphase_factor(k);
  out[0] = z.re; out[1] = z.im;
}

/* ---- CPHASEK (Eq. cphasek): diag(1, 1, 1, e^{2 pi i / 2^k}); only the
 * amplitudes with both bits set change.  k = 1 is CPHASEA = diag(1,1,1,-1). */
void or_cphase(double* psi, int n, int c, int t, int k) {
  const int64_t N = (int64_t)1 << n;
  const int64_t sc = (int64_t)1 << c, st = (int64_t)1 << t;
  const cplx ph = cphase_factor(k);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    if ((i & sc) && (i & st)) store(psi, i, cmul(ph, load(psi, i)));
  }
}

/* ---- SWAP of two qubits (App. A): the basis index has bits a and b
 * exchanged; amplitudes with differing bits trade places. */
void or_swap(double* psi, int n, int a, int b) {
  const int64_t N = (int64_t)1 << n;
  const int64_t sa = (int64_t)1 << a, sb = (int64_t)1 << b;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    if ((i & sa) && !(i & sb)) {
      const int64_t j = i - sa + sb;
      const cplx x = load(psi, i), y = load(psi, j);
      store(psi, i, y);
      store(psi, j, x);
    }
  }
}

/* Hadamard (Eq. NOTH): (sigma_x + sigma_z)/sqrt(2). */
static void hadamard_matrix(double* U) {
  const double s = 1.0 / sqrt(2.0);
  const double h[8] = {s, 0, s, 0, s, 0, -s, 0};
  memcpy(U, h, sizeof h);
}

/* ---- HALL (Eq. HALL): the one-qubit Hadamard on every qubit, applied as
 * n_q separate OneOpA calls, exactly as the paper's subroutine HALL does. */
void or_hall(double* psi, int n) {
  double H[8];
  hadamard_matrix(H);
  for (int t = 0; t < n; ++t) or_apply_1q(psi, n, t, H);
}

/* ---- HALL2 (sec. 4.3): dense Walsh-Hadamard with signs
 * s_{n,n'} = (-1)^{#bits set in both n and n'}, normalised by 2^{-n_q/2}.
 * O(4^n); only for small n.  Writes out-of-place. */
void or_hall2(const double* psi, double* out, int n) {
  const int64_t N = (int64_t)1 << n;
  const double norm = 1.0 / sqrt(ldexp(1.0, n));
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < N; ++r) {
    cplx acc = cx(0.0, 0.0);
    for (int64_t c = 0; c < N; ++c) {
      const int odd = __builtin_popcountll((unsigned long long)(r & c)) & 1;
      const cplx v = load(psi, c);
      acc = odd ? cx(acc.re - v.re, acc.im - v.im) : cadd(acc, v);
    }
    store(out, r, cx(acc.re * norm, acc.im * norm));
  }
}

/* ---- Grover oracle (Eq. oracle1): C(n_x) -> -C(n_x) for each marked item. */
void or_oracle(double* psi, int n, const uint64_t* marked, int n_marked) {
  (void)n;
  for (int m = 0; m < n_marked; ++m) {
    const uint64_t i = marked[m];
    psi[2 * i] = -psi[2 * i];
    psi[2 * i + 1] = -psi[2 * i + 1];
  }
}

/* ---- Inv = 2|0..0><0..0| - I (Eq. inversion): every amplitude except n = 0
 * changes sign. */
void or_inv(double* psi, int n) {
  const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 1; i < N; ++i) {
    psi[2 * i] = -psi[2 * i];
    psi[2 * i + 1] = -psi[2 * i + 1];
  }
}

/* ---- Grover operator G = HALL . Inv . HALL . Oracle (sec. 5.1), applied
 * literally from right to left. */
void or_grover_step(double* psi, int n, const uint64_t* marked, int n_marked) {
  or_oracle(psi, n, marked, n_marked);
  or_hall(psi, n);
  or_inv(psi, n);
  or_hall(psi, n);
}

/* ---- QFT circuit of Appendix A, in the paper's own qubit labels
 * (i_s = 1 is the most significant qubit, bit t = n - i_s):
 *   for ic = 1 .. n-1:  Hadamard on qubit ic, then for k = ic+1 .. n the
 *   CPHASEK between qubits k and ic with phase index k+1-ic;
 *   a final Hadamard on qubit n; then SWAP(i, n+1-i) for i = 1 .. n/2.
 * CPHASEK is symmetric in its two qubits. */
void or_qft(double* psi, int n) {
  double H[8];
  hadamard_matrix(H);
  for (int ic = 1; ic <= n - 1; ++ic) {
    or_apply_1q(psi, n, n - ic, H);
    for (int k = ic + 1; k <= n; ++k) or_cphase(psi, n, n - k, n - ic, k + 1 - ic);
  }
  or_apply_1q(psi, n, 0, H);
  for (int i = 1; i <= n / 2; ++i) or_swap(psi, n, n - i, i - 1);
}

/* ---- Born-rule probabilities and the norm (sec. 2: |C_0|^2 + |C_1|^2 = 1).
 * p_i = re*re + im*im, each product and the sum rounded separately. */
void or_probs(const double* psi, int n, double* p) {
  const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    const double re = psi[2 * i], im = psi[2 * i + 1];
    const double a = re * re;
    const double b = im * im;
    p[i] = a + b;
  }
}
/* serial, index order */
double or_norm(const double* psi, int n) {
  const int64_t N = (int64_t)1 << n;
  double s = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    const double re = psi[2 * i], im = psi[2 * i + 1];
    s += re * re + im * im;
  }
  return s;
}

/* <psi|P|psi> for the Pauli string P = i^{|x&z|} X^x Z^z, i.e. X on the bits
 * of xmask only, Z on zmask only, Y where both are set.  (P psi)[j ^ x] =
 * i^{|x&z|} (-1)^{|j & z|} psi[j].  Serial sum in index order; out = re, im. */
void or_expect_pauli(const double* psi, int n, uint64_t xmask, uint64_t zmask, double* out) {
  const int64_t N = (int64_t)1 << n;
  const int ny = __builtin_popcountll((unsigned long long)(xmask & zmask)) & 3;
  static const cplx ipow[4] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
  cplx acc = cx(0, 0);
  for (int64_t j = 0; j < N; ++j) {
    const int sgn = __builtin_popcountll((unsigned long long)(j & zmask)) & 1;
    cplx v = load(psi, j);
    if (sgn) v = cx(-v.re, -v.im);
    v = cmul(ipow[ny], v);
    const cplx w = load(psi, (int64_t)((uint64_t)j ^ xmask));
    /* conj(w) * v */
    acc = cadd(acc, cx(w.re * v.re + w.im * v.im, w.re * v.im - w.im * v.re));
  }
  out[0] = acc.re;
  out[1] = acc.im;
}

/* out = P psi for the Pauli string above (out-of-place). */
void or_apply_pauli(const double* psi, double* out, int n, uint64_t xmask, uint64_t zmask) {
  const int64_t N = (int64_t)1 << n;
  const int ny = __builtin_popcountll((unsigned long long)(xmask & zmask)) & 3;
  static const cplx ipow[4] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
  for (int64_t j = 0; j < N; ++j) {
    const int sgn = __builtin_popcountll((unsigned long long)(j & zmask)) & 1;
    cplx v = load(psi, j);
    if (sgn) v = cx(-v.re, -v.im);
    store(out, (int64_t)((uint64_t)j ^ xmask), cmul(ipow[ny], v));
  }
}

/* ---- Philox4x32-10 counter-based generator, from Salmon, Moraes, Dror and
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11: ten rounds of
 *   (L0,R0,L1,R1) -> (hi(M1*R1) ^ L0 ^ k0, lo(M1*R1), hi(M0*R0) ^ L1 ^ k1, lo(M0*R0))
 * written on the 4-word counter (c0,c1,c2,c3) = (R0,L0,R1,L1), with the key
 * advanced by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    const uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ---- Seeded measurement (Born rule, sec. 2; ProjA/Randx are named by the
 * paper without a definition).  Our definition, the same on every device:
 *   w_i = trunc(p_i * 2^62) as an unsigned 64-bit integer (p_i <= 2),
 *   W_i = w_0 + ... + w_i exactly (integer prefix sum), total = W_{N-1};
 *   shot s draws Philox4x32-10 with counter (s_lo, s_hi, 0, 0) and key
 *   (seed_lo, seed_hi); r = x0 * 2^32 + x1; target = floor(r * total / 2^64);
 *   the outcome is the smallest i with W_i > target.
 * Writes the integer cdf (N entries) and the outcomes (shots entries).
 * Returns 0, or 1 if the probabilities are unusable (a p_i outside [0, 2] or
 * a zero total). */
int or_sample_from_probs(const double* p, int n, uint64_t seed, int64_t shots,
                         uint64_t* cdf, uint64_t* outcomes) {
  const int64_t N = (int64_t)1 << n;
  uint64_t run = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (!(p[i] >= 0.0 && p[i] <= 2.0)) return 1;
    const double scaled = p[i] * 4611686018427387904.0; /* 2^62, exact */
    const uint64_t w = (uint64_t)scaled;                 /* truncation */
    run += w;
    cdf[i] = run;
  }
  const uint64_t total = run;
  if (total == 0) return 1;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t s = 0; s < shots; ++s) {
    const uint32_t ctr[4] = {(uint32_t)(uint64_t)s, (uint32_t)((uint64_t)s >> 32), 0u, 0u};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    const uint64_t r = ((uint64_t)x[0] << 32) | x[1];
    const uint64_t target = (uint64_t)(((unsigned __int128)r * total) >> 64);
    /* smallest i with cdf[i] > target: linear scan, the plain definition */
    int64_t i = 0;
    while (cdf[i] <= target) ++i;
    outcomes[s] = (uint64_t)i;
  }
  return 0;
}

/* ---- Shor's state, Eq. Shor2 (sec. 5.2): register 1 = the high n1 = n - n2
 * bits, register 2 = the low n2 bits; psi = 2^{-n1/2} sum_j |j>|x^j mod M>,
 * with x^j mod M built by repeated multiplication, f(j+1) = f(j) x mod M. */
void or_shor_prepare(double* psi, int n, int n2, uint64_t x, uint64_t M) {
  const int n1 = n - n2;
  const int64_t N = (int64_t)1 << n;
  memset(psi, 0, sizeof(double) * 2 * (size_t)N);
  const double a = 1.0 / sqrt(ldexp(1.0, n1));
  uint64_t f = 1 % M;
  for (int64_t j = 0; j < ((int64_t)1 << n1); ++j) {
    psi[2 * ((j << n2) | (int64_t)f)] = a;
    f = (f * x) % M;
  }
}

/* ---- ProjA (Eq. projreg2): keep the amplitudes whose bits [lo, lo+w)
 * equal `value`, renormalise (Born rule); returns the outcome probability. */
double or_project(double* psi, int n, int lo, int w, uint64_t value) {
  const int64_t N = (int64_t)1 << n;
  const uint64_t mask = ((uint64_t)1 << w) - 1;
  double p = 0.0;
  for (int64_t i = 0; i < N; ++i)
    if ((((uint64_t)i >> lo) & mask) == value) p += psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
  const double f = p > 0.0 ? 1.0 / sqrt(p) : 0.0;
  for (int64_t i = 0; i < N; ++i) {
    if ((((uint64_t)i >> lo) & mask) == value) {
      psi[2 * i] *= f;
      psi[2 * i + 1] *= f;
    } else {
      psi[2 * i] = 0.0;
      psi[2 * i + 1] = 0.0;
    }
  }
  return p;
}

/* ---- The Appendix A loop on the register of qubits [lo, lo+w): the
 * register's paper label ic = 1 .. w is bit t = lo + w - ic. */
void or_qft_range(double* psi, int n, int lo, int w) {
  double H[8];
  hadamard_matrix(H);
  for (int ic = 1; ic <= w - 1; ++ic) {
    or_apply_1q(psi, n, lo + w - ic, H);
    for (int k = ic + 1; k <= w; ++k) or_cphase(psi, n, lo + w - k, lo + w - ic, k + 1 - ic);
  }
  or_apply_1q(psi, n, lo, H);
  for (int i = 1; i <= w / 2; ++i) or_swap(psi, n, lo + w - i, lo + i - 1);
}
