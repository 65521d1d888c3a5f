"""CPU oracle for the state-vector gate engine -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.  The gate
routines live in plain C (qc_oracle.c, complex128, every operation rounded on
its own); this module loads them with ctypes and composes them into the
paper's algorithms exactly in the paper's order:

* Grover (sec. 5.1): G = HALL . Inv . HALL . Oracle, starting from HALL|0..0>.
* QFT (Appendix A): the Hadamard / CPHASEK ladder followed by the pair swaps.
* measurement: Born rule (sec. 2) with the seeded integer-CDF sampler.
* noisy trajectories (sec. 6.3 "multiverse" noise, read as per-gate Pauli
  noise): the literal gate sequence with a Pauli inserted after each gate
  whose Philox draw fires.
* adjoint gradient of <psi|H|psi> for the layered RY/RZ + CNOT-ring ansatz
  (not in the paper): forward, then uncompute with U^dagger while carrying
  lambda = H psi; dE/dtheta_j = Im <lambda_j| P_j |psi_j>.

Conventions: qubit t is bit t of the basis index (t = n_q - i_s in the
paper's labels, where i_s = 1 is the most significant qubit).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        sig = {
            "or_set_threads": (None, [ctypes.c_int]),
            "or_get_threads": (ctypes.c_int, []),
            "or_apply_1q": (None, [_dp, ctypes.c_int, ctypes.c_int, _dp]),
            "or_apply_2q": (None, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]),
            "or_apply_ctrl": (None, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]),
            "or_cnot": (None, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "or_cphase": (None, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "or_cphase_factor": (None, [ctypes.c_int, _dp]),
            "or_swap": (None, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "or_hall": (None, [_dp, ctypes.c_int]),
            "or_hall2": (None, [_dp, _dp, ctypes.c_int]),
            "or_oracle": (None, [_dp, ctypes.c_int, _u64p, ctypes.c_int]),
            "or_inv": (None, [_dp, ctypes.c_int]),
            "or_grover_step": (None, [_dp, ctypes.c_int, _u64p, ctypes.c_int]),
            "or_qft": (None, [_dp, ctypes.c_int]),
            "or_probs": (None, [_dp, ctypes.c_int, _dp]),
            "or_norm": (ctypes.c_double, [_dp, ctypes.c_int]),
            "or_expect_pauli": (None, [_dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _dp]),
            "or_apply_pauli": (None, [_dp, _dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]),
            "or_philox4x32_10": (None, [_u32p, _u32p, _u32p]),
            "or_sample_from_probs": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_uint64,
                                                    ctypes.c_int64, _u64p, _u64p]),
            "or_shor_prepare": (None, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]),
            "or_project": (ctypes.c_double, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]),
            "or_qft_range": (None, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _state_ptr(psi: np.ndarray):
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    return psi.ctypes.data_as(_dp)


def _mat(U) -> np.ndarray:
    """2x2 complex matrix or 8 interleaved doubles -> 8 doubles."""
    U = np.asarray(U)
    if U.dtype.kind == "c":
        U = np.stack([U.real, U.imag], axis=-1)
    return np.ascontiguousarray(U, dtype=np.float64).reshape(-1)


def set_threads(k: int) -> None:
    lib().or_set_threads(int(k))


def get_threads() -> int:
    return int(lib().or_get_threads())


# ------------------------------------------------------------ basic gates ----

def zero_state(n: int, basis: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[basis] = 1.0
    return psi


def apply_1q(psi, n, t, U):
    lib().or_apply_1q(_state_ptr(psi), n, t, _d(_mat(U)))
    return psi


def apply_2q(psi, n, t1, t2, V):
    lib().or_apply_2q(_state_ptr(psi), n, t1, t2, _d(_mat(V)))
    return psi


def dense_offsets(qubits) -> np.ndarray:
    """offs[l] = sum_b bit b of l placed at qubit qubits[b] (qubits[0] is
    the least significant bit of the local index l)."""
    k = len(qubits)
    offs = np.zeros(1 << k, dtype=np.int64)
    for l in range(1 << k):
        for b, q in enumerate(qubits):
            if (l >> b) & 1:
                offs[l] |= 1 << q
    return offs


def apply_dense(psi, n, qubits, U):
    """A dense 2^k x 2^k operator on k qubits (the paper's OneOpA and TwoOpA,
    sec. 3-4, extended to k qubits): for every assignment g of the other
    n - k qubits, the 2^k amplitudes C[g | offs[l]] are replaced by
    sum_l' U[l][l'] C[g | offs[l']]."""
    U = np.asarray(U, dtype=complex)
    offs = dense_offsets(qubits)
    mask = int(offs[-1])
    base = np.array([i for i in range(1 << n) if i & mask == 0], dtype=np.int64)
    idx = base[:, None] + offs[None, :]
    psi[idx] = psi[idx] @ U.T
    return psi


def apply_ops(psi, n, ops):
    """A circuit applied literally, one operator after another (OneOpA,
    CNOT, CPHASEK, SWAP and controlled-U of sec. 3-4 and App. A): ops are
    (kind, q0, q1, k, U) with kind 1 = U on q0, 2 = CNOT(q0 -> q1),
    3 = CPHASEK(q0, q1, k), 4 = SWAP(q0, q1), 5 = U on q1 controlled by q0."""
    for kind, q0, q1, k, U in ops:
        if kind == 1:
            apply_1q(psi, n, q0, U)
        elif kind == 2:
            cnot(psi, n, q0, q1)
        elif kind == 3:
            cphase(psi, n, q0, q1, k)
        elif kind == 4:
            swap(psi, n, q0, q1)
        elif kind == 5:
            apply_ctrl(psi, n, q0, q1, U)
        else:
            raise ValueError("unknown operator kind %d" % kind)
    return psi


def hamiltonian_step(psi, n, dt, terms):
    """One first-order step of Hamiltonian evolution (sec. 7, hbar = 1):
    psi <- [1 - i dt (H1 + H2)] psi, with H a sum of one- and two-body terms
    (qubits, h): h is the 2x2 or 4x4 Hermitian matrix on those qubits
    (local bit b on qubits[b]).  Each term's action h psi is taken on the
    state before the step."""
    src = psi.copy()
    for qubits, h in terms:
        psi += -1j * dt * apply_dense(src.copy(), n, list(qubits), h)
    return psi


def apply_ctrl(psi, n, c, t, U):
    lib().or_apply_ctrl(_state_ptr(psi), n, c, t, _d(_mat(U)))
    return psi


def cnot(psi, n, c, t):
    lib().or_cnot(_state_ptr(psi), n, c, t)
    return psi


def cphase(psi, n, c, t, k):
    lib().or_cphase(_state_ptr(psi), n, c, t, k)
    return psi


def cphase_factor(k: int) -> complex:
    out = np.zeros(2)
    lib().or_cphase_factor(k, _d(out))
    return complex(out[0], out[1])


def swap(psi, n, a, b):
    lib().or_swap(_state_ptr(psi), n, a, b)
    return psi


def hall(psi, n):
    lib().or_hall(_state_ptr(psi), n)
    return psi


def hall2(psi, n) -> np.ndarray:
    out = np.empty_like(psi)
    lib().or_hall2(_state_ptr(psi), _state_ptr(out), n)
    return out


def oracle_flip(psi, n, marked):
    m = np.ascontiguousarray(marked, dtype=np.uint64)
    lib().or_oracle(_state_ptr(psi), n, m.ctypes.data_as(_u64p), len(m))
    return psi


def inv(psi, n):
    lib().or_inv(_state_ptr(psi), n)
    return psi


def grover_step(psi, n, marked):
    m = np.ascontiguousarray(marked, dtype=np.uint64)
    lib().or_grover_step(_state_ptr(psi), n, m.ctypes.data_as(_u64p), len(m))
    return psi


def qft(psi, n):
    lib().or_qft(_state_ptr(psi), n)
    return psi


def shor_prepare(n, n2, x, M) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().or_shor_prepare(_state_ptr(psi), n, n2, x, M)
    return psi


def project(psi, n, lo, w, value) -> float:
    return float(lib().or_project(_state_ptr(psi), n, lo, w, value))


def qft_range(psi, n, lo, w):
    lib().or_qft_range(_state_ptr(psi), n, lo, w)
    return psi


def probs(psi, n) -> np.ndarray:
    p = np.empty(1 << n, dtype=np.float64)
    lib().or_probs(_state_ptr(psi), n, _d(p))
    return p


def norm(psi, n) -> float:
    return float(lib().or_norm(_state_ptr(psi), n))


def expect_pauli(psi, n, xmask: int, zmask: int) -> complex:
    out = np.zeros(2)
    lib().or_expect_pauli(_state_ptr(psi), n, xmask, zmask, _d(out))
    return complex(out[0], out[1])


def apply_pauli(psi, n, xmask: int, zmask: int) -> np.ndarray:
    out = np.empty_like(psi)
    lib().or_apply_pauli(_state_ptr(psi), _state_ptr(out), n, xmask, zmask)
    return out


# ----------------------------------------------------------------- Philox ----

def philox4x32_10(ctr, key) -> tuple[int, int, int, int]:
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


# ------------------------------------------------------------ measurement ----

TWO62 = 4611686018427387904.0


def integer_cdf(p: np.ndarray) -> np.ndarray:
    """W_i = sum_{j<=i} trunc(p_j * 2^62), exact unsigned 64-bit integers."""
    if np.any(~((p >= 0.0) & (p <= 2.0))):
        raise ValueError("probabilities outside [0, 2]")
    w = (p * TWO62).astype(np.uint64)  # truncation toward zero
    return np.cumsum(w, dtype=np.uint64)


def sample_targets(seed: int, shots: int, total: int) -> list[int]:
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    out = []
    for s in range(shots):
        x = philox4x32_10((s & 0xFFFFFFFF, (s >> 32) & 0xFFFFFFFF, 0, 0), key)
        r = (x[0] << 32) | x[1]
        out.append((r * int(total)) >> 64)
    return out


def sample_from_probs(p: np.ndarray, seed: int, shots: int) -> np.ndarray:
    """Seeded Born-rule samples: smallest i with W_i > target (integer CDF)."""
    cdf = integer_cdf(p)
    total = int(cdf[-1])
    if total == 0:
        raise ValueError("zero state")
    tg = np.array(sample_targets(seed, shots, total), dtype=np.uint64)
    return np.searchsorted(cdf, tg, side="right").astype(np.uint64)


def sample_from_probs_c(p: np.ndarray, n: int, seed: int, shots: int) -> np.ndarray:
    """Same definition via the C routine (linear scan); small n only."""
    cdf = np.empty(1 << n, dtype=np.uint64)
    out = np.empty(shots, dtype=np.uint64)
    rc = lib().or_sample_from_probs(_d(np.ascontiguousarray(p)), n, seed, shots,
                                    cdf.ctypes.data_as(_u64p), out.ctypes.data_as(_u64p))
    if rc != 0:
        raise ValueError("bad probabilities")
    return out


# ------------------------------------------------------------- algorithms ----

H_MAT = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
X_MAT = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y_MAT = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z_MAT = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def grover_run(n: int, marked, iters: int) -> np.ndarray:
    """HALL|0..0>, then `iters` applications of G (sec. 5.1)."""
    psi = zero_state(n)
    hall(psi, n)
    for _ in range(iters):
        grover_step(psi, n, marked)
    return psi


def random_circuit_run(circ, psi: np.ndarray | None = None) -> np.ndarray:
    """Apply a workloads.RandomCircuit: per layer U(2) on qubits 0..n-1 then
    the layer's brick-wall CNOTs."""
    n = circ.n
    if psi is None:
        psi = zero_state(n)
    for l in range(circ.layers):
        for q in range(n):
            apply_1q(psi, n, q, circ.U[l, q])
        for (c, t) in circ.cnot_pairs(l):
            cnot(psi, n, c, t)
    return psi


# ----------------------------------------------------- noisy trajectories ----

TAG_NOISE = 0x4E4F4953
TAG_MEAS = 0x4D454153
TAG_READ = 0x52454144


def noise_draw(seed: int, inst: int, stage: int, q: int, thr: int) -> int:
    """Pauli error at noise location (instance, stage, qubit): 0 none, 1 X,
    2 Y, 3 Z.  Philox counter (inst, stage, q, 'NOIS'), key = seed; the error
    fires when word 0 < thr; its type is floor(word1 * 3 / 2^32)."""
    x = philox4x32_10((inst, stage, q, TAG_NOISE), (seed & 0xFFFFFFFF, seed >> 32))
    if x[0] >= thr:
        return 0
    return 1 + ((x[1] * 3) >> 32)


_PAULI = {1: X_MAT, 2: Y_MAT, 3: Z_MAT}


def trajectory_run(n: int, marked: int, iters: int, seed: int, inst: int,
                   thr_gate: int) -> tuple[np.ndarray, int]:
    """One noisy Grover trajectory, literal gate order.  Stage 0 is the
    initial HALL (a draw after each H on its qubit); iteration r has stages
    1+4r (after the oracle, one draw per qubit), 2+4r (after each H of the
    first HALL), 3+4r (after Inv), 4+4r (after each H of the second HALL).
    Returns (final state, number of Pauli errors applied)."""
    psi = zero_state(n)
    errs = 0

    def noise(stage, q):
        nonlocal errs
        e = noise_draw(seed, inst, stage, q, thr_gate)
        if e:
            apply_1q(psi, n, q, _PAULI[e])
            errs += 1

    def noisy_hall(stage):
        for q in range(n):
            apply_1q(psi, n, q, H_MAT)
            noise(stage, q)

    noisy_hall(0)
    m = np.array([marked], dtype=np.uint64)
    for r in range(iters):
        s = 1 + 4 * r
        oracle_flip(psi, n, m)
        for q in range(n):
            noise(s, q)
        noisy_hall(s + 1)
        inv(psi, n)
        for q in range(n):
            noise(s + 2, q)
        noisy_hall(s + 3)
    return psi, errs


def readout_success(p: np.ndarray, n: int, marked: int, p_ro: float) -> float:
    """Probability that the read-out bit string equals `marked` when each
    measured bit flips independently with probability p_ro:
    sum_j p_j p_ro^d (1-p_ro)^(n-d), d = Hamming distance of j and marked."""
    j = np.arange(1 << n, dtype=np.uint64)
    d = np.zeros(1 << n, dtype=np.int64)
    x = j ^ np.uint64(marked)
    for b in range(n):
        d += ((x >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    w = (p_ro ** d) * ((1.0 - p_ro) ** (n - d))
    return float(np.sum(p * w))


def readout_weights_c64(psi64: np.ndarray) -> np.ndarray:
    """Integer read-out weights of a complex64 state, the rule the batched
    trajectories measure with: w_j = trunc(re_j^2 2^62) + trunc(im_j^2 2^62).
    Every step is exact in binary64 (a float's square has at most 48
    significant bits, and 2^62 only shifts the exponent)."""
    re = np.ascontiguousarray(psi64).real.astype(np.float64)
    im = np.ascontiguousarray(psi64).imag.astype(np.float64)
    return (re * re * TWO62).astype(np.uint64) + (im * im * TWO62).astype(np.uint64)


def trajectory_measure_weights(w: np.ndarray, n: int, seed: int, inst: int, thr_ro: int) -> int:
    """One seeded measurement of the instance from integer weights w (the
    integer-CDF rule of the sampler with counter (inst, 0xFFFFFFFF, 0,
    'MEAS')), then each bit q flips when the Philox draw (inst, 0xFFFFFFFF,
    q, 'READ') has word 0 < thr_ro."""
    cdf = np.cumsum(np.asarray(w, dtype=np.uint64), dtype=np.uint64)
    total = int(cdf[-1])
    key = (seed & 0xFFFFFFFF, seed >> 32)
    x = philox4x32_10((inst, 0xFFFFFFFF, 0, TAG_MEAS), key)
    r = (x[0] << 32) | x[1]
    target = (r * total) >> 64
    out = int(np.searchsorted(cdf, np.uint64(target), side="right"))
    for q in range(n):
        y = philox4x32_10((inst, 0xFFFFFFFF, q, TAG_READ), key)
        if y[0] < thr_ro:
            out ^= 1 << q
    return out


def trajectory_measure(p: np.ndarray, n: int, seed: int, inst: int, thr_ro: int) -> int:
    """trajectory_measure_weights with the weights trunc(p_j 2^62) of the
    probabilities p (the sampler's rule)."""
    integer_cdf(p)  # validates p
    return trajectory_measure_weights((p * TWO62).astype(np.uint64), n, seed, inst, thr_ro)


# ------------------------------------------------------ adjoint gradient ----

def ry(theta: float) -> np.ndarray:
    c, s = math.cos(theta / 2.0), math.sin(theta / 2.0)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(theta: float) -> np.ndarray:
    return np.array([[complex(math.cos(theta / 2), -math.sin(theta / 2)), 0],
                     [0, complex(math.cos(theta / 2), math.sin(theta / 2))]],
                    dtype=np.complex128)


def ansatz_gates(circ):
    """Flat gate list of a workloads.AnsatzCircuit: ('ry'|'rz', q, k) with
    parameter index k, or ('cnot', c, t)."""
    n = circ.n
    g = []
    for l in range(circ.layers):
        for q in range(n):
            g.append(("ry", q, l * 2 * n + 2 * q))
            g.append(("rz", q, l * 2 * n + 2 * q + 1))
        for i in range(n):
            g.append(("cnot", i, (i + 1) % n))
    return g


def _apply_gate(psi, n, gate, theta, dagger=False):
    kind = gate[0]
    if kind == "cnot":
        cnot(psi, n, gate[1], gate[2])
        return
    U = ry(theta[gate[2]]) if kind == "ry" else rz(theta[gate[2]])
    if dagger:
        U = U.conj().T
    apply_1q(psi, n, gate[1], U)


def ansatz_forward(circ, theta=None) -> np.ndarray:
    theta = circ.theta if theta is None else theta
    psi = zero_state(circ.n)
    for gate in ansatz_gates(circ):
        _apply_gate(psi, circ.n, gate, theta)
    return psi


def hamiltonian_apply(psi, n, terms) -> np.ndarray:
    out = np.zeros_like(psi)
    for (x, z, c) in terms:
        out += c * apply_pauli(psi, n, x, z)
    return out


def energy(psi, n, terms) -> float:
    return float(sum(c * expect_pauli(psi, n, x, z).real for (x, z, c) in terms))


def adjoint_gradient(circ, terms, theta=None) -> tuple[float, np.ndarray]:
    """E(theta) and dE/dtheta by uncomputation (no stored intermediate
    states).  For gate j with generator P_j (U_j = exp(-i theta P_j / 2)):
    dE/dtheta_j = 2 Re <lambda_j| (-i/2) P_j |psi_j> = Im <lambda_j|P_j|psi_j>,
    psi_j the state after gate j, lambda_j = U_{j+1}^dag..U_G^dag H psi."""
    theta = circ.theta if theta is None else theta
    n = circ.n
    psi = ansatz_forward(circ, theta)
    E = energy(psi, n, terms)
    lam = hamiltonian_apply(psi, n, terms)
    grad = np.zeros(circ.n_params)
    for gate in reversed(ansatz_gates(circ)):
        if gate[0] in ("ry", "rz"):
            q = gate[1]
            P = Y_MAT if gate[0] == "ry" else Z_MAT
            Ppsi = psi.copy()
            apply_1q(Ppsi, n, q, P)
            grad[gate[2]] = np.vdot(lam, Ppsi).imag
        _apply_gate(psi, n, gate, theta, dagger=True)
        _apply_gate(lam, n, gate, theta, dagger=True)
    return E, grad
