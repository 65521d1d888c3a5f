"""Python binding of the GB300 state-vector gate engine (libqcgb300.so).

Argument marshalling only: every operation runs in the CUDA library behind
the C ABI of include/qc.h.  There is no CPU fallback -- if the library is
not built, importing the functions raises.  PyTorch supplies device memory
and streams (tensors are wrapped by pointer, streams by their handle).

The qubit convention is the library's: qubit t is bit t of the basis index
(t = n_q - i_s in the QCMPI paper's labels, where i_s = 1 is the most
significant qubit).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

QC_OK, QC_EINVAL, QC_ENOMEM, QC_ECUDA, QC_ETIMEOUT = 0, 1, 2, 3, 4
QC_C128, QC_C64 = 0, 1
QC_MAX_QUBITS = 34
QC_MAX_MARKED = 1024
QC_TRAJ_MAX_QUBITS = 22
QC_G_RX, QC_G_RY, QC_G_RZ, QC_G_CNOT, QC_G_H = 0, 1, 2, 3, 4

LIB_PATH = _build.LIB


class QCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("qc status %d: %s" % (status, msg))
        self.status = status


class TrajDesc(ctypes.Structure):
    _fields_ = [("n_inst", ctypes.c_int32), ("nq", ctypes.POINTER(ctypes.c_int32)),
                ("marked", ctypes.POINTER(ctypes.c_uint64)), ("iters", ctypes.POINTER(ctypes.c_int32)),
                ("seed", ctypes.c_uint64), ("thr_gate", ctypes.c_uint32),
                ("thr_readout", ctypes.c_uint32), ("p_readout", ctypes.c_double)]


class TrajOut(ctypes.Structure):
    _fields_ = [("p_success", ctypes.c_void_p), ("p_readout", ctypes.c_void_p),
                ("outcome", ctypes.c_void_p), ("n_errors", ctypes.c_void_p)]


class Gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("param", ctypes.c_int32)]


class PauliTerm(ctypes.Structure):
    _fields_ = [("xmask", ctypes.c_uint64), ("zmask", ctypes.c_uint64), ("coeff", ctypes.c_double)]


_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_U64P = ctypes.POINTER(ctypes.c_uint64)
_I = ctypes.c_int
_U64 = ctypes.c_uint64
_I64 = ctypes.c_int64

# name -> argument types (all return qc_status unless noted)
_SIGS = {
    "qc_state_alloc": [_I, _I, _VP, ctypes.POINTER(_VP)],
    "qc_state_wrap": [_VP, _I, _I, _VP, ctypes.POINTER(_VP)],
    "qc_state_free": [_VP],
    "qc_state_reset": [_VP, _U64],
    "qc_state_uniform": [_VP],
    "qc_state_info": [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "qc_state_set_stream": [_VP, _VP],
    "qc_state_invalidate": [_VP],
    "qc_apply_1q": [_VP, _I, _DP],
    "qc_apply_ctrl": [_VP, _I, _I, _DP],
    "qc_cnot": [_VP, _I, _I],
    "qc_cphase": [_VP, _I, _I, _I],
    "qc_swap": [_VP, _I, _I],
    "qc_hall": [_VP],
    "qc_apply_1q_layer": [_VP, _DP, _U64],
    "qc_grover_step": [_VP, _U64P, _I],
    "qc_grover_run": [_VP, _U64P, _I, _I],
    "qc_grover_partial": [_VP, _U64P, _I, _DP],
    "qc_grover_apply_mean": [_VP, _U64P, _I, _DP],
    "qc_qft": [_VP],
    "qc_apply_2q": [_VP, _I, _I, _DP],
    "qc_shor_prepare": [_VP, _I, _U64, _U64],
    "qc_project": [_VP, _I, _I, _U64, _DP],
    "qc_qft_range": [_VP, _I, _I],
    "qc_norm": [_VP, _DP],
    "qc_probs": [_VP, _VP],
    "qc_expect_pauli": [_VP, _U64, _U64, _DP],
    "qc_renormalize": [_VP, _DP],
    "qc_sample": [_VP, _U64, _I64, _VP],
    "qc_probs_sample": [_VP, _VP, _U64, _I64, _VP],
    "qc_sample_noalloc": [_VP, _I, _I, _U64, _I64, _VP, _VP],
    "qc_traj_plan_create": [ctypes.POINTER(TrajDesc), _VP, _I, ctypes.POINTER(_VP)],
    "qc_traj_plan_run": [_VP, ctypes.POINTER(TrajOut)],
    "qc_traj_plan_run_states": [_VP, ctypes.POINTER(TrajOut), _VP, _VP],
    "qc_traj_plan_info": [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "qc_traj_plan_free": [_VP],
    "qc_circuit_forward": [_I, _I, _I, ctypes.POINTER(Gate), _I, _VP, _I64, _VP, _VP],
    "qc_adjoint_grad": [_I, _I, _I, ctypes.POINTER(Gate), _I, _VP, _I64, _I,
                        ctypes.POINTER(PauliTerm), _I, _VP, _VP, _VP, _VP, _VP],
    "qc_wigner_d": [_I, ctypes.c_double, ctypes.c_double, ctypes.c_double, _DP],
    "qc_apply_dense": [_VP, _I, ctypes.POINTER(_I), _DP],
    "qc_dense_timeout_selftest": [_VP, ctypes.c_uint32],
    "qc_hamiltonian_step": [_VP, ctypes.c_double, _VP, _I],
    "qc_fused_plan_create": [_I, _VP, _I, _I, _I, ctypes.POINTER(_VP)],
    "qc_fused_plan_info": [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "qc_fused_plan_run": [_VP, _VP],
    "qc_fused_plan_block": [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), _DP],
    "qc_fused_plan_free": [_VP],
    "qc_density_matrix": [_VP, _I, _I, _I, _DP, _VP, _VP],
    "qc_mixed_spectrum": [_VP, _I, _I, _I, _DP, _DP, _DP, _VP],
}

_lib = None


def lib():
    """Load libqcgb300.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise ImportError("libqcgb300.so is not built: %s" % path)
        L = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            if not hasattr(L, name):
                continue  # calling a missing export raises AttributeError: no fallback
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.qc_last_error.restype = ctypes.c_char_p
        L.qc_last_error.argtypes = []
        L.qc_version.restype = ctypes.c_char_p
        L.qc_version.argtypes = []
        L.qc_kernel_launches.restype = ctypes.c_ulonglong
        L.qc_kernel_launches.argtypes = []
        _lib = L
    return _lib


def last_error() -> str:
    return lib().qc_last_error().decode()


def _check(st: int):
    if st != QC_OK:
        raise QCError(st, last_error())


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _mat8(U) -> np.ndarray:
    U = np.asarray(U)
    if U.dtype.kind == "c":
        U = np.stack([U.real, U.imag], axis=-1)
    a = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
    if a.size != 8:
        raise ValueError("a 2x2 operator needs 8 doubles")
    return a


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


# ----------------------------------------------------------- raw C calls ----
# Same names as the C ABI; handles are ctypes.c_void_p.

def qc_state_alloc(n: int, dt: int = QC_C128, stream=None):
    h = ctypes.c_void_p()
    _check(lib().qc_state_alloc(n, dt, _stream_handle(stream), ctypes.byref(h)))
    return h


def qc_state_wrap(dev_ptr: int, n: int, dt: int, stream=None):
    h = ctypes.c_void_p()
    _check(lib().qc_state_wrap(ctypes.c_void_p(dev_ptr), n, dt, _stream_handle(stream), ctypes.byref(h)))
    return h


def qc_state_free(h):
    _check(lib().qc_state_free(h))


def qc_state_reset(h, basis: int = 0):
    _check(lib().qc_state_reset(h, basis))


def qc_state_uniform(h):
    _check(lib().qc_state_uniform(h))


def qc_state_set_stream(h, stream):
    _check(lib().qc_state_set_stream(h, _stream_handle(stream)))


def qc_state_invalidate(h):
    _check(lib().qc_state_invalidate(h))


def qc_apply_1q(h, t: int, U):
    _check(lib().qc_apply_1q(h, t, _dptr(_mat8(U))))


def qc_apply_ctrl(h, c: int, t: int, U):
    _check(lib().qc_apply_ctrl(h, c, t, _dptr(_mat8(U))))


def qc_cnot(h, c: int, t: int):
    _check(lib().qc_cnot(h, c, t))


def qc_cphase(h, c: int, t: int, k: int):
    _check(lib().qc_cphase(h, c, t, k))


def qc_swap(h, a: int, b: int):
    _check(lib().qc_swap(h, a, b))


def qc_hall(h):
    _check(lib().qc_hall(h))


def _layer_ops(U, n: int) -> np.ndarray:
    """n one-qubit operators as the 8 n doubles the C call reads: either
    complex (n, 2, 2) matrices or (n, 8) interleaved (re, im) rows."""
    U = np.asarray(U)
    if U.dtype.kind == "c":
        U = np.stack([U.real, U.imag], axis=-1)
    a = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
    if a.size != 8 * n:
        raise ValueError("a layer on %d qubits needs %d operators (8 doubles each), got %d doubles" % (n, n, a.size))
    return a


def qc_apply_1q_layer(h, U, mask: int):
    _, n, _ = qc_state_info(h)
    a = _layer_ops(U, n)
    _check(lib().qc_apply_1q_layer(h, _dptr(a), mask))


def _marked(marked) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(marked, dtype=np.uint64).reshape(-1))


def qc_grover_step(h, marked):
    m = _marked(marked)
    _check(lib().qc_grover_step(h, m.ctypes.data_as(_U64P), len(m)))


def qc_grover_run(h, marked, iters: int):
    m = _marked(marked)
    _check(lib().qc_grover_run(h, m.ctypes.data_as(_U64P), len(m), iters))


def _marked0(marked) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(marked, dtype=np.uint64).reshape(-1))


def qc_grover_partial(h, marked_local) -> complex:
    """S_r - 2 sum_{marked} C of one shard (qc_grover_partial)."""
    m = _marked0(marked_local)
    out = np.zeros(2)
    _check(lib().qc_grover_partial(h, m.ctypes.data_as(_U64P) if m.size else None, int(m.size), _dptr(out)))
    return complex(out[0], out[1])


def qc_grover_apply_mean(h, marked_local, mean: complex):
    m = _marked0(marked_local)
    mv = np.array([mean.real, mean.imag])
    _check(lib().qc_grover_apply_mean(h, m.ctypes.data_as(_U64P) if m.size else None, int(m.size), _dptr(mv)))


def qc_qft(h):
    _check(lib().qc_qft(h))


def qc_apply_2q(h, t1: int, t2: int, V):
    V = np.asarray(V)
    if V.dtype.kind == "c":
        V = np.stack([V.real, V.imag], axis=-1)
    a = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
    if a.size != 32:
        raise ValueError("a 4x4 operator needs 32 doubles")
    _check(lib().qc_apply_2q(h, t1, t2, _dptr(a)))


def qc_apply_dense(h, qubits, U):
    """A dense 2^k x 2^k operator on k qubits (local bit b on qubits[b])."""
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    U = np.asarray(U)
    if U.dtype.kind == "c":
        U = np.stack([U.real, U.imag], axis=-1)
    a = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
    if a.size != 2 * (1 << (2 * q.size)):
        raise ValueError("a 2^k x 2^k operator needs 2 * 4^k doubles")
    _check(lib().qc_apply_dense(h, int(q.size), q.ctypes.data_as(ctypes.POINTER(_I)), _dptr(a)))


QC_OP_1Q, QC_OP_CNOT, QC_OP_CPHASE, QC_OP_SWAP, QC_OP_CTRL = 1, 2, 3, 4, 5


class QCOp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32), ("k", ctypes.c_int32),
                ("m", ctypes.c_double * 8)]


class FusedPlan:
    """A circuit grouped into dense blocks (qc_fused_plan_*).  ops: list of
    (kind, q0, q1, k, U) with U a 2x2 matrix or None."""

    def __init__(self, n: int, ops, kmax: int = 5, pad: bool = True):
        arr = (QCOp * max(1, len(ops)))()
        for i, (kind, q0, q1, k, U) in enumerate(ops):
            arr[i].kind, arr[i].q0, arr[i].q1, arr[i].k = int(kind), int(q0), int(q1), int(k)
            if U is not None:
                u = np.asarray(U)
                if u.shape == (2, 2):  # a matrix (real or complex), not interleaved doubles
                    u = u.astype(complex)
                if u.dtype.kind == "c":
                    u = np.stack([u.real, u.imag], axis=-1)
                flat = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
                for e in range(8):
                    arr[i].m[e] = float(flat[e])
        self.h = ctypes.c_void_p()
        _check(lib().qc_fused_plan_create(n, ctypes.cast(arr, ctypes.c_void_p), len(ops), kmax, int(pad),
                                          ctypes.byref(self.h)))

    def info(self):
        nb, km = _I(), _I()
        _check(lib().qc_fused_plan_info(self.h, ctypes.byref(nb), ctypes.byref(km)))
        return nb.value, km.value

    def block(self, i: int):
        """(qubits, U) of block i."""
        k = _I()
        qs = (_I * 6)()
        _check(lib().qc_fused_plan_block(self.h, i, ctypes.byref(k), qs, None))
        U = np.zeros(2 << (2 * k.value))
        _check(lib().qc_fused_plan_block(self.h, i, None, None, _dptr(U)))
        d = 1 << k.value
        return [qs[j] for j in range(k.value)], (U[0::2] + 1j * U[1::2]).reshape(d, d)

    def run(self, state_h):
        _check(lib().qc_fused_plan_run(state_h, self.h))

    def close(self):
        if self.h:
            lib().qc_fused_plan_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HTerm(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("qubits", ctypes.c_int32 * 2), ("h", ctypes.c_double * 32)]


def qc_dense_timeout_selftest(h, spin_limit: int) -> int:
    """Runs the tensor-core block's timeout path; returns the status code
    (QC_ETIMEOUT when the path works) instead of raising."""
    return int(lib().qc_dense_timeout_selftest(h, int(spin_limit)))


def qc_hamiltonian_step(h, dt: float, terms):
    """psi <- [1 - i dt sum h_t] psi; terms: list of (qubits, 2x2 or 4x4 matrix)."""
    arr = (HTerm * max(1, len(terms)))()
    for i, (qs, m) in enumerate(terms):
        m = np.asarray(m, dtype=complex)
        arr[i].k = len(qs)
        for b, q in enumerate(qs):
            arr[i].qubits[b] = int(q)
        flat = np.stack([m.real, m.imag], axis=-1).reshape(-1)
        for e, x in enumerate(flat):
            arr[i].h[e] = float(x)
    _check(lib().qc_hamiltonian_step(h, dt, ctypes.cast(arr, ctypes.c_void_p), len(terms)))


def qc_shor_prepare(h, n2: int, x: int, M: int):
    _check(lib().qc_shor_prepare(h, n2, x, M))


def qc_project(h, lo: int, width: int, value: int) -> float:
    out = ctypes.c_double()
    _check(lib().qc_project(h, lo, width, value, ctypes.byref(out)))
    return out.value


def qc_qft_range(h, lo: int, width: int):
    _check(lib().qc_qft_range(h, lo, width))


def qc_wigner_d(twoj: int, alpha: float, beta: float, gamma: float = 0.0) -> np.ndarray:
    """D^{twoj/2}(alpha, beta, gamma) as a complex (twoj+1) x (twoj+1) matrix."""
    dim = twoj + 1
    out = np.zeros(2 * dim * dim)
    _check(lib().qc_wigner_d(twoj, alpha, beta, gamma, _dptr(out)))
    return (out[0::2] + 1j * out[1::2]).reshape(dim, dim)


def _weights(P, B):
    w = np.ascontiguousarray(P, dtype=np.float64)
    if w.size != B:
        raise ValueError("need one weight per state")
    return w


def qc_density_matrix(psi_ptr: int, n: int, dt: int, B: int, P, rho_ptr: int, stream: int = 0):
    w = _weights(P, B)
    _check(lib().qc_density_matrix(ctypes.c_void_p(psi_ptr), n, dt, B, _dptr(w), ctypes.c_void_p(rho_ptr),
                                   ctypes.c_void_p(stream)))


def qc_mixed_spectrum(psi_ptr: int, n: int, dt: int, B: int, P, stream: int = 0):
    """(eigenvalues descending, (trace, purity, entropy))."""
    w = _weights(P, B)
    ev = np.zeros(B)
    st = np.zeros(3)
    _check(lib().qc_mixed_spectrum(ctypes.c_void_p(psi_ptr), n, dt, B, _dptr(w), _dptr(ev), _dptr(st),
                                   ctypes.c_void_p(stream)))
    return ev, tuple(st)


def qc_norm(h) -> float:
    out = ctypes.c_double()
    _check(lib().qc_norm(h, ctypes.byref(out)))
    return out.value


def qc_probs(h, out_dev_ptr: int):
    _check(lib().qc_probs(h, ctypes.c_void_p(out_dev_ptr)))


def qc_expect_pauli(h, xmask: int, zmask: int) -> complex:
    out = (ctypes.c_double * 2)()
    _check(lib().qc_expect_pauli(h, xmask, zmask, out))
    return complex(out[0], out[1])


def qc_renormalize(h) -> float:
    out = ctypes.c_double()
    _check(lib().qc_renormalize(h, ctypes.byref(out)))
    return out.value


def qc_sample(h, seed: int, shots: int, out_dev_ptr: int):
    _check(lib().qc_sample(h, seed, shots, ctypes.c_void_p(out_dev_ptr)))


def qc_probs_sample(h, probs_dev_ptr: int, seed: int, shots: int, out_dev_ptr: int):
    _check(lib().qc_probs_sample(h, ctypes.c_void_p(probs_dev_ptr), seed, shots, ctypes.c_void_p(out_dev_ptr)))


# --------------------------------------------------- torch-facing helpers ----

# ---- the remaining entry points under their C names (argument marshalling
# only; the classes below wrap the same calls for everyday use) ----

def qc_version() -> str:
    return lib().qc_version().decode()


def qc_last_error() -> str:
    return last_error()


def qc_kernel_launches() -> int:
    return int(lib().qc_kernel_launches())


def qc_state_info(h):
    """(device pointer, n, dtype) of a state handle."""
    p, n, dt = _VP(), _I(), _I()
    _check(lib().qc_state_info(h, ctypes.byref(p), ctypes.byref(n), ctypes.byref(dt)))
    return p.value, n.value, dt.value


def qc_sample_noalloc(psi_dev_ptr: int, n: int, dt: int, seed: int, shots: int, out_dev_ptr: int, stream=None):
    _check(lib().qc_sample_noalloc(_VP(psi_dev_ptr), n, dt, seed, shots, _VP(out_dev_ptr), _stream_handle(stream)))


def _gate_array(gates):
    if isinstance(gates, ctypes.Array):
        return gates, len(gates)
    gl = [tuple(int(v) for v in g) for g in gates]
    return (Gate * max(1, len(gl)))(*[Gate(*g) for g in gl]), len(gl)


def _term_array(terms):
    if isinstance(terms, ctypes.Array):
        return terms, len(terms)
    tl = [(int(x), int(z), float(c)) for (x, z, c) in terms]
    return (PauliTerm * max(1, len(tl)))(*[PauliTerm(*t) for t in tl]), len(tl)


def qc_circuit_forward(n: int, dt: int, B: int, gates, theta_dev_ptr: int, theta_stride: int, psi_dev_ptr: int,
                       stream=None):
    """gates: (kind, q0, q1, param) tuples or a Gate array."""
    ga, ng = _gate_array(gates)
    _check(lib().qc_circuit_forward(n, dt, B, ga, ng, _VP(theta_dev_ptr), theta_stride, _VP(psi_dev_ptr),
                                    _stream_handle(stream)))


def qc_adjoint_grad(n: int, dt: int, B: int, gates, theta_dev_ptr: int, theta_stride: int, n_params: int, terms,
                    psi_dev_ptr: int, lam_dev_ptr: int, energy_dev_ptr: int, grad_dev_ptr: int, stream=None):
    """gates as for qc_circuit_forward; terms: (xmask, zmask, coeff) tuples or
    a PauliTerm array."""
    ga, ng = _gate_array(gates)
    ta, nt = _term_array(terms)
    _check(lib().qc_adjoint_grad(n, dt, B, ga, ng, _VP(theta_dev_ptr), theta_stride, n_params, ta, nt,
                                 _VP(psi_dev_ptr), _VP(lam_dev_ptr), _VP(energy_dev_ptr), _VP(grad_dev_ptr),
                                 _stream_handle(stream)))


def qc_fused_plan_create(n: int, ops, kmax: int = 5, pad: bool = True):
    """A plan handle for ops as FusedPlan takes them; free with
    qc_fused_plan_free."""
    plan = FusedPlan(n, ops, kmax=kmax, pad=pad)
    h, plan.h = plan.h, None  # hand the handle over
    return h


def qc_fused_plan_info(plan):
    nb, km = _I(), _I()
    _check(lib().qc_fused_plan_info(plan, ctypes.byref(nb), ctypes.byref(km)))
    return nb.value, km.value


def qc_fused_plan_block(plan, i: int):
    """(qubits, U) of block i."""
    k = _I()
    qs = (_I * 6)()
    _check(lib().qc_fused_plan_block(plan, i, ctypes.byref(k), qs, None))
    U = np.zeros(2 << (2 * k.value))
    _check(lib().qc_fused_plan_block(plan, i, None, None, _dptr(U)))
    d = 1 << k.value
    return [qs[j] for j in range(k.value)], (U[0::2] + 1j * U[1::2]).reshape(d, d)


def qc_fused_plan_run(state_h, plan):
    _check(lib().qc_fused_plan_run(state_h, plan))


def qc_fused_plan_free(plan):
    _check(lib().qc_fused_plan_free(plan))


def qc_traj_plan_create(desc: "TrajDesc", stream=None, autotune: bool = True):
    h = _VP()
    _check(lib().qc_traj_plan_create(ctypes.byref(desc), _stream_handle(stream), int(bool(autotune)), ctypes.byref(h)))
    return h


def qc_traj_plan_run(plan, out: "TrajOut"):
    _check(lib().qc_traj_plan_run(plan, ctypes.byref(out)))


def qc_traj_plan_run_states(plan, out: "TrajOut", state_off_dev_ptr: int, states_dev_ptr: int):
    _check(lib().qc_traj_plan_run_states(plan, ctypes.byref(out), _VP(state_off_dev_ptr), _VP(states_dev_ptr)))


def qc_traj_plan_info(plan):
    v = [_I(), _I(), _I()]
    _check(lib().qc_traj_plan_info(plan, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def qc_traj_plan_free(plan):
    _check(lib().qc_traj_plan_free(plan))


def torch_dtype(dt: int):
    import torch
    return torch.complex128 if dt == QC_C128 else torch.complex64


class State:
    """A state vector held in a torch tensor (complex128 or complex64) and
    wrapped by a qc_state handle.  Methods map one-to-one onto the C ABI."""

    def __init__(self, n: int, dt: int = QC_C128, device="cuda", tensor=None, stream=None):
        import torch
        self.n, self.dt = n, dt
        if tensor is None:
            tensor = torch.empty(1 << n, dtype=torch_dtype(dt), device=device)
        assert tensor.is_cuda and tensor.is_contiguous() and tensor.numel() == (1 << n)
        self.tensor = tensor
        self.h = qc_state_wrap(tensor.data_ptr(), n, dt, stream)
        if tensor is not None and stream is None:
            pass

    def close(self):
        if self.h is not None:
            qc_state_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state preparation
    def reset(self, basis: int = 0):
        qc_state_reset(self.h, basis)
        return self

    def uniform(self):
        qc_state_uniform(self.h)
        return self

    def load(self, vec):
        """Copy a host vector into the state (marks cached reductions stale)."""
        import torch
        self.tensor.copy_(torch.as_tensor(np.asarray(vec)).to(self.tensor.dtype))
        qc_state_invalidate(self.h)
        return self

    def numpy(self) -> np.ndarray:
        import torch
        torch.cuda.synchronize()
        return self.tensor.cpu().numpy()

    # gates
    def apply_1q(self, t, U):
        qc_apply_1q(self.h, t, U)

    def apply_ctrl(self, c, t, U):
        qc_apply_ctrl(self.h, c, t, U)

    def cnot(self, c, t):
        qc_cnot(self.h, c, t)

    def cphase(self, c, t, k):
        qc_cphase(self.h, c, t, k)

    def swap(self, a, b):
        qc_swap(self.h, a, b)

    def hall(self):
        qc_hall(self.h)

    def apply_1q_layer(self, U, mask=None):
        if mask is None:
            mask = (1 << self.n) - 1
        qc_apply_1q_layer(self.h, U, mask)

    def grover_step(self, marked):
        qc_grover_step(self.h, marked)

    def grover_run(self, marked, iters):
        qc_grover_run(self.h, marked, iters)

    def qft(self):
        qc_qft(self.h)

    # reductions
    def norm(self) -> float:
        return qc_norm(self.h)

    def probs(self):
        import torch
        p = torch.empty(1 << self.n, dtype=torch.float64, device=self.tensor.device)
        qc_probs(self.h, p.data_ptr())
        return p

    def expect_pauli(self, xmask, zmask) -> complex:
        return qc_expect_pauli(self.h, xmask, zmask)

    def renormalize(self) -> float:
        return qc_renormalize(self.h)

    def sample(self, seed, shots):
        import torch
        out = torch.empty(max(shots, 1), dtype=torch.int64, device=self.tensor.device)
        qc_sample(self.h, seed, shots, out.data_ptr())
        return out[:shots]

    def probs_sample(self, seed, shots):
        """(probabilities, outcomes) as probs() and sample(seed, shots) give
        them, from one read of the state."""
        import torch
        p = torch.empty(1 << self.n, dtype=torch.float64, device=self.tensor.device)
        out = torch.empty(max(shots, 1), dtype=torch.int64, device=self.tensor.device)
        qc_probs_sample(self.h, p.data_ptr(), seed, shots, out.data_ptr())
        return p, out[:shots]


def version() -> str:
    return lib().qc_version().decode()


def kernel_launches() -> int:
    """Kernels this library has launched in this process so far."""
    return int(lib().qc_kernel_launches())


# ------------------------------------------ the adjoint gradient in autograd --

class Circuit:
    """A parameterised circuit on n qubits and a Hamiltonian, for
    energy(theta, circuit).  gates: (kind, q0, q1, param) with the QC_G_*
    kinds (param indexes theta for rotations; q1 only for CNOT); terms:
    Pauli terms (xmask, zmask, coeff) with real coefficients."""

    def __init__(self, n: int, gates, terms, dt: int = QC_C128):
        self.n, self.dt = int(n), int(dt)
        gl = [tuple(int(v) for v in g) for g in gates]
        tl = [(int(x), int(z), float(c)) for (x, z, c) in terms]
        self.n_gates, self.n_terms = len(gl), len(tl)
        self.gates = (Gate * max(1, len(gl)))(*[Gate(*g) for g in gl])
        self.terms = (PauliTerm * max(1, len(tl)))(*[PauliTerm(*t) for t in tl])
        rot = [g[3] for g in gl if g[0] in (QC_G_RX, QC_G_RY, QC_G_RZ)]
        self.n_params = max(rot) + 1 if rot else 0

    def energy_and_grad(self, theta):
        """E_b and dE_b/dtheta for theta of shape (B, P) (float64, CUDA): one
        qc_adjoint_grad call (forward, then the adjoint backward sweep)."""
        import torch
        B, P = theta.shape
        psi = torch.empty(B << self.n, dtype=torch_dtype(self.dt), device=theta.device)
        lam = torch.empty_like(psi)
        E = torch.empty(B, dtype=torch.float64, device=theta.device)
        grad = torch.empty(B, P, dtype=torch.float64, device=theta.device)
        _check(lib().qc_adjoint_grad(self.n, self.dt, B, self.gates, self.n_gates, _VP(theta.data_ptr()), P, P,
                                     self.terms, self.n_terms, _VP(psi.data_ptr()), _VP(lam.data_ptr()),
                                     _VP(E.data_ptr()), _VP(grad.data_ptr()), _stream_handle(None)))
        return E, grad

    def energy(self, theta):
        """E_b for theta of shape (B, P): the forward pass and the Pauli
        expectations, no backward sweep."""
        import torch
        B, P = theta.shape
        psi = torch.empty(B << self.n, dtype=torch_dtype(self.dt), device=theta.device)
        _check(lib().qc_circuit_forward(self.n, self.dt, B, self.gates, self.n_gates, _VP(theta.data_ptr()), P,
                                        _VP(psi.data_ptr()), _stream_handle(None)))
        E = torch.empty(B, dtype=torch.float64)
        for b in range(B):
            s = State(self.n, self.dt, tensor=psi[b << self.n:(b + 1) << self.n])
            E[b] = sum(c * s.expect_pauli(x, z).real for (x, z, c) in
                       ((t.xmask, t.zmask, t.coeff) for t in self.terms[:self.n_terms]))
            s.close()
        return E.to(theta.device)


_ADJ = None


def _adjoint_function():
    """torch.autograd.Function whose forward runs the adjoint method: the
    energy and its whole gradient come from one forward and one backward
    sweep over the state (uncomputation with U^dagger, no stored
    intermediate states); backward only scales the saved gradient."""
    global _ADJ
    if _ADJ is None:
        import torch
        from torch.autograd.function import once_differentiable

        class AdjointEnergy(torch.autograd.Function):
            @staticmethod
            def forward(ctx, theta, circuit):
                if not theta.is_cuda:
                    raise ValueError("energy(): theta must be a CUDA tensor (there is no CPU path)")
                vec = theta.dim() == 1
                th = (theta.detach().unsqueeze(0) if vec else theta.detach()).to(torch.float64).contiguous()
                if th.shape[1] < circuit.n_params:
                    raise ValueError("energy(): theta has %d angles, the circuit uses %d"
                                     % (th.shape[1], circuit.n_params))
                if ctx.needs_input_grad[0]:
                    E, grad = circuit.energy_and_grad(th)
                    ctx.save_for_backward(grad)
                else:
                    E = circuit.energy(th)
                ctx.vec, ctx.tdtype = vec, theta.dtype
                return E[0] if vec else E

            @staticmethod
            @once_differentiable
            def backward(ctx, gE):
                (grad,) = ctx.saved_tensors
                g = (gE.reshape(-1, 1).to(torch.float64) * grad).to(ctx.tdtype)
                return (g[0] if ctx.vec else g), None

        _ADJ = AdjointEnergy
    return _ADJ


def energy(theta, circuit: Circuit):
    """E(theta) = <psi(theta)|H|psi(theta)> for theta of shape (P,) or (B, P),
    differentiable in theta through the adjoint gradient kernels."""
    return _adjoint_function().apply(theta, circuit)


# ------------------------------------------------- batched noisy trajectories --

def _threshold(p: float) -> int:
    """floor(p * 2^32), the integer threshold of a draw (qc_traj_desc)."""
    if not 0.0 <= p <= 1.0:
        raise ValueError("probability %r outside [0, 1]" % (p,))
    return min(int(math.floor(p * 4294967296.0)), 0xFFFFFFFF)


class TrajectoryPlan:
    """A batch of noisy Grover trajectories (qc_traj_plan_*): nq, marked and
    iters per instance, per-gate Pauli noise p_gate and read-out flips
    p_readout.  Creating it validates and uploads the batch and (autotune)
    times the launch shapes; run() executes every instance in one persistent
    launch and returns device tensors p_success, p_readout, outcome and
    n_errors."""

    def __init__(self, nq, marked, iters, seed: int, p_gate: float = 1e-3, p_readout: float = 1e-3,
                 autotune: bool = True, stream=None):
        self._nq = np.ascontiguousarray(nq, dtype=np.int32)
        self._mk = np.ascontiguousarray(marked, dtype=np.uint64)
        self._it = np.ascontiguousarray(iters, dtype=np.int32)
        if not (len(self._nq) == len(self._mk) == len(self._it)):
            raise ValueError("nq, marked and iters need one entry per instance")
        self.n_inst = len(self._nq)
        d = TrajDesc(self.n_inst, self._nq.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                     self._mk.ctypes.data_as(_U64P), self._it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                     int(seed), _threshold(p_gate), _threshold(p_readout), float(p_readout))
        self.h = ctypes.c_void_p()
        _check(lib().qc_traj_plan_create(ctypes.byref(d), _stream_handle(stream), int(bool(autotune)),
                                         ctypes.byref(self.h)))

    @property
    def shape(self):
        """(CTAs per instance, threads per CTA, grid) of the chosen launch."""
        v = [ctypes.c_int(), ctypes.c_int(), ctypes.c_int()]
        _check(lib().qc_traj_plan_info(self.h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def run(self, keep=()):
        """Runs every instance.  keep: instance indices whose final complex64
        states (the ones their read-outs are drawn from) are returned too,
        as out["states"][i]."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        out = {"p_success": torch.empty(self.n_inst, dtype=torch.float64, device=dev),
               "p_readout": torch.empty(self.n_inst, dtype=torch.float64, device=dev),
               "outcome": torch.empty(self.n_inst, dtype=torch.int64, device=dev),
               "n_errors": torch.empty(self.n_inst, dtype=torch.int32, device=dev)}
        o = TrajOut(out["p_success"].data_ptr(), out["p_readout"].data_ptr(), out["outcome"].data_ptr(),
                    out["n_errors"].data_ptr())
        keep = sorted(set(int(i) for i in keep))
        if not keep:
            _check(lib().qc_traj_plan_run(self.h, ctypes.byref(o)))
            return out
        off = np.full(self.n_inst, np.iinfo(np.uint64).max, dtype=np.uint64)
        pos = 0
        for i in keep:
            off[i] = pos
            pos += 1 << int(self._nq[i])
        states = torch.empty(pos, dtype=torch.complex64, device=dev)
        off_d = torch.from_numpy(off.view(np.int64)).to(dev)
        _check(lib().qc_traj_plan_run_states(self.h, ctypes.byref(o), _VP(off_d.data_ptr()),
                                             _VP(states.data_ptr())))
        out["states"] = {i: states[int(off[i]):int(off[i]) + (1 << int(self._nq[i]))] for i in keep}
        out["_state_offsets"] = off_d  # kept alive until the run has finished
        return out

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().qc_traj_plan_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
