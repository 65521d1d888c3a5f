"""Shared pieces of the sharded-state tests: a circuit that touches every
combination of local and global qubits, its full-state oracle result, and a
per-shard step built on the oracle (for ranks on the CPU)."""
import numpy as np

import oracle as O
import workloads as W


def circuit(n, seed):
    """HALL, a Haar U(2) on every qubit, CNOT / controlled-U / CPHASEK on
    pairs that mix the highest (global) and lowest (local) qubits, SWAPs,
    three Grover steps with marked items spread over the ranks, the QFT and
    a few more one-qubit gates."""
    g = W.rng(seed)
    ops = [("hall",)]
    U = W.haar_u2(g, n)
    for t in range(n):
        ops.append(("1q", t, U[t]))
    pairs = [(0, n - 1), (n - 1, 0), (n - 1, n - 2), (n - 2, n - 1), (1, 2), (n - 3, 1), (2, n - 2)]
    for k, (c, t) in enumerate(pairs):
        ops.append(("cnot", c, t))
        ops.append(("ctrl", c, t, W.haar_u2(g, 1)[0]))
        ops.append(("cphase", c, t, 1 + k % 4))
    ops += [("swap", 0, n - 1), ("swap", 2, n - 2), ("1q", n - 1, W.haar_u2(g, 1)[0]), ("cnot", n - 1, 0)]
    marked = [int(x) for x in W.marked_indices(g, n, 5)]
    for _ in range(3):
        ops.append(("grover", marked))
    ops.append(("qft",))
    for t in (n - 1, 0, n // 2):
        ops.append(("1q", t, W.haar_u2(g, 1)[0]))
    return ops


def run_oracle(n, ops):
    psi = O.zero_state(n)
    for op in ops:
        apply_full(psi, n, op)
    return psi


def apply_full(psi, n, op):
    k = op[0]
    if k == "hall":
        O.hall(psi, n)
    elif k == "1q":
        O.apply_1q(psi, n, op[1], op[2])
    elif k == "cnot":
        O.cnot(psi, n, op[1], op[2])
    elif k == "ctrl":
        O.apply_ctrl(psi, n, op[1], op[2], op[3])
    elif k == "cphase":
        O.cphase(psi, n, op[1], op[2], op[3])
    elif k == "swap":
        O.swap(psi, n, op[1], op[2])
    elif k == "grover":
        O.grover_step(psi, n, np.asarray(op[1], dtype=np.uint64))
    elif k == "qft":
        O.qft(psi, n)


def run_sharded(S, ops):
    S.reset(0)
    for op in ops:
        k = op[0]
        if k == "hall":
            S.hall()
        elif k == "1q":
            S.apply_1q(op[1], op[2])
        elif k == "cnot":
            S.cnot(op[1], op[2])
        elif k == "ctrl":
            S.apply_ctrl(op[1], op[2], op[3])
        elif k == "cphase":
            S.cphase(op[1], op[2], op[3])
        elif k == "swap":
            S.swap(op[1], op[2])
        elif k == "grover":
            S.grover_step(op[1])
        elif k == "qft":
            S.qft()
    return S.gather()


class OracleShardOps:
    """The per-shard step on the CPU: the oracle's gates on a numpy shard of
    nl qubits (a torch view of it is what the ranks exchange).  The Grover
    pass is its definition: flip the marked items, then C -> 2m - C with the
    mean m of the whole (flipped) state."""

    def __init__(self, nl):
        import torch
        self.nl = nl
        self.psi = np.zeros(1 << nl, dtype=np.complex128)
        self.tensor = torch.from_numpy(self.psi)
        self.device = "cpu"

    def zero(self, local_index=None):
        self.psi[:] = 0
        if local_index is not None:
            self.psi[local_index] = 1.0

    def invalidate(self):
        pass

    def apply_1q(self, q, U):
        O.apply_1q(self.psi, self.nl, q, U)

    def apply_ctrl(self, c, t, U):
        O.apply_ctrl(self.psi, self.nl, c, t, U)

    def cnot(self, c, t):
        O.cnot(self.psi, self.nl, c, t)

    def cphase(self, c, t, k):
        O.cphase(self.psi, self.nl, c, t, k)

    def hadamard_layer(self, mask):
        for q in range(self.nl):
            if (mask >> q) & 1:
                O.apply_1q(self.psi, self.nl, q, O.H_MAT)

    def grover_partial(self, marked_local):
        idx = np.asarray(marked_local, dtype=np.int64)
        return complex(self.psi.sum() - 2.0 * self.psi[idx].sum())

    def grover_apply(self, marked_local, mean):
        idx = np.asarray(marked_local, dtype=np.int64)
        self.psi[idx] = -self.psi[idx]
        self.psi[:] = 2.0 * mean - self.psi

    def norm2(self):
        return float(np.vdot(self.psi, self.psi).real)
