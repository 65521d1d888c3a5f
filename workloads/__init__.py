"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds input generation only -- no gate arithmetic, no simulation.
Every random quantity the method consumes as *input* (gate matrices, marked
items, rotation angles, instance sizes) is drawn here from numpy's PCG64 with
an explicit seed and handed to both sides.  Random numbers the method draws
*inside* a run (noise, measurement) come from Philox4x32-10, which each side
implements on its own.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def haar_u2(g: np.random.Generator, count: int) -> np.ndarray:
    """Haar-random U(2) matrices, shape (count, 8) as interleaved row-major
    (re, im) doubles.  Euler-Hurwitz parametrisation: e^{i a} [[e^{i psi} cos
    phi, e^{i chi} sin phi], [-e^{-i chi} sin phi, e^{-i psi} cos phi]] with
    phi = asin(sqrt(xi)), xi ~ U[0,1) and a, psi, chi ~ U[0, 2 pi)."""
    xi = g.random(count)
    a, psi, chi = (g.random((3, count)) * 2.0 * math.pi)
    phi = np.arcsin(np.sqrt(xi))
    e = np.exp(1j * a)
    u00 = e * np.exp(1j * psi) * np.cos(phi)
    u01 = e * np.exp(1j * chi) * np.sin(phi)
    u10 = -e * np.exp(-1j * chi) * np.sin(phi)
    u11 = e * np.exp(-1j * psi) * np.cos(phi)
    m = np.stack([u00, u01, u10, u11], axis=1)
    return np.ascontiguousarray(np.stack([m.real, m.imag], axis=2).reshape(count, 8))


def marked_indices(g: np.random.Generator, n: int, count: int) -> np.ndarray:
    """`count` distinct marked items in [0, 2^n), drawn without replacement
    (sorted ascending)."""
    N = 1 << n
    if count > N:
        raise ValueError("more marked items than basis states")
    out: set[int] = set()
    while len(out) < count:
        out.add(int(g.integers(0, N)))
    return np.array(sorted(out), dtype=np.uint64)


def grover_iterations(n: int) -> int:
    """floor(pi/4 * sqrt(2^n)): the iteration count of sec. 5.1, rounded down."""
    return int(math.floor(math.pi / 4.0 * math.sqrt(2.0 ** n)))


def random_state(g: np.random.Generator, n: int) -> np.ndarray:
    """Normalised complex128 state with Gaussian amplitudes."""
    v = g.standard_normal(1 << n) + 1j * g.standard_normal(1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex128)


# ---------------------------------------------------------------- configs ----

@dataclass
class RandomCircuit:
    """Random circuit of `layers` layers on n qubits: a Haar U(2) on every qubit
    (qubit 0 first), then a brick wall of CNOT(i, i+1) on pairs starting at
    bit 0 in even layers and bit 1 in odd layers (no wrap-around)."""
    n: int
    layers: int
    U: np.ndarray  # (layers, n, 8)

    def cnot_pairs(self, layer: int) -> list[tuple[int, int]]:
        start = layer % 2
        return [(i, i + 1) for i in range(start, self.n - 1, 2)]


def random_circuit(n: int, layers: int, seed: int) -> RandomCircuit:
    g = rng(seed)
    U = haar_u2(g, layers * n).reshape(layers, n, 8)
    return RandomCircuit(n=n, layers=layers, U=U)


@dataclass
class TrajectoryBatch:
    """Noisy-trajectory instances: qubit count, marked item and iteration count
    per instance, plus the noise probabilities as 32-bit integer thresholds
    (an event fires when a 32-bit Philox word is below the threshold)."""
    nq: np.ndarray       # int32 (n_inst,)
    marked: np.ndarray   # uint64 (n_inst,)
    iters: np.ndarray    # int32 (n_inst,)
    p_gate: float
    p_readout: float
    seed: int

    @property
    def thr_gate(self) -> int:
        return prob_threshold(self.p_gate)

    @property
    def thr_readout(self) -> int:
        return prob_threshold(self.p_readout)


def prob_threshold(p: float) -> int:
    """floor(p * 2^32), clamped to [0, 2^32 - 1]."""
    return int(min(max(math.floor(p * 4294967296.0), 0), 4294967295))


def trajectory_batch(n_inst: int, n_lo: int, n_hi: int, seed: int,
                     p_gate: float = 1e-3, p_readout: float = 1e-3) -> TrajectoryBatch:
    g = rng(seed)
    nq = g.integers(n_lo, n_hi + 1, size=n_inst).astype(np.int32)
    marked = np.array([int(g.integers(0, 1 << int(k))) for k in nq], dtype=np.uint64)
    iters = np.array([grover_iterations(int(k)) for k in nq], dtype=np.int32)
    return TrajectoryBatch(nq=nq, marked=marked, iters=iters, p_gate=p_gate,
                           p_readout=p_readout, seed=seed)


@dataclass
class AnsatzCircuit:
    """Layered ansatz: per layer, RY(theta[l,q,0]) then RZ(theta[l,q,1]) on
    every qubit q (q = 0 first), then CNOT(i, (i+1) mod n) for i = 0..n-1.
    Angles are flat with index l*2n + 2q + j."""
    n: int
    layers: int
    theta: np.ndarray  # (layers*2n,) float64

    @property
    def n_params(self) -> int:
        return self.layers * 2 * self.n


def ansatz(n: int, layers: int, seed: int, batch: int = 1) -> list[AnsatzCircuit]:
    g = rng(seed)
    th = g.random((batch, layers * 2 * n)) * 2.0 * math.pi
    return [AnsatzCircuit(n=n, layers=layers, theta=th[b].copy()) for b in range(batch)]


def ansatz_hamiltonian(n: int) -> list[tuple[int, int, float]]:
    """H = Z0 Z1 + 0.1 * sum_i X_i as (xmask, zmask, coefficient) Pauli terms,
    qubit 0 = least significant bit."""
    terms = [(0, 0b11, 1.0)]
    terms += [(1 << i, 0, 0.1) for i in range(n)]
    return terms


@dataclass
class MultiverseNoise:
    """One intrusion per noisy universe (sec. 6.3 "Noise scenarios"):
    universe 0 runs without noise; universe b >= 1 gets a Wigner rotation
    D^{1/2}(alpha, beta, 0) on qubit qhit (kind 1) or D^{3/2}(alpha, beta, 0)
    on the pair (qhit, qhit2) (kind 2) before iteration eloc (eloc = iters
    puts it after the last one).  P holds the universes' weights."""
    kind: np.ndarray    # (B,) int: 0 none, 1 one-qubit, 2 two-qubit
    qhit: np.ndarray    # (B,) int
    qhit2: np.ndarray   # (B,) int (kind 2 only)
    eloc: np.ndarray    # (B,) int in [0, iters]
    alpha: np.ndarray   # (B,) float in [0, 2 pi)
    beta: np.ndarray    # (B,) float in [0, pi]
    P: np.ndarray       # (B,) float, sum 1


def multiverse_noise(B: int, n: int, iters: int, seed: int, two_qubit_every: int = 4,
                     P: np.ndarray | None = None) -> MultiverseNoise:
    """Seeded intrusion list: every `two_qubit_every`-th noisy universe
    gets the two-qubit D^{3/2}, the others the one-qubit D^{1/2}; the
    universes are equally weighted unless P is given."""
    g = rng(seed)
    kind = np.zeros(B, dtype=np.int32)
    qhit = np.zeros(B, dtype=np.int32)
    qhit2 = np.zeros(B, dtype=np.int32)
    eloc = np.zeros(B, dtype=np.int32)
    alpha = np.zeros(B)
    beta = np.zeros(B)
    for b in range(1, B):
        kind[b] = 2 if (two_qubit_every and n >= 2 and b % two_qubit_every == 0) else 1
        qhit[b] = int(g.integers(0, n))
        if kind[b] == 2:
            q2 = int(g.integers(0, n - 1))
            qhit2[b] = q2 + (q2 >= qhit[b])
        eloc[b] = int(g.integers(0, iters + 1))
        alpha[b] = g.random() * 2.0 * math.pi
        beta[b] = g.random() * math.pi
    w = np.full(B, 1.0 / B) if P is None else np.asarray(P, dtype=float)
    return MultiverseNoise(kind=kind, qhit=qhit, qhit2=qhit2, eloc=eloc, alpha=alpha, beta=beta, P=w)
