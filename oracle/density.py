"""Oracle for the paper's noise intrusions and ensemble density matrix --
TEST INFRASTRUCTURE ONLY (imported by tests/, smoke() and bench.py's CPU
leg, never by the CUDA library).

* Wigner rotation matrices D^j(alpha, beta, gamma) (sec. 6.3, "Noise
  scenarios": D2 = D^{1/2}, a one-qubit intrusion; D4 = D^{3/2}, a
  two-qubit one), from the textbook sum formula for the reduced matrix
  d^j_{m'm}(beta) and D^j_{m'm} = e^{-i m' alpha} d^j_{m'm}(beta)
  e^{-i m gamma}, rows and columns ordered m = j, j-1, ..., -j.
* A multiverse (sec. 6.2-6.3): B copies of Grover's algorithm, each with
  at most one intrusion U on qubit(s) `qhit` before iteration `eloc`.
* The ensemble density matrix (sec. 6.1):
  <n|rho|n'> = sum_alpha P_alpha C_alpha(n) C_alpha(n')^*, its eigenvalues
  (numpy.linalg.eigvalsh, a library step), trace, purity Tr rho^2 and the
  von Neumann entropy -sum lambda ln lambda (natural logarithm).
"""
from __future__ import annotations

import math

import numpy as np

from . import apply_1q, apply_2q, grover_step, hall, zero_state


def wigner_small_d(twoj: int, beta: float) -> np.ndarray:
    """d^j_{m'm}(beta) for j = twoj/2, by the sum over s of
    (-1)^(m'-m+s) cos(b/2)^(2j+m-m'-2s) sin(b/2)^(m'-m+2s) with the
    factorial weights sqrt((j+m')!(j-m')!(j+m)!(j-m)!) /
    ((j+m-s)! s! (m'-m+s)! (j-m'-s)!)."""
    dim = twoj + 1
    d = np.zeros((dim, dim))
    c, s_ = math.cos(beta / 2.0), math.sin(beta / 2.0)
    f = math.factorial
    for r in range(dim):          # m' = j - r, in units of 1/2: twomp = twoj - 2r
        for col in range(dim):    # m = j - col
            jpmp, jmmp = twoj - r, r           # j+m', j-m' (integers)
            jpm, jmm = twoj - col, col         # j+m, j-m
            mp_m = col - r                     # m' - m
            tot = 0.0
            for s in range(0, dim + 1):
                a1, a2, a3 = jpm - s, mp_m + s, jmmp - s
                if a1 < 0 or a2 < 0 or a3 < 0:
                    continue
                ec = twoj - mp_m - 2 * s       # 2j + m - m' - 2s
                es = mp_m + 2 * s              # m' - m + 2s
                term = (-1.0) ** (mp_m + s) * c ** ec * s_ ** es
                term /= f(a1) * f(s) * f(a2) * f(a3)
                tot += term
            d[r, col] = math.sqrt(f(jpmp) * f(jmmp) * f(jpm) * f(jmm)) * tot
    return d


def wigner_D(twoj: int, alpha: float, beta: float, gamma: float) -> np.ndarray:
    """D^j_{m'm}(alpha, beta, gamma) = e^{-i m' alpha} d^j_{m'm}(beta) e^{-i m gamma}."""
    d = wigner_small_d(twoj, beta)
    m = np.array([(twoj - 2 * r) / 2.0 for r in range(twoj + 1)])
    return np.exp(-1j * m * alpha)[:, None] * d * np.exp(-1j * m * gamma)[None, :]


def multiverse_grover(n: int, marked: int, iters: int, noise) -> np.ndarray:
    """B final states (rows) of Grover's algorithm (HALL|0>, then `iters`
    literal Grover operators), universe b receiving noise[b] = (kind,
    qubits, eloc, U) before iteration eloc: kind 0 = none, 1 = a one-qubit
    U on qubits[0], 2 = a two-qubit V on (qubits[0], qubits[1]).  An eloc
    equal to `iters` puts the intrusion after the last iteration."""
    out = np.zeros((len(noise), 1 << n), dtype=complex)
    for b, (kind, qubits, eloc, U) in enumerate(noise):
        psi = zero_state(n)
        hall(psi, n)
        for it in range(iters + 1):
            if kind and it == eloc:
                if kind == 1:
                    apply_1q(psi, n, qubits[0], U)
                else:
                    apply_2q(psi, n, qubits[0], qubits[1], U)
            if it < iters:
                grover_step(psi, n, [marked])
        out[b] = psi
    return out


def density_matrix(states: np.ndarray, P) -> np.ndarray:
    """<n|rho|n'> = sum_alpha P_alpha C_alpha(n) C_alpha(n')^* (the plain
    definition, one outer product per universe)."""
    rho = np.zeros((states.shape[1], states.shape[1]), dtype=complex)
    for a in range(states.shape[0]):
        rho += P[a] * np.outer(states[a], states[a].conj())
    return rho


def spectrum(rho: np.ndarray) -> np.ndarray:
    """Eigenvalues of the Hermitian rho, descending."""
    return np.sort(np.linalg.eigvalsh(rho))[::-1]


def entropy(evals, cut: float = 1e-14) -> float:
    """-sum lambda ln lambda over the eigenvalues above `cut`."""
    ev = np.asarray(evals, dtype=float)
    ev = ev[ev > cut]
    return float(-np.sum(ev * np.log(ev)))


def purity(rho: np.ndarray) -> float:
    """Tr rho^2."""
    return float(np.real(np.trace(rho @ rho)))
