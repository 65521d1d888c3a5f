"""Pins of the oracle's noise intrusions and density matrix (sec. 6.1-6.3),
against facts the paper and the mathematics fix.  No GPU.

* D^j(alpha, beta, gamma) = exp(-i alpha J_z) exp(-i beta J_y)
  exp(-i gamma J_z) with the spin matrices built from the ladder operator
  (the generator definition, independent of the sum formula), for
  j = 1/2 .. 2; unitarity; D^{1/2}(0, pi, 0) is the Pauli product -i Y
  (the paper: "within a phase, ... one of the Pauli operators").
* A pure state has eigenvalues {1, 0, ...} and entropy 0, Tr rho = 1 and
  rho^2 = rho (the paper's statements about the pure-state density matrix).
* An equal mixture of orthogonal states has eigenvalues P_alpha and entropy
  -sum P ln P (closed form).
* Unitary intrusions keep Tr rho = 1 while Tr rho^2 drops below 1 and the
  success probability <m|rho|m> drops below the noiseless one (sec. 6.3).
* The nonzero eigenvalues of rho equal those of the B x B Gram matrix
  P^{1/2} Psi Psi^dagger P^{1/2} (the identity the GPU path relies on).
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.density as D
import workloads as W

sl = pytest.importorskip("scipy.linalg")


def spin(twoj):
    j = twoj / 2.0
    m = [j - r for r in range(twoj + 1)]
    Jp = np.zeros((twoj + 1, twoj + 1))
    for c in range(1, twoj + 1):  # J+ |m> = sqrt(j(j+1) - m(m+1)) |m+1>
        Jp[c - 1, c] = math.sqrt(j * (j + 1) - m[c] * (m[c] + 1))
    Jy = (Jp - Jp.T) / 2j
    return Jy, np.diag(m)


@pytest.mark.parametrize("twoj", [1, 2, 3, 4])
def test_wigner_matches_generators(twoj):
    Jy, Jz = spin(twoj)
    for (a, b, g) in [(0.0, 0.3, 0.0), (0.7, 1.1, -0.4), (5.9, 2.9, 1.3), (1.0, math.pi, 0.0)]:
        ref = sl.expm(-1j * a * Jz) @ sl.expm(-1j * b * Jy) @ sl.expm(-1j * g * Jz)
        got = D.wigner_D(twoj, a, b, g)
        assert np.max(np.abs(got - ref)) < 1e-13
        assert np.max(np.abs(got @ got.conj().T - np.eye(twoj + 1))) < 1e-13


def test_wigner_half_special_cases():
    Y = np.array([[0, -1j], [1j, 0]])
    assert np.max(np.abs(D.wigner_D(1, 0.0, math.pi, 0.0) - (-1j) * Y)) < 1e-15
    a = 0.37
    assert np.max(np.abs(D.wigner_D(1, a, 0.0, 0.0) - np.diag([np.exp(-0.5j * a), np.exp(0.5j * a)]))) < 1e-15


def test_pure_state_density_matrix():
    psi = W.random_state(W.rng(1), 6)
    rho = D.density_matrix(psi[None, :], [1.0])
    assert abs(np.trace(rho) - 1.0) < 1e-13
    assert np.max(np.abs(rho @ rho - rho)) < 1e-13
    ev = D.spectrum(rho)
    assert abs(ev[0] - 1.0) < 1e-12 and np.max(np.abs(ev[1:])) < 1e-12
    assert abs(D.entropy(ev, cut=1e-10)) < 1e-10


def test_orthogonal_mixture_closed_form():
    n, P = 5, np.array([0.5, 0.3, 0.2])
    states = np.zeros((3, 1 << n), dtype=complex)
    for a, idx in enumerate((3, 17, 30)):
        states[a, idx] = np.exp(1j * a)
    rho = D.density_matrix(states, P)
    ev = D.spectrum(rho)
    assert np.max(np.abs(ev[:3] - np.sort(P)[::-1])) < 1e-15
    assert abs(D.entropy(ev) + np.sum(P * np.log(P))) < 1e-14
    assert abs(D.purity(rho) - np.sum(P ** 2)) < 1e-15


def intrusions(mv, b):
    kind = int(mv.kind[b])
    if kind == 0:
        return (0, (), 0, None)
    if kind == 1:
        return (1, (int(mv.qhit[b]),), int(mv.eloc[b]), D.wigner_D(1, mv.alpha[b], mv.beta[b], 0.0))
    return (2, (int(mv.qhit[b]), int(mv.qhit2[b])), int(mv.eloc[b]), D.wigner_D(3, mv.alpha[b], mv.beta[b], 0.0))


def test_multiverse_noise_lowers_purity_and_success():
    n, m = 7, 45
    k = W.grover_iterations(n)
    mv = W.multiverse_noise(12, n, k, seed=9)
    states = D.multiverse_grover(n, m, k, [intrusions(mv, b) for b in range(12)])
    rho = D.density_matrix(states, mv.P)
    assert abs(np.trace(rho).real - 1.0) < 1e-13  # unitary noise keeps unit trace
    pur = D.purity(rho)
    assert pur < 1.0 - 1e-3
    ev = D.spectrum(rho)
    assert np.min(ev) > -1e-13
    assert abs(np.sum(ev ** 2) - pur) < 1e-12
    assert D.entropy(ev) > 1e-3
    # universe 0 is the noiseless Grover state of the closed form
    th = math.asin(2 ** (-n / 2))
    assert abs(abs(states[0, m]) ** 2 - math.sin((2 * k + 1) * th) ** 2) < 1e-12
    assert rho[m, m].real < abs(states[0, m]) ** 2
    # identical universes: a pure ensemble
    same = D.density_matrix(np.repeat(states[:1], 4, axis=0), np.full(4, 0.25))
    assert abs(D.purity(same) - 1.0) < 1e-12


def test_gram_spectrum_equals_rho_spectrum():
    n, B = 6, 5
    g = W.rng(4)
    states = np.stack([W.random_state(g, n) for _ in range(B)])
    P = g.random(B)
    P /= P.sum()
    rho = D.density_matrix(states, P)
    Gm = np.sqrt(P)[:, None] * (states.conj() @ states.T) * np.sqrt(P)[None, :]
    ev_g = np.sort(np.linalg.eigvalsh(Gm))[::-1]
    ev_r = D.spectrum(rho)
    assert np.max(np.abs(ev_r[:B] - ev_g)) < 1e-13
    assert np.max(np.abs(ev_r[B:])) < 1e-13
