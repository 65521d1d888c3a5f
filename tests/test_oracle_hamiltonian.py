"""Pins of the oracle's first-order Hamiltonian step (sec. 7:
|Psi(t + dt)> = [1 - i (H1 + H2) dt] |Psi(t)>, hbar = 1).  No GPU.

* Against I - i dt H with H assembled from numpy.kron products of the
  one- and two-body terms and identities (contiguous pairs).
* H = sum_q Z_q acts diagonally: psi_j -> (1 - i dt sum_q (-1)^{j_q}) psi_j.
* The step agrees with exp(-i H dt) up to O(dt^2): the local error ratio
  between dt and dt/2 is about 4.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

sl = pytest.importorskip("scipy.linalg")

X = np.array([[0, 1], [1, 0]], dtype=complex)
Z = np.diag([1.0, -1.0]).astype(complex)


def herm(g, d):
    A = g.standard_normal((d, d)) + 1j * g.standard_normal((d, d))
    return (A + A.conj().T) / 2


def terms_and_dense(n, g):
    terms, H = [], np.zeros((1 << n, 1 << n), dtype=complex)
    for q in range(n):
        h = herm(g, 2)
        terms.append(([q], h))
        H += np.kron(np.eye(1 << (n - q - 1)), np.kron(h, np.eye(1 << q)))
    for q in range(n - 1):
        h = herm(g, 4)
        terms.append(([q, q + 1], h))  # local bit 0 on q, bit 1 on q+1
        H += np.kron(np.eye(1 << (n - q - 2)), np.kron(h, np.eye(1 << q)))
    return terms, H


def test_step_equals_identity_minus_i_dt_h():
    n, dt = 5, 0.013
    g = W.rng(7)
    terms, H = terms_and_dense(n, g)
    v = W.random_state(g, n)
    got = O.hamiltonian_step(v.copy(), n, dt, terms)
    ref = (np.eye(1 << n) - 1j * dt * H) @ v
    assert np.max(np.abs(got - ref)) < 1e-14


def test_sum_of_z_is_diagonal():
    n, dt = 6, 0.05
    v = W.random_state(W.rng(8), n)
    got = O.hamiltonian_step(v.copy(), n, dt, [([q], Z) for q in range(n)])
    j = np.arange(1 << n)
    s = sum(1 - 2 * ((j >> q) & 1) for q in range(n))
    assert np.max(np.abs(got - (1 - 1j * dt * s) * v)) < 1e-15


def test_first_order_in_dt():
    n = 4
    g = W.rng(9)
    terms, H = terms_and_dense(n, g)
    v = W.random_state(g, n)
    errs = []
    for dt in (0.02, 0.01):
        got = O.hamiltonian_step(v.copy(), n, dt, terms)
        errs.append(np.linalg.norm(got - sl.expm(-1j * dt * H) @ v))
    assert 3.5 < errs[0] / errs[1] < 4.5
