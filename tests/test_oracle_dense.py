"""Pins of the oracle's dense k-qubit block (OneOpA / TwoOpA of sec. 3-4
extended to k qubits).  No GPU.

* k = 1 equals the C oracle's OneOpA for every target, and k = 2 with
  qubits (t2, t1) equals its TwoOpA(t1, t2) (quartet position
  2 q_{t1} + q_{t2}, Eq. twoopB).
* A block built as the Kronecker product of one-qubit matrices equals
  those one-qubit gates applied one after another.
* Against the full 2^n x 2^n operator built with numpy.kron and identities
  (brute force) for random unitaries on random qubit sets.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def unitary(g, d):
    A = g.standard_normal((d, d)) + 1j * g.standard_normal((d, d))
    Q, _ = np.linalg.qr(A)
    return Q


def test_k1_is_oneopa_and_k2_is_twoopa():
    n = 6
    g = W.rng(1)
    for t in range(n):
        U = unitary(g, 2)
        v = W.random_state(g, n)
        assert np.max(np.abs(O.apply_dense(v.copy(), n, [t], U) - O.apply_1q(v.copy(), n, t, U))) < 1e-15
    for t1 in range(n):
        for t2 in range(n):
            if t1 != t2:
                V = unitary(g, 4)
                v = W.random_state(g, n)
                a = O.apply_dense(v.copy(), n, [t2, t1], V)
                b = O.apply_2q(v.copy(), n, t1, t2, V)
                assert np.max(np.abs(a - b)) < 1e-14


def test_kron_block_equals_sequential_gates():
    n, qs = 8, [5, 0, 3]
    g = W.rng(2)
    Us = [unitary(g, 2) for _ in qs]
    big = np.array([[1.0]])
    for U in Us:  # local bit b = qubit qs[b]: qs[0] is the least significant factor
        big = np.kron(U, big)
    v = W.random_state(g, n)
    a = O.apply_dense(v.copy(), n, qs, big)
    b = v.copy()
    for q, U in zip(qs, Us):
        O.apply_1q(b, n, q, U)
    assert np.max(np.abs(a - b)) < 1e-14


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_against_full_operator(k):
    n = 6
    g = W.rng(10 + k)
    qs = list(g.permutation(n)[:k])
    U = unitary(g, 1 << k)
    # full operator: <i|F|j> = U[l(i)][l(j)] if i and j agree off the block
    offs = O.dense_offsets(qs)
    mask = int(offs[-1])
    F = np.zeros((1 << n, 1 << n), dtype=complex)
    loc = {int(o): l for l, o in enumerate(offs)}
    for i in range(1 << n):
        for j in range(1 << n):
            if i & ~mask == j & ~mask:
                F[i, j] = U[loc[i & mask], loc[j & mask]]
    v = W.random_state(g, n)
    assert np.max(np.abs(O.apply_dense(v.copy(), n, qs, U) - F @ v)) < 1e-14
    assert abs(np.linalg.norm(O.apply_dense(v.copy(), n, qs, U)) - 1.0) < 1e-13


@pytest.mark.parametrize("q0,k", [(0, 3), (2, 2), (3, 3), (1, 5)])
def test_contiguous_block_is_kron_with_identities(q0, k):
    # qubit 0 is the least significant bit, so the operator on the
    # contiguous qubits q0 .. q0+k-1 is I (x) U (x) I with U in the middle
    n = 7
    g = W.rng(20 + q0 + k)
    U = unitary(g, 1 << k)
    F = np.kron(np.eye(1 << (n - q0 - k)), np.kron(U, np.eye(1 << q0)))
    v = W.random_state(g, n)
    got = O.apply_dense(v.copy(), n, list(range(q0, q0 + k)), U)
    assert np.max(np.abs(got - F @ v)) < 1e-14
