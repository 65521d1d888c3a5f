"""Pins of the CPU oracle's gate routines against dense linear algebra, the
paper's worked examples and textbook identities (no GPU)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle as O
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rand_state(n, seed):
    return W.random_state(W.rng(seed), n)


def tensor_apply(psi, n, op, qubits):
    """Apply a 2^k x 2^k operator on bit positions `qubits` (first = most
    significant within the operator's own index) by reshaping the state into
    an n-way tensor whose axis a holds bit n-1-a.  An independent formulation
    of sec. 3 / sec. 4 (tensor contraction instead of pair loops)."""
    k = len(qubits)
    T = psi.reshape([2] * n)
    axes = [n - 1 - q for q in qubits]
    opT = op.reshape([2] * (2 * k))
    out = np.tensordot(opT, T, axes=(list(range(k, 2 * k)), axes))
    out = np.moveaxis(out, list(range(k)), axes)
    return out.reshape(-1)


def kron_1q(n, t, U):
    """Full 2^n matrix of a one-qubit operator on bit t, built as the tensor
    product I x .. x U x .. x I with the paper's q_1 (MSB) leftmost."""
    M = np.eye(1)
    for q in range(n - 1, -1, -1):
        M = np.kron(M, U if q == t else np.eye(2))
    return M


def test_1q_vs_kron_all_t():
    g = W.rng(1)
    for n in range(1, 7):
        for t in range(n):
            U = W.haar_u2(g, 1)[0]
            Uc = U[0::2] + 1j * U[1::2]
            psi = rand_state(n, 100 * n + t)
            ref = kron_1q(n, t, Uc.reshape(2, 2)) @ psi
            got = O.apply_1q(psi.copy(), n, t, U)
            assert np.max(np.abs(got - ref)) < 1e-14


def test_1q_transposed_matrix_fails():
    # a plausible mistake (U transposed) must be caught by the kron pin
    n, t = 3, 1
    U = W.haar_u2(W.rng(5), 1)[0]
    Uc = (U[0::2] + 1j * U[1::2]).reshape(2, 2)
    psi = rand_state(n, 7)
    ref = kron_1q(n, t, Uc.T) @ psi
    got = O.apply_1q(psi.copy(), n, t, U)
    assert np.max(np.abs(got - ref)) > 1e-3


def test_paper_partner_examples():
    ex = json.load(open(os.path.join(GOLD, "paper_partner_examples.json")))
    X = O.X_MAT
    for e in ex["one_qubit"]:
        n = e["n_q"]
        t = n - e["i_s"]
        pairs = e.get("all_pairs", [e.get("partners")])
        for a, b in pairs:
            psi = O.zero_state(n, a)
            O.apply_1q(psi, n, t, X)
            assert abs(psi[b] - 1) == 0 and np.count_nonzero(psi) == 1
    for e in ex["two_qubit"]:
        n = e["n_q"]
        t1, t2 = n - e["i_s1"], n - e["i_s2"]
        quartet = e["quartet"]
        # a 4x4 cyclic shift moves quartet position a to a+1 (mod 4)
        V = np.roll(np.eye(4), 1, axis=0).astype(np.complex128)
        for pos, idx in enumerate(quartet):
            psi = O.zero_state(n, idx)
            O.apply_2q(psi, n, t1, t2, V)
            assert psi[quartet[(pos + 1) % 4]] == 1 and np.count_nonzero(psi) == 1


def test_2q_vs_tensor():
    g = W.rng(3)
    for n in (2, 3, 5):
        for t1 in range(n):
            for t2 in range(n):
                if t1 == t2:
                    continue
                A = g.standard_normal((4, 4)) + 1j * g.standard_normal((4, 4))
                V, _ = np.linalg.qr(A)
                psi = rand_state(n, 31 * t1 + t2 + n)
                ref = tensor_apply(psi, n, V, [t1, t2])
                got = O.apply_2q(psi.copy(), n, t1, t2, V)
                assert np.max(np.abs(got - ref)) < 1e-13


def test_ctrl_cnot_cphase_vs_tensor():
    g = W.rng(4)
    n = 5
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            U = W.haar_u2(g, 1)[0]
            Uc = (U[0::2] + 1j * U[1::2]).reshape(2, 2)
            CU = np.eye(4, dtype=np.complex128)
            CU[2:, 2:] = Uc
            psi = rand_state(n, 7 * c + t)
            assert np.max(np.abs(O.apply_ctrl(psi.copy(), n, c, t, U)
                                 - tensor_apply(psi, n, CU, [c, t]))) < 1e-14
            CN = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
            got = O.cnot(psi.copy(), n, c, t)
            assert np.array_equal(got, tensor_apply(psi, n, CN, [c, t]))  # a permutation: exact
            for k in (1, 2, 3, 5):
                D = np.diag([1, 1, 1, np.exp(2j * np.pi / 2 ** k)])
                assert np.max(np.abs(O.cphase(psi.copy(), n, c, t, k)
                                     - tensor_apply(psi, n, D, [c, t]))) < 1e-15


def test_cphase_identities():
    n = 4
    psi = rand_state(n, 9)
    a = O.cphase(psi.copy(), n, 1, 3, 1)
    b = O.apply_2q(psi.copy(), n, 1, 3, np.diag([1, 1, 1, -1]).astype(np.complex128))
    assert np.array_equal(a, b)  # CPHASEK(k=1) is CPHASEA exactly
    for k in (1, 2, 3, 4):
        x = psi.copy()
        for _ in range(2 ** k):
            O.cphase(x, n, 0, 2, k)
        assert np.max(np.abs(x - psi)) < 1e-14
    assert O.cphase_factor(1) == -1 and O.cphase_factor(2) == 1j


def test_swap_is_bit_permutation():
    n = 5
    psi = rand_state(n, 11)
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            got = O.swap(psi.copy(), n, a, b)
            idx = np.arange(1 << n)
            ba, bb = (idx >> a) & 1, (idx >> b) & 1
            src = idx ^ ((ba ^ bb) << a) ^ ((ba ^ bb) << b)
            assert np.array_equal(got, psi[src])


def test_hall_uniform_and_involution():
    for n in (1, 2, 4, 6, 10):
        psi = O.zero_state(n)
        O.hall(psi, n)
        assert np.max(np.abs(psi - 2.0 ** (-n / 2))) < 1e-15
        x = rand_state(n, n)
        y = O.hall(O.hall(x.copy(), n), n)
        assert np.max(np.abs(x - y)) < 1e-14


def test_hall_vs_hall2_and_scipy_hadamard():
    for n in (1, 3, 6, 9):
        x = rand_state(n, 50 + n)
        a = O.hall(x.copy(), n)
        b = O.hall2(x, n)  # the paper's sign rule s_{n,n'} (sec. 4.3)
        Hs = scipy.linalg.hadamard(1 << n) / 2 ** (n / 2)  # Sylvester ordering
        c = Hs @ x
        assert np.max(np.abs(a - b)) < 1e-13
        assert np.max(np.abs(a - c)) < 1e-13


def grover_closed_form(n, marked, k):
    N, M = 2 ** n, len(marked)
    th = math.asin(math.sqrt(M / N))
    a = math.sin((2 * k + 1) * th) / math.sqrt(M)
    b = math.cos((2 * k + 1) * th) / math.sqrt(N - M) if N > M else 0.0
    v = np.full(N, b, dtype=np.complex128)
    v[np.asarray(marked, dtype=np.int64)] = a
    return v


@pytest.mark.parametrize("n,M,k", [(3, 1, 1), (6, 1, 6), (8, 3, 5), (10, 1, 25), (9, 8, 4), (7, 2, 13)])
def test_grover_closed_form(n, M, k):
    marked = W.marked_indices(W.rng(n * 100 + M), n, M)
    psi = O.grover_run(n, marked, k)
    ref = grover_closed_form(n, marked, k)
    assert np.max(np.abs(psi - ref)) < 1e-12


def test_grover_c1_success():
    # 10 qubits, one marked item, 25 iterations: sin^2(51 asin(2^-5))
    psi = O.grover_run(10, [123], W.grover_iterations(10))
    assert W.grover_iterations(10) == 25
    ps = abs(psi[123]) ** 2
    assert abs(ps - math.sin(51 * math.asin(2 ** -5)) ** 2) < 1e-13
    assert abs(ps - 0.99946) < 1e-5


def test_qft_basis_states_analytic():
    for n in (1, 2, 3, 5, 7):
        N = 2 ** n
        for m in range(0, N, max(1, N // 7)):
            psi = O.qft(O.zero_state(n, m), n)
            ref = np.exp(2j * np.pi * m * np.arange(N) / N) / math.sqrt(N)
            assert np.max(np.abs(psi - ref)) < 1e-13


def test_qft_vs_numpy_ifft_and_dense():
    for n in (4, 8, 12):
        x = rand_state(n, 70 + n)
        got = O.qft(x.copy(), n)
        ref = np.fft.ifft(x) * math.sqrt(2 ** n)  # +i sign, 1/sqrt(N)
        assert np.max(np.abs(got - ref)) < 1e-12
    n = 6
    N = 2 ** n
    F = np.exp(2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N) / math.sqrt(N)
    x = rand_state(n, 3)
    assert np.max(np.abs(O.qft(x.copy(), n) - F @ x)) < 1e-13


def test_qft_powers():
    n = 7
    N = 2 ** n
    x = rand_state(n, 8)
    y2 = O.qft(O.qft(x.copy(), n), n)
    assert np.max(np.abs(y2 - x[(-np.arange(N)) % N])) < 1e-13
    y4 = O.qft(O.qft(y2, n), n)
    assert np.max(np.abs(y4 - x)) < 1e-13


def test_probs_norm_expect():
    n = 6
    x = rand_state(n, 12) * 1.3
    p = O.probs(x, n)
    assert np.max(np.abs(p - np.abs(x) ** 2)) < 1e-16
    assert abs(O.norm(x, n) - np.sum(np.abs(x) ** 2)) < 1e-14
    # <Z0 Z1>, <X_3>, <Y_2 X_0>: against dense Kronecker Pauli strings
    Z, X, Y = O.Z_MAT, O.X_MAT, O.Y_MAT
    for xm, zm in [(0, 0b11), (0b1000, 0), (0b101, 0b100), (0b110, 0b011)]:
        M = np.eye(1)
        for q in range(n - 1, -1, -1):
            bx, bz = (xm >> q) & 1, (zm >> q) & 1
            M = np.kron(M, Y if (bx and bz) else X if bx else Z if bz else np.eye(2))
        ref = np.vdot(x, M @ x)
        assert abs(O.expect_pauli(x, n, xm, zm) - ref) < 1e-13
        assert np.max(np.abs(O.apply_pauli(x, n, xm, zm) - M @ x)) < 1e-15


def test_haar_u2_unitary():
    U = W.haar_u2(W.rng(0), 64)
    for u in U:
        m = (u[0::2] + 1j * u[1::2]).reshape(2, 2)
        assert np.max(np.abs(m @ m.conj().T - np.eye(2))) < 1e-14
