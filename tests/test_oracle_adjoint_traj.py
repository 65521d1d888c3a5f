"""Pins of the oracle's adjoint gradient (finite differences, the
parameter-shift rule, dense brute force) and of its noisy-trajectory replay
(the noiseless closed form, a dense-matrix replay of the literal gate list,
and enumeration of read-out flip patterns).  No GPU."""
import itertools
import math

import numpy as np

import oracle as O
import workloads as W

from test_oracle_gates import grover_closed_form


def small_ansatz(n=4, layers=3, seed=2):
    return W.ansatz(n, layers, seed)[0]


def test_forward_vs_dense():
    c = small_ansatz()
    n = c.n
    M = np.eye(1 << n, dtype=np.complex128)
    for g in O.ansatz_gates(c):
        if g[0] == "cnot":
            CN = np.zeros((1 << n, 1 << n))
            for i in range(1 << n):
                j = i ^ (1 << g[2]) if (i >> g[1]) & 1 else i
                CN[j, i] = 1
            M = CN @ M
        else:
            U = O.ry(c.theta[g[2]]) if g[0] == "ry" else O.rz(c.theta[g[2]])
            Mq = np.eye(1)
            for q in range(n - 1, -1, -1):
                Mq = np.kron(Mq, U if q == g[1] else np.eye(2))
            M = Mq @ M
    psi = O.ansatz_forward(c)
    assert np.max(np.abs(psi - M[:, 0])) < 1e-13


def test_adjoint_vs_param_shift_and_fd():
    c = small_ansatz(n=5, layers=4, seed=3)
    terms = W.ansatz_hamiltonian(c.n)
    E, g = O.adjoint_gradient(c, terms)
    assert abs(E - O.energy(O.ansatz_forward(c), c.n, terms)) < 1e-14
    th = c.theta
    for k in range(c.n_params):
        tp, tm = th.copy(), th.copy()
        tp[k] += math.pi / 2
        tm[k] -= math.pi / 2
        ps = 0.5 * (O.energy(O.ansatz_forward(c, tp), c.n, terms)
                    - O.energy(O.ansatz_forward(c, tm), c.n, terms))
        assert abs(g[k] - ps) < 1e-12
        h = 1e-4
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (O.energy(O.ansatz_forward(c, tp), c.n, terms)
              - O.energy(O.ansatz_forward(c, tm), c.n, terms)) / (2 * h)
        assert abs(g[k] - fd) < 1e-8  # O(h^2) truncation


def test_trajectory_noiseless_is_grover():
    for n, m in ((5, 3), (8, 200)):
        it = W.grover_iterations(n)
        psi, errs = O.trajectory_run(n, m, it, seed=1, inst=0, thr_gate=0)
        assert errs == 0
        assert np.max(np.abs(psi - grover_closed_form(n, [m], it))) < 1e-12


def _dense(n, U, q):
    M = np.eye(1)
    for b in range(n - 1, -1, -1):
        M = np.kron(M, U if b == q else np.eye(2))
    return M


def test_trajectory_dense_replay():
    # every location's Philox draw decides its Pauli independently of the
    # replay; rebuild the literal gate product densely and compare
    n, marked, iters, seed, inst = 3, 5, 2, 99, 7
    thr = W.prob_threshold(0.35)
    psi, errs = O.trajectory_run(n, marked, iters, seed, inst, thr)
    P = {1: O.X_MAT, 2: O.Y_MAT, 3: O.Z_MAT}
    N = 1 << n
    v = np.zeros(N, dtype=np.complex128)
    v[0] = 1
    count = 0

    def noise(stage, q):
        nonlocal v, count
        e = O.noise_draw(seed, inst, stage, q, thr)
        if e:
            v = _dense(n, P[e], q) @ v
            count += 1

    def hall(stage):
        nonlocal v
        for q in range(n):
            v = _dense(n, O.H_MAT, q) @ v
            noise(stage, q)

    orac = np.eye(N)
    orac[marked, marked] = -1
    invm = -np.eye(N)
    invm[0, 0] = 1
    hall(0)
    for r in range(iters):
        s = 1 + 4 * r
        v = orac @ v
        for q in range(n):
            noise(s, q)
        hall(s + 1)
        v = invm @ v
        for q in range(n):
            noise(s + 2, q)
        hall(s + 3)
    assert count == errs and errs > 0
    assert np.max(np.abs(psi - v)) < 1e-13


def test_noise_draw_rate():
    thr = W.prob_threshold(0.1)
    hits = sum(1 for s in range(200) for q in range(50) if O.noise_draw(3, 1, s, q, thr))
    assert abs(hits / 10000 - 0.1) < 0.015


def test_readout_success_enumeration():
    n, marked, pr = 3, 6, 0.2
    x = W.random_state(W.rng(1), n)
    p = O.probs(x, n)
    tot = 0.0
    for j in range(1 << n):
        for flips in itertools.product([0, 1], repeat=n):
            f = sum(b << i for i, b in enumerate(flips))
            w = np.prod([pr if b else 1 - pr for b in flips])
            if j ^ f == marked:
                tot += p[j] * w
    assert abs(O.readout_success(p, n, marked, pr) - tot) < 1e-15


def test_readout_weights_c64_exact():
    # trunc(re^2 2^62) + trunc(im^2 2^62) of float32 parts, against exact
    # rational arithmetic (Fraction) on random, tiny and edge values
    from fractions import Fraction
    g = np.random.default_rng(3)
    re = np.concatenate([g.standard_normal(300) * 0.01, [0.0, -0.0, 1.0, -0.5, 2.0 ** -40, 3e-30, 1.0 - 2 ** -24]])
    im = np.concatenate([g.standard_normal(300) * 0.003, [1.0, 0.25, 0.0, -0.75, 2.0 ** -31, 1e-20, 2 ** -12]])
    psi = (re + 1j * im).astype(np.complex64)
    w = O.readout_weights_c64(psi)
    for j in range(len(psi)):
        r, i = Fraction(float(psi[j].real)), Fraction(float(psi[j].imag))
        ref = int(r * r * 2 ** 62) + int(i * i * 2 ** 62)  # int() truncates toward zero
        assert int(w[j]) == ref


def test_measure_from_weights_matches_probability_rule():
    # the weight form of the read-out equals the probability form when the
    # weights are trunc(p 2^62), and a weight moved across the target's
    # boundary moves the outcome (the replay is sensitive to the weights)
    g = np.random.default_rng(4)
    n = 9
    p = g.random(1 << n)
    p /= p.sum()
    for inst in range(20):
        a = O.trajectory_measure(p, n, 77, inst, 0)
        b = O.trajectory_measure_weights((p * O.TWO62).astype(np.uint64), n, 77, inst, 0)
        assert a == b
    w = (p * O.TWO62).astype(np.uint64)
    out = O.trajectory_measure_weights(w, n, 77, 0, 0)
    w2 = w.copy()
    w2[out] = 0  # nothing left at the drawn outcome: the draw must land elsewhere
    assert O.trajectory_measure_weights(w2, n, 77, 0, 0) != out
