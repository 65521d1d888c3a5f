"""GPU parity of gate fusion (qc_fused_plan_*) against the oracle's literal
gate-by-gate application: random circuits (the 24-qubit workload's
structure on fewer qubits) and mixed operator kinds, block sizes 2..6,
padded (complex64 5-qubit blocks on the tensor cores) and unpadded."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0902_0699_gb300 as q
    q.lib()
    return q


def circuit_ops(circ):
    ops = []
    for l in range(circ.layers):
        for q in range(circ.n):
            ops.append((1, q, 0, 0, circ.U[l, q]))
        for (c, t) in circ.cnot_pairs(l):
            ops.append((2, c, t, 0, None))
    return ops


def mixed_ops(n, count, seed):
    g = W.rng(seed)
    us = W.haar_u2(g, count)
    ops = []
    for i in range(count):
        kind = int(g.integers(1, 6))
        a, b = (int(x) for x in g.permutation(n)[:2])
        ops.append((kind, a, b, int(g.integers(1, 6)), us[i] if kind in (1, 5) else None))
    return ops


def run(qc, n, dt, ops, kmax, pad, seed):
    v = W.random_state(W.rng(seed), n)
    s = qc.State(n, dt)
    s.load(v)
    plan = qc.FusedPlan(n, ops, kmax=kmax, pad=pad)
    plan.run(s.h)
    got = s.numpy()
    x = v.astype(np.complex64).astype(np.complex128) if dt == 1 else v.copy()
    ref = O.apply_ops(x, n, [(k, a, b, kk, None if U is None else np.asarray(U)) for (k, a, b, kk, U) in ops])
    nb, _ = plan.info()
    plan.close()
    return np.max(np.abs(got - ref)), nb


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("kmax,pad", [(5, True), (5, False), (3, False), (6, True), (2, False)])
def test_random_circuit_fused(qc, dt, kmax, pad):
    n = 11
    circ = W.random_circuit(n, 8, seed=24)
    ops = circuit_ops(circ)
    err, nb = run(qc, n, dt, ops, kmax, pad, seed=5)
    assert err <= (1e-12 if dt == 0 else 2e-5)
    assert nb < len(ops)  # fusion reduced the number of passes


@pytest.mark.parametrize("dt", [0, 1])
def test_mixed_kinds_fused(qc, dt):
    n = 9
    ops = mixed_ops(n, 120, seed=17)
    err, nb = run(qc, n, dt, ops, 5, True, seed=6)
    assert err <= (1e-12 if dt == 0 else 2e-5)


def test_large_state_tensor_core_blocks(qc):
    n = 16
    circ = W.random_circuit(n, 4, seed=3)
    err, nb = run(qc, n, 1, circuit_ops(circ), 5, True, seed=7)
    assert err <= 2e-5


def test_fuse_invalid(qc):
    with pytest.raises(qc.QCError):
        qc.FusedPlan(4, [(2, 1, 1, 0, None)])
    with pytest.raises(qc.QCError):
        qc.FusedPlan(4, [(1, 4, 0, 0, np.eye(2))])
    with pytest.raises(qc.QCError):
        qc.FusedPlan(4, [(1, 0, 0, 0, np.eye(2))], kmax=7)


@pytest.mark.parametrize("dt", [0, 1])
def test_fused_two_qubit_state(qc, dt):
    # the smallest circuit with two-qubit operators: blocks hold the whole state
    g = W.rng(4)
    u = W.haar_u2(g, 3)
    ops = [(1, 0, 0, 0, u[0]), (2, 0, 1, 0, None), (1, 1, 0, 0, u[1]), (3, 1, 0, 3, None),
           (4, 0, 1, 0, None), (5, 1, 0, 0, u[2])]
    for kmax in (2, 5):
        err, nb = run(qc, 2, dt, ops, kmax, True, seed=9)
        assert err <= (1e-13 if dt == 0 else 2e-6)
        assert nb == 1
