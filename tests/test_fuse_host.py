"""Host logic of gate fusion (plan creation only; no device call): block
counts for circuits whose grouping is fixed by the rules, and argument
checks."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def qc():
    import paper_0902_0699_gb300 as q
    q.lib()
    return q


def test_disjoint_one_qubit_gates_fill_blocks(qc):
    ops = [(1, q, 0, 0, np.eye(2)) for q in range(10)]
    assert qc.FusedPlan(10, ops, kmax=5, pad=False).info() == (2, 5)
    assert qc.FusedPlan(10, ops, kmax=2, pad=False).info() == (5, 2)


def test_dependency_keeps_order(qc):
    # CNOT(0,1), then a gate on qubit 1 and on qubit 7: with kmax = 2 the
    # first block is {0,1} (CNOT + the qubit-1 gate), the qubit-7 gate needs
    # a second block; a later CNOT(1,7) waits for both
    ops = [(2, 0, 1, 0, None), (1, 1, 0, 0, np.eye(2)), (1, 7, 0, 0, np.eye(2)), (2, 1, 7, 0, None)]
    nb, _ = qc.FusedPlan(8, ops, kmax=2, pad=False).info()
    assert nb == 2  # {0,1}: ops 0,1; {7,1}: ops 2,3


def test_plan_rejects_bad_operators(qc):
    with pytest.raises(qc.QCError):
        qc.FusedPlan(4, [(9, 0, 1, 0, None)])
    with pytest.raises(qc.QCError):
        qc.FusedPlan(4, [(3, 0, 1, 0, None)])  # CPHASE needs k >= 1


def test_plan_blocks_are_unitary_and_bounded(qc):
    import workloads as W
    n, layers = 10, 6
    circ = W.random_circuit(n, layers, seed=24)
    ops = []
    for l in range(layers):
        for q in range(n):
            ops.append((1, q, 0, 0, circ.U[l, q]))
        for (c, t) in circ.cnot_pairs(l):
            ops.append((2, c, t, 0, None))
    p = qc.FusedPlan(n, ops, kmax=5, pad=True)
    nb, km = p.info()
    for i in range(nb):
        qs, U = p.block(i)
        assert len(qs) == 5 and len(set(qs)) == 5 and all(0 <= q < n for q in qs)
        assert np.max(np.abs(U @ U.conj().T - np.eye(32))) < 1e-13
