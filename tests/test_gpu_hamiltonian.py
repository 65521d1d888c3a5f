"""GPU parity of the first-order Hamiltonian step (sec. 7) against the
oracle through the C ABI, for one- and two-body terms on neighbouring and
scattered qubits, both dtypes, and its argument checks."""
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


def herm(g, d):
    A = g.standard_normal((d, d)) + 1j * g.standard_normal((d, d))
    return (A + A.conj().T) / 2


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [2, 10, 15])
def test_step_vs_oracle(qc, dt, n):
    g = W.rng(n + 40 * dt)
    terms = [([q], herm(g, 2)) for q in range(n)]
    terms += [([q, (q + 1) % n], herm(g, 4)) for q in range(n - 1)]
    terms += [([int(a), int(b)], herm(g, 4)) for a, b in [g.permutation(n)[:2] for _ in range(3)]]
    s = qc.State(n, dt)
    v = W.random_state(g, n)
    s.load(v)
    x = v.astype(np.complex64).astype(np.complex128) if dt == 1 else v.copy()
    for step_dt in (0.01, 0.02):
        qc.qc_hamiltonian_step(s.h, step_dt, terms)
        O.hamiltonian_step(x, n, step_dt, terms)
    assert np.max(np.abs(s.numpy() - x)) <= (1e-12 if dt == 0 else 2e-5)


def test_hamiltonian_invalid(qc):
    s = qc.State(4, 0)
    with pytest.raises(qc.QCError):
        qc.qc_hamiltonian_step(s.h, 0.1, [([0, 0], np.eye(4))])
    with pytest.raises(qc.QCError):
        qc.qc_hamiltonian_step(s.h, 0.1, [([4], np.eye(2))])
    with pytest.raises(qc.QCError):
        qc.qc_hamiltonian_step(s.h, float("nan"), [([1], np.eye(2))])
