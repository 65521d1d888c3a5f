"""GPU parity of TwoOpA and of the Shor steps (state preparation, ProjA,
register QFT) against the CPU oracle, through the C ABI."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

from test_oracle_shor import period, probshor, sizes

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def qc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0902_0699_gb300 as q
    q.lib()
    return q


def unitary4(seed):
    g = np.random.default_rng(seed)
    A = g.standard_normal((4, 4)) + 1j * g.standard_normal((4, 4))
    Q, _ = np.linalg.qr(A)
    return Q


@pytest.mark.parametrize("dt", [0, 1])
def test_apply_2q_all_pairs(qc, dt):
    n = 6
    s = qc.State(n, dt)
    v = W.random_state(W.rng(1), n)
    s.load(v)
    ref = v.astype(np.complex64).astype(np.complex128) if dt else v.copy()
    k = 0
    for t1 in range(n):
        for t2 in range(n):
            if t1 == t2:
                continue
            V = unitary4(k)
            k += 1
            qc.qc_apply_2q(s.h, t1, t2, V)
            O.apply_2q(ref, n, t1, t2, V)
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt] * 10


@pytest.mark.parametrize("dt", [0, 1])
def test_apply_2q_large(qc, dt):
    n = 19
    s = qc.State(n, dt)
    v = W.random_state(W.rng(2), n)
    s.load(v)
    ref = v.astype(np.complex64).astype(np.complex128) if dt else v.copy()
    for (t1, t2) in ((0, 18), (17, 3), (9, 10)):
        V = unitary4(t1 * 31 + t2)
        qc.qc_apply_2q(s.h, t1, t2, V)
        O.apply_2q(ref, n, t1, t2, V)
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt] * 4


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("M,x", [(15, 7), (21, 2), (33, 5)])
def test_shor_steps_vs_oracle_and_probshor(qc, dt, M, x):
    n1, n2 = sizes(M)
    n = n1 + n2
    s = qc.State(n, dt)
    qc.qc_shor_prepare(s.h, n2, x, M)
    ref = O.shor_prepare(n, n2, x, M)
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt]
    k = x % M
    pk = qc.qc_project(s.h, 0, n2, k)
    pr = O.project(ref, n, 0, n2, k)
    assert abs(pk - pr) <= 1e-12 if dt == 0 else abs(pk - pr) <= 1e-6
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt]
    qc.qc_qft_range(s.h, n2, n1)
    O.qft_range(ref, n, n2, n1)
    got = s.numpy()
    assert np.max(np.abs(got - ref)) <= TOL[dt] * 4
    # Eq. probshor on the GPU's own probabilities
    D = sum(1 for j in range(2 ** n1) if pow(x, j, M) == k)
    p = s.probs().cpu().numpy().reshape(2 ** n1, 2 ** n2)[:, k]
    assert np.max(np.abs(p - probshor(n1, D, period(x, M)))) <= (1e-12 if dt == 0 else 1e-5)


def test_shor_invalid(qc):
    s = qc.State(8, 0)
    with pytest.raises(qc.QCError):
        qc.qc_shor_prepare(s.h, 4, 7, 17)  # M > 2^n2
    with pytest.raises(qc.QCError):
        qc.qc_project(s.h, 6, 3, 0)  # register beyond n
    with pytest.raises(qc.QCError):
        qc.qc_apply_2q(s.h, 2, 2, np.eye(4, dtype=complex))


@pytest.mark.parametrize("dt", [0, 1])
def test_shor_smallest_modulus(qc, dt):
    # M = 3, x = 2 (period 2): n1 = 4, n2 = 2
    M, x = 3, 2
    n1, n2 = sizes(M)
    n = n1 + n2
    s = qc.State(n, dt)
    qc.qc_shor_prepare(s.h, n2, x, M)
    ref = O.shor_prepare(n, n2, x, M)
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt]
    pk = qc.qc_project(s.h, 0, n2, 1)
    assert abs(pk - O.project(ref, n, 0, n2, 1)) <= (1e-12 if dt == 0 else 1e-6)
    qc.qc_qft_range(s.h, n2, n1)
    O.qft_range(ref, n, n2, n1)
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt] * 4
