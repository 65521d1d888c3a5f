"""GPU parity of the dense k-qubit block against the oracle, through the C
ABI: the CUDA-core kernel for k = 1..6 (both dtypes), the tensor-core
kernel (complex64, k = 5) on contiguous and scattered qubits, full and
partial 128-group tiles, and agreement with TwoOpA."""
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


def unitary(g, d):
    A = g.standard_normal((d, d)) + 1j * g.standard_normal((d, d))
    Q, _ = np.linalg.qr(A)
    return Q


def run(qc, n, dt, qubits, U, seed):
    s = qc.State(n, dt)
    v = W.random_state(W.rng(seed), n)
    s.load(v)
    x = v.astype(np.complex64).astype(np.complex128) if dt == 1 else v.copy()
    qc.qc_apply_dense(s.h, qubits, U)
    got = s.numpy()
    ref = O.apply_dense(x, n, list(qubits), U)
    return np.max(np.abs(got - ref))


@pytest.mark.parametrize("n,qubits", [(12, [0, 1, 2, 3, 4]), (14, [0, 1, 2, 3, 4]), (11, [0, 1, 2, 3, 4]),
                                      (22, [0, 1, 2, 3, 4]), (13, [7, 2, 11, 0, 5]),
                                      (9, [4, 0, 8, 2, 6]), (5, [0, 1, 2, 3, 4]), (16, [15, 3, 9, 1, 12])])
def test_tensor_core_block_c64(qc, n, qubits):
    U = unitary(W.rng(n + sum(qubits)), 32)
    assert run(qc, n, 1, qubits, U, seed=n) <= 1e-5


@pytest.mark.parametrize("qubits", [[0, 1, 2, 3, 4], [5, 6, 7, 8, 9], [19, 3, 14, 9, 11]])
def test_tensor_core_block_c64_relative_accuracy(qc, qubits):
    # The bf16 digit slices keep a block at FP32-class accuracy relative to
    # the state (not to 1e-5 absolute, which a single bf16 or TF32 product
    # would also meet at small n): every output is rounded once from sums
    # that are exact or 2^-8 below the result, so the error is a few 2^-25
    # of the row scale and has no sign preference.  The fitted scale
    # <ref, got>/<ref, ref> - 1 then averages 2^20 independent errors; a
    # truncating accumulation (what FP32 sums on the tensor cores do) would
    # show here as a uniform shrink of about 1e-7 per chained product.
    n = 20
    U = unitary(W.rng(900 + sum(qubits)), 32)
    s = qc.State(n, 1)
    v = W.random_state(W.rng(901), n)
    s.load(v)
    x = v.astype(np.complex64).astype(np.complex128)
    qc.qc_apply_dense(s.h, qubits, U)
    got = s.numpy().astype(np.complex128)
    ref = O.apply_dense(x, n, list(qubits), U)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1.5e-7
    scale = np.vdot(ref, got) / np.vdot(ref, ref) - 1
    assert abs(scale) <= 2e-8


def test_tensor_core_block_chain_keeps_the_norm(qc):
    # 200 blocks in a row on one state: without a bias the norm drifts like a
    # random walk of ~2^-25 steps, far below 1e-5
    n = 16
    s = qc.State(n, 1)
    s.load(W.random_state(W.rng(77), n))
    g = W.rng(78)
    for i in range(200):
        qs = [int(q) for q in g.permutation(n)[:5]]
        qc.qc_apply_dense(s.h, qs, unitary(g, 32))
    assert abs(s.norm() - 1.0) <= 1e-5


def test_tensor_core_wait_timeout_selftest(qc):
    # the bounded mbarrier wait runs out (no MMA issued, nothing asynchronous
    # in flight): the call reports QC_ETIMEOUT, the state is untouched and
    # the next block on the same stream is correct
    n = 12
    s = qc.State(n, 1)
    v = W.random_state(W.rng(3), n)
    s.load(v)
    before = s.numpy()
    assert qc.qc_dense_timeout_selftest(s.h, 1024) == qc.QC_ETIMEOUT
    assert "timed out" in qc.last_error()
    assert np.array_equal(s.numpy(), before)
    U = unitary(W.rng(4), 32)
    qc.qc_apply_dense(s.h, [0, 1, 2, 3, 4], U)
    ref = O.apply_dense(before.astype(np.complex128), n, [0, 1, 2, 3, 4], U)
    assert np.max(np.abs(s.numpy() - ref)) <= 1e-6
    with pytest.raises(qc.QCError):  # the limit is validated
        qc._check(qc.qc_dense_timeout_selftest(s.h, 0))


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_cuda_core_block(qc, dt, k):
    if dt == 1 and k == 5:
        pytest.skip("complex64 k = 5 runs on the tensor cores (tested above)")
    n = 11
    g = W.rng(100 + k)
    qubits = [int(x) for x in g.permutation(n)[:k]]
    U = unitary(g, 1 << k)
    tol = 1e-12 if dt == 0 else 1e-5
    assert run(qc, n, dt, qubits, U, seed=k) <= tol


@pytest.mark.parametrize("dt", [0, 1])
def test_k2_equals_twoopa(qc, dt):
    n = 8
    V = unitary(W.rng(5), 4)
    a = qc.State(n, dt)
    b = qc.State(n, dt)
    v = W.random_state(W.rng(6), n)
    a.load(v)
    b.load(v)
    qc.qc_apply_dense(a.h, [1, 6], V)
    qc.qc_apply_2q(b.h, 6, 1, V)
    assert np.max(np.abs(a.numpy() - b.numpy())) <= (1e-13 if dt == 0 else 2e-6)


def test_dense_invalid(qc):
    s = qc.State(6, 0)
    with pytest.raises(qc.QCError):
        qc.qc_apply_dense(s.h, [1, 1], np.eye(4, dtype=complex))
    with pytest.raises(qc.QCError):
        qc.qc_apply_dense(s.h, [6], np.eye(2, dtype=complex))
    with pytest.raises(qc.QCError):
        qc.qc_apply_dense(s.h, [0, 1, 2, 3, 4, 5, 0], np.eye(128, dtype=complex))  # k = 7 > 6
