"""GPU parity of the tile passes that are compiled per group size, through
the C ABI, against the oracle: the QFT (Appendix A) and HALL (Eq. HALL) at
every state size whose plan gives a group size with its own instantiation.

Plans: the complex128 QFT takes a lowest group of 12 qubits and groups of
at most 9 above it (k_qft_c128_k<K>, K in {3..9, 12}); the complex64 QFT a
lowest group of 13 and groups of at most 9 (k_qft_db_c64_k<K>, K in
{3..9, 13}); HALL a lowest group of 12 (13) qubits and groups of at most 10
above it (k_wht_c128_top<L>, L in {3..10, 12}; k_wht_c64_top<L>, L in
{4..10, 13}).  For n up to 22 a single group sits above the lowest one, so
n - 12 (n - 13) is the group size, and the sizes below cover every
instantiation; the other sizes take the general kernels, also compared."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def qc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0902_0699_gb300 as q
    q.lib()
    return q


def as_dt(v, dt):
    return v.astype(np.complex64).astype(np.complex128) if dt == 1 else v


# complex128: 12 + K for K = 1..10 (1, 2 and 10 take the general QFT kernel);
# complex64: 13 + K for K = 1..9
QFT_N = {0: [13, 14, 15, 16, 17, 18, 19, 20, 21, 22], 1: [14, 15, 16, 17, 18, 19, 20, 21, 22]}


@pytest.mark.parametrize("dt,n", [(dt, n) for dt in (0, 1) for n in QFT_N[dt]])
def test_qft_every_compiled_group_size(qc, dt, n):
    v = as_dt(W.random_state(W.rng(700 + n), n), dt)
    s = qc.State(n, dt)
    s.load(v)
    s.qft()
    ref = O.qft(v.copy(), n)
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt] * max(1, n / 4)
    s.close()


# HALL on a random state: 12 + L (complex128) and 13 + L (complex64)
HALL_N = {0: [14, 15, 16, 17, 18, 19, 20, 21, 22], 1: [16, 17, 18, 19, 20, 21, 22, 23]}


@pytest.mark.parametrize("dt,n", [(dt, n) for dt in (0, 1) for n in HALL_N[dt]])
def test_hall_every_compiled_group_size(qc, dt, n):
    v = as_dt(W.random_state(W.rng(800 + n), n), dt)
    s = qc.State(n, dt)
    s.load(v)
    s.hall()
    ref = v.copy()
    for q in range(n):
        O.apply_1q(ref, n, q, O.H_MAT)
    assert np.max(np.abs(s.numpy() - ref)) <= (1e-13 if dt == 0 else 1e-5)
    s.close()
