"""GPU parity of the Hadamard-layer passes (HALL, Eq. HALL, and layers made
of Hadamards only), through the C ABI: complex128 in exact 64-bit fixed
point with one rounding in and one out, complex64 in FP32.  Against the
oracle's n separate OneOpA calls, on subsets of qubits (odd and even counts
per tile group, only low or only high qubits), plus exact properties: HALL
of |0..0> is exactly uniform for even n, HALL^2 = I, and a wide dynamic
range inside one tile keeps its absolute accuracy."""
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


H = O.H_MAT
TOL = {0: 1e-13, 1: 1e-5}  # complex128: the fixed-point passes round once in, once out


def layer_ref(v, n, mask):
    ref = v.copy()
    for q in range(n):
        if (mask >> q) & 1:
            O.apply_1q(ref, n, q, H)
    return ref


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [12, 13, 16, 21, 24])
def test_hadamard_layers_vs_oracle(qc, dt, n):
    g = W.rng(300 + n)
    v = W.random_state(g, n)
    x = v.astype(np.complex64).astype(np.complex128) if dt == 1 else v
    full = (1 << n) - 1
    masks = [full, full & ~(1 << (n // 2)), (1 << 5) - 1, full ^ ((1 << (n - 3)) - 1), 1 << (n - 1),
             int(g.integers(1, 1 << n))]
    for mask in masks:
        s = qc.State(n, dt)
        s.load(x)
        Us = np.stack([H] * n)
        s.apply_1q_layer(Us, mask)
        assert np.max(np.abs(s.numpy() - layer_ref(x, n, mask))) <= TOL[dt], hex(mask)
        s.close()


@pytest.mark.parametrize("n", [12, 20, 26])
def test_hall_of_zero_state_is_exactly_uniform(qc, n):
    s = qc.State(n, 0).reset(0)
    s.hall()
    got = s.numpy()
    assert np.all(got == complex(2.0 ** (-n / 2), 0.0))
    s.close()


@pytest.mark.parametrize("dt", [0, 1])
def test_hall_twice_is_identity(qc, dt):
    n = 20
    v = W.random_state(W.rng(9), n)
    s = qc.State(n, dt)
    s.load(v)
    before = s.numpy()
    s.hall()
    s.hall()
    assert np.max(np.abs(s.numpy() - before)) <= (2e-16 if dt == 0 else 2e-6)
    s.close()


def test_hall_wide_dynamic_range_c128(qc):
    # one amplitude near 1 and the rest spread over 1e-3 .. 1e-13 in every
    # tile: the fixed point is set by each tile's largest magnitude, so the
    # small ones keep an absolute accuracy of 2^-51 of it
    n = 16
    g = W.rng(11)
    v = (g.standard_normal(1 << n) + 1j * g.standard_normal(1 << n)) * 10.0 ** g.uniform(-13, -3, 1 << n)
    v[12345] = 0.9
    s = qc.State(n, 0)
    s.load(v)
    s.hall()
    assert np.max(np.abs(s.numpy() - layer_ref(v, n, (1 << n) - 1))) <= 1e-15
    s.close()
