"""GPU parity of the noise intrusions and the ensemble density matrix
(sec. 6.1-6.3) against the oracle, through the C ABI: the Wigner
operators, rho element by element, and its spectrum, trace, purity and
entropy from the Gram route; then the paper's multiverse Grover scenario
(one D2 or D4 intrusion per noisy universe) run with the gate API."""
import numpy as np
import pytest

import oracle as O
import oracle.density as D
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-6}


@pytest.fixture(scope="module")
def qc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0902_0699_gb300 as q
    q.lib()
    return q


def batch(qc, states, dt):
    import torch
    t = torch.tensor(np.asarray(states), dtype=qc.torch_dtype(dt), device="cuda").contiguous()
    return t


def as_dt(x, dt):
    return x.astype(np.complex64).astype(np.complex128) if dt == 1 else x


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n,B", [(3, 1), (7, 5), (9, 19), (6, 70)])
def test_density_matrix_vs_oracle(qc, dt, n, B):
    import torch
    g = W.rng(n * 100 + B)
    states = np.stack([W.random_state(g, n) for _ in range(B)])
    P = g.random(B)
    P /= P.sum()
    t = batch(qc, states, dt)
    rho = torch.empty((1 << n) * (1 << n), dtype=t.dtype, device="cuda")
    qc.qc_density_matrix(t.data_ptr(), n, dt, B, P, rho.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = rho.cpu().numpy().astype(np.complex128).reshape(1 << n, 1 << n)
    ref = D.density_matrix(as_dt(states, dt), P)
    assert np.max(np.abs(got - ref)) <= TOL[dt]
    assert np.max(np.abs(got - got.conj().T)) <= TOL[dt]


@pytest.mark.parametrize("n,B", [(1, 1), (4, 2), (8, 33), (11, 64), (12, 7)])
def test_density_matrix_tensor_cores_c64(qc, n, B):
    # complex64 rho on the tensor cores: 128 x 32 tiles over K = 2B (one or
    # two 64-wide chunks, padded), bf16 digit slices with exact leading sums.
    # Against the oracle on the same complex64 inputs: FP32-class error
    # relative to the largest entry, Hermitian to that level, and a trace
    # with no drift (a truncating accumulation would shrink it)
    import torch
    g = W.rng(n * 31 + B)
    states = np.stack([W.random_state(g, n) for _ in range(B)])
    P = g.random(B)
    P /= P.sum()
    t = batch(qc, states, 1)
    N = 1 << n
    rho = torch.empty(N * N, dtype=torch.complex64, device="cuda")
    qc.qc_density_matrix(t.data_ptr(), n, 1, B, P, rho.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = rho.cpu().numpy().astype(np.complex128).reshape(N, N)
    ref = D.density_matrix(as_dt(states, 1), P)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 3e-7 * scale
    assert np.max(np.abs(got - got.conj().T)) <= 3e-7 * scale
    assert abs(np.trace(got).real - np.trace(ref).real) <= 1e-6


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n,B", [(1, 2), (6, 7), (10, 16), (12, 64)])
def test_mixed_spectrum_vs_oracle(qc, dt, n, B):
    g = W.rng(n * 7 + B)
    states = np.stack([W.random_state(g, n) for _ in range(B)])
    P = g.random(B)
    P /= P.sum()
    t = batch(qc, states, dt)
    ev, (tr, pur, ent) = qc.qc_mixed_spectrum(t.data_ptr(), n, dt, B, P)
    x = as_dt(states, dt)
    rho = D.density_matrix(x, P)
    ref = D.spectrum(rho)
    k = min(B, 1 << n)
    tol = 1e-11 if dt == 0 else 1e-5
    assert np.max(np.abs(ev[:k] - ref[:k])) <= tol
    assert np.all(np.abs(ev[k:]) <= tol)  # rank <= 2^n
    assert abs(tr - np.trace(rho).real) <= tol
    assert abs(pur - D.purity(rho)) <= tol
    assert abs(ent - D.entropy(ref, cut=1e-14)) <= 10 * tol


def test_pure_and_orthogonal_ensembles(qc):
    n = 8
    psi = W.random_state(W.rng(3), n)
    t = batch(qc, np.repeat(psi[None, :], 4, axis=0), 0)
    ev, (tr, pur, ent) = qc.qc_mixed_spectrum(t.data_ptr(), n, 0, 4, np.full(4, 0.25))
    assert abs(ev[0] - 1.0) <= 1e-12 and np.max(np.abs(ev[1:])) <= 1e-12
    assert abs(tr - 1.0) <= 1e-12 and abs(pur - 1.0) <= 1e-12 and abs(ent) <= 1e-10
    st = np.zeros((3, 1 << n), dtype=complex)
    for a, i in enumerate((1, 77, 200)):
        st[a, i] = 1.0
    P = np.array([0.5, 0.3, 0.2])
    ev, (tr, pur, ent) = qc.qc_mixed_spectrum(batch(qc, st, 0).data_ptr(), n, 0, 3, P)
    assert np.max(np.abs(ev - P)) <= 1e-14
    assert abs(ent + np.sum(P * np.log(P))) <= 1e-13


@pytest.mark.parametrize("twoj", [1, 3])
def test_wigner_operators(qc, twoj):
    for (a, b, g) in [(0.3, 1.2, 0.0), (5.1, 2.9, 0.7), (1.0, np.pi, 0.0)]:
        assert np.max(np.abs(qc.qc_wigner_d(twoj, a, b, g) - D.wigner_D(twoj, a, b, g))) <= 1e-15


@pytest.mark.parametrize("dt", [0, 1])
def test_multiverse_grover_scenario(qc, dt):
    import torch
    n, m, B = 9, 300, 24
    k = W.grover_iterations(n)
    mv = W.multiverse_noise(B, n, k, seed=31)
    # oracle: literal gate sequence per universe
    plan = []
    for b in range(B):
        if mv.kind[b] == 0:
            plan.append((0, (), 0, None))
        elif mv.kind[b] == 1:
            plan.append((1, (int(mv.qhit[b]),), int(mv.eloc[b]), D.wigner_D(1, mv.alpha[b], mv.beta[b], 0.0)))
        else:
            plan.append((2, (int(mv.qhit[b]), int(mv.qhit2[b])), int(mv.eloc[b]),
                         D.wigner_D(3, mv.alpha[b], mv.beta[b], 0.0)))
    ref_states = D.multiverse_grover(n, m, k, plan)
    # GPU: each universe a slice of one batch buffer, driven through the C ABI
    t = torch.empty((B, 1 << n), dtype=qc.torch_dtype(dt), device="cuda")
    for b in range(B):
        s = qc.State(n, dt, tensor=t[b])
        s.uniform()
        for it in range(k + 1):
            if mv.kind[b] and it == mv.eloc[b]:
                if mv.kind[b] == 1:
                    s.apply_1q(int(mv.qhit[b]), qc.qc_wigner_d(1, mv.alpha[b], mv.beta[b], 0.0))
                else:
                    qc.qc_apply_2q(s.h, int(mv.qhit[b]), int(mv.qhit2[b]),
                                   qc.qc_wigner_d(3, mv.alpha[b], mv.beta[b], 0.0))
            if it < k:
                s.grover_step([m])
        s.close()
    torch.cuda.synchronize()
    got = t.cpu().numpy().astype(np.complex128)
    tol = 1e-12 if dt == 0 else 2e-5
    assert np.max(np.abs(got - ref_states)) <= tol
    ev, (tr, pur, ent) = qc.qc_mixed_spectrum(t.data_ptr(), n, dt, B, mv.P)
    rho = D.density_matrix(ref_states, mv.P)
    ref = D.spectrum(rho)
    assert abs(tr - 1.0) <= 10 * tol  # unitary intrusions keep unit trace
    assert abs(pur - D.purity(rho)) <= 10 * tol and pur < 1.0 - 1e-3
    assert np.max(np.abs(ev - ref[:B])) <= 10 * tol
    assert abs(ent - D.entropy(ref)) <= 100 * tol


def test_density_invalid(qc):
    import torch
    t = torch.zeros(4 << 4, dtype=torch.complex128, device="cuda")
    for args in [(t.data_ptr(), 0, 0, 4, np.full(4, 0.25)), (t.data_ptr(), 4, 0, 0, np.zeros(0)),
                 (t.data_ptr(), 4, 0, 4, np.array([0.5, -0.1, 0.3, 0.3])),
                 (t.data_ptr(), 4, 0, 65, np.full(65, 1 / 65))]:
        with pytest.raises(qc.QCError):
            qc.qc_mixed_spectrum(*args)
    with pytest.raises(qc.QCError):
        qc.qc_density_matrix(t.data_ptr(), 16, 0, 4, np.full(4, 0.25), t.data_ptr())
    with pytest.raises(qc.QCError):
        qc.qc_wigner_d(2, 0.1, 0.2, 0.3)


@pytest.mark.parametrize("dt", [0, 1])
def test_mixed_spectrum_non_finite_gram(qc, dt):
    # a NaN amplitude makes the Gram matrix non-finite: the solver reports it
    # (QC_ECUDA) instead of returning eigenvalues
    n, B = 5, 3
    g = W.rng(77)
    states = np.stack([W.random_state(g, n) for _ in range(B)])
    states[1, 7] = np.nan
    t = batch(qc, states, dt)
    with pytest.raises(qc.QCError, match="non-finite"):
        qc.qc_mixed_spectrum(t.data_ptr(), n, dt, B, np.full(B, 1.0 / B))
    # the next call on finite data is unaffected
    states[1, 7] = 0.5
    t = batch(qc, states, dt)
    ev, (tr, pur, ent) = qc.qc_mixed_spectrum(t.data_ptr(), n, dt, B, np.full(B, 1.0 / B))
    assert np.all(np.isfinite(ev)) and np.isfinite(tr)
