"""GPU parity of the adjoint gradient and of the batched noisy trajectories
against the CPU oracle, through the C ABI."""
import ctypes
import math

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


def ansatz_gate_array(qc, circ):
    gates = []
    for g in O.ansatz_gates(circ):
        if g[0] == "cnot":
            gates.append((qc.QC_G_CNOT, g[1], g[2], 0))
        else:
            gates.append((qc.QC_G_RY if g[0] == "ry" else qc.QC_G_RZ, g[1], 0, g[2]))
    arr = (qc.Gate * len(gates))(*[qc.Gate(*t) for t in gates])
    return arr, len(gates)


def terms_array(qc, terms):
    return (qc.PauliTerm * len(terms))(*[qc.PauliTerm(x, z, c) for (x, z, c) in terms])


def run_adjoint(qc, circs, dt):
    import torch
    n = circs[0].n
    B = len(circs)
    P = circs[0].n_params
    theta = torch.tensor(np.stack([c.theta for c in circs]), dtype=torch.float64, device="cuda")
    cdt = torch.complex128 if dt == 0 else torch.complex64
    psi = torch.empty(B << n, dtype=cdt, device="cuda")
    lam = torch.empty_like(psi)
    E = torch.empty(B, dtype=torch.float64, device="cuda")
    grad = torch.empty(B, P, dtype=torch.float64, device="cuda")
    gates, ng = ansatz_gate_array(qc, circs[0])
    terms = W.ansatz_hamiltonian(n)
    st = torch.cuda.current_stream().cuda_stream
    rc = qc.lib().qc_adjoint_grad(n, dt, B, gates, ng, ctypes.c_void_p(theta.data_ptr()), P, P,
                                  terms_array(qc, terms), len(terms), ctypes.c_void_p(psi.data_ptr()),
                                  ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                  ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(st))
    assert rc == 0, qc.last_error()
    torch.cuda.synchronize()
    return E.cpu().numpy(), grad.cpu().numpy(), psi.cpu().numpy().reshape(B, -1)


def run_forward(qc, circs, dt):
    import torch
    n, B, P = circs[0].n, len(circs), circs[0].n_params
    theta = torch.tensor(np.stack([c.theta for c in circs]), dtype=torch.float64, device="cuda")
    cdt = torch.complex128 if dt == 0 else torch.complex64
    psi = torch.empty(B << n, dtype=cdt, device="cuda")
    gates, ng = ansatz_gate_array(qc, circs[0])
    rc = qc.lib().qc_circuit_forward(n, dt, B, gates, ng, ctypes.c_void_p(theta.data_ptr()), P,
                                     ctypes.c_void_p(psi.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, qc.last_error()
    torch.cuda.synchronize()
    return psi.cpu().numpy().reshape(B, -1)


@pytest.mark.parametrize("dt", [0, 1])
def test_forward_vs_oracle(qc, dt):
    circs = W.ansatz(8, 4, seed=5, batch=3)
    got = run_forward(qc, circs, dt)
    for b, c in enumerate(circs):
        ref = O.ansatz_forward(c)
        assert np.max(np.abs(got[b] - ref)) <= (1e-12 if dt == 0 else 1e-5)


@pytest.mark.parametrize("dt", [0, 1])
def test_adjoint_small_all_angles(qc, dt):
    circs = W.ansatz(6, 5, seed=11, batch=2)
    E, g, psi = run_adjoint(qc, circs, dt)
    terms = W.ansatz_hamiltonian(6)
    for b, c in enumerate(circs):
        Er, gr = O.adjoint_gradient(c, terms)
        tol = 1e-12 if dt == 0 else 2e-5
        assert abs(E[b] - Er) <= tol
        assert np.max(np.abs(g[b] - gr)) <= tol


@pytest.mark.parametrize("dt", [0, 1])
def test_adjoint_unfused_gate_list(qc, dt):
    # rotations interleaved with H, RX and partial CNOT chains: no pass fusion
    import torch
    n, B = 5, 2
    rng = W.rng(21)
    gl, ora = [], []
    k = 0
    for l in range(3):
        for q in range(n):
            kind = (l + q) % 3  # RX, RY, RZ
            gl.append(qc.Gate(kind, q, 0, k))
            ora.append(("rx" if kind == 0 else "ry" if kind == 1 else "rz", q, k))
            k += 1
            if q % 2 == 0:
                gl.append(qc.Gate(qc.QC_G_H, q, 0, 0))
                ora.append(("h", q, 0))
        for (c, t) in ((0, 1), (2, 4), (4, 3)):
            gl.append(qc.Gate(qc.QC_G_CNOT, c, t, 0))
            ora.append(("cnot", c, t))
    P = k
    theta = rng.random((B, P)) * 6.28
    terms = W.ansatz_hamiltonian(n) + [(0b10100, 0b00110, 0.3)]

    def mats(g, th, dag=False):
        if g[0] == "h":
            return O.H_MAT
        a = th[g[2]] * (-1 if dag else 1)
        if g[0] == "rx":
            return np.array([[math.cos(a / 2), -1j * math.sin(a / 2)], [-1j * math.sin(a / 2), math.cos(a / 2)]])
        return O.ry(a) if g[0] == "ry" else O.rz(a)

    def fwd(th):
        psi = O.zero_state(n)
        for g in ora:
            if g[0] == "cnot":
                O.cnot(psi, n, g[1], g[2])
            else:
                O.apply_1q(psi, n, g[1], mats(g, th))
        return psi
    gates = (qc.Gate * len(gl))(*gl)
    tarr = (qc.PauliTerm * len(terms))(*[qc.PauliTerm(x, z, c) for (x, z, c) in terms])
    th_d = torch.tensor(theta, dtype=torch.float64, device="cuda")
    cdt = torch.complex128 if dt == 0 else torch.complex64
    psi = torch.empty(B << n, dtype=cdt, device="cuda")
    lam = torch.empty_like(psi)
    E = torch.empty(B, dtype=torch.float64, device="cuda")
    grad = torch.empty(B, P, dtype=torch.float64, device="cuda")
    rc = qc.lib().qc_adjoint_grad(n, dt, B, gates, len(gl), ctypes.c_void_p(th_d.data_ptr()), P, P, tarr,
                                  len(terms), ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                                  ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, qc.last_error()
    torch.cuda.synchronize()
    tol = 1e-12 if dt == 0 else 2e-5
    for b in range(B):
        Er = O.energy(fwd(theta[b]), n, terms)
        assert abs(E[b].item() - Er) <= tol
        for kk in range(P):  # parameter shift on the oracle forward
            tp, tm = theta[b].copy(), theta[b].copy()
            tp[kk] += math.pi / 2
            tm[kk] -= math.pi / 2
            ps = 0.5 * (O.energy(fwd(tp), n, terms) - O.energy(fwd(tm), n, terms))
            assert abs(grad[b, kk].item() - ps) <= tol


def test_adjoint_n20_sampled_angles_param_shift(qc):
    # full-size circuit (n = 20, 50 layers, 2000 angles), complex128; the
    # oracle's adjoint for all angles, plus parameter shift on a sample
    circs = W.ansatz(20, 50, seed=0, batch=1)
    E, g, _ = run_adjoint(qc, circs, 0)
    terms = W.ansatz_hamiltonian(20)
    Er, gr = O.adjoint_gradient(circs[0], terms)
    assert abs(E[0] - Er) <= 1e-11
    assert np.max(np.abs(g[0] - gr)) <= 1e-11
    rng = W.rng(99)
    c = circs[0]
    for k in rng.choice(c.n_params, 3, replace=False):
        tp, tm = c.theta.copy(), c.theta.copy()
        tp[k] += math.pi / 2
        tm[k] -= math.pi / 2
        ps = 0.5 * (O.energy(O.ansatz_forward(c, tp), 20, terms) - O.energy(O.ansatz_forward(c, tm), 20, terms))
        assert abs(g[0][k] - ps) <= 1e-10


def test_adjoint_c64_batch_vs_c128(qc):
    circs = W.ansatz(12, 10, seed=3, batch=4)
    E64, g64, _ = run_adjoint(qc, circs, 1)
    E128, g128, _ = run_adjoint(qc, circs, 0)
    assert np.max(np.abs(E64 - E128)) <= 1e-5
    assert np.max(np.abs(g64 - g128)) <= 1e-5


def run_traj(qc, tb, autotune=0, keep=()):
    """Runs the batch through the C ABI (twice: the second run replays the
    captured graph).  keep: instances whose final complex64 states come back
    too (qc_traj_plan_run_states), as a dict index -> numpy array."""
    import torch
    n_inst = len(tb.nq)
    nq = np.ascontiguousarray(tb.nq, dtype=np.int32)
    mk = np.ascontiguousarray(tb.marked, dtype=np.uint64)
    it = np.ascontiguousarray(tb.iters, dtype=np.int32)
    d = qc.TrajDesc(n_inst, nq.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    mk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                    it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), tb.seed, tb.thr_gate,
                    tb.thr_readout, tb.p_readout)
    plan = ctypes.c_void_p()
    st = torch.cuda.current_stream().cuda_stream
    rc = qc.lib().qc_traj_plan_create(ctypes.byref(d), ctypes.c_void_p(st), autotune, ctypes.byref(plan))
    assert rc == 0, qc.last_error()
    ps = torch.empty(n_inst, dtype=torch.float64, device="cuda")
    pr = torch.empty_like(ps)
    oc = torch.empty(n_inst, dtype=torch.int64, device="cuda")
    ne = torch.empty(n_inst, dtype=torch.int32, device="cuda")
    out = qc.TrajOut(ps.data_ptr(), pr.data_ptr(), oc.data_ptr(), ne.data_ptr())
    keep = sorted(set(int(i) for i in keep))
    off = np.full(n_inst, np.iinfo(np.uint64).max, dtype=np.uint64)
    pos = 0
    for i in keep:
        off[i] = pos
        pos += 1 << int(tb.nq[i])
    states = torch.full((max(pos, 1),), float("nan"), dtype=torch.complex64, device="cuda")
    off_d = torch.from_numpy(off.view(np.int64)).cuda()
    for _ in range(2):  # second run replays the captured graph
        if keep:
            rc = qc.lib().qc_traj_plan_run_states(plan, ctypes.byref(out), ctypes.c_void_p(off_d.data_ptr()),
                                                  ctypes.c_void_p(states.data_ptr()))
        else:
            rc = qc.lib().qc_traj_plan_run(plan, ctypes.byref(out))
        assert rc == 0, qc.last_error()
    torch.cuda.synchronize()
    info = [ctypes.c_int(), ctypes.c_int(), ctypes.c_int()]
    qc.lib().qc_traj_plan_info(plan, *[ctypes.byref(x) for x in info])
    qc.lib().qc_traj_plan_free(plan)
    sv = states.cpu().numpy()
    kept = {i: sv[int(off[i]):int(off[i]) + (1 << int(tb.nq[i]))] for i in keep}
    return (ps.cpu().numpy(), pr.cpu().numpy(), oc.cpu().numpy().astype(np.uint64),
            ne.cpu().numpy(), [x.value for x in info], kept)


def check_instance(tb, i, ps, pr, oc, ne, kept):
    """One instance against the oracle's literal replay: the error count
    exactly, the final state (normalised) and both success probabilities
    within the complex64 tolerance, and the seeded outcome exactly, replayed
    from the integer weights of the kernel's own final state."""
    n, m, k = int(tb.nq[i]), int(tb.marked[i]), int(tb.iters[i])
    psi, errs = O.trajectory_run(n, m, k, tb.seed, int(i), tb.thr_gate)
    assert ne[i] == errs
    prob = O.probs(psi, n)
    assert abs(ps[i] - prob[m] / prob.sum()) <= 1e-5
    assert abs(pr[i] - O.readout_success(prob, n, m, tb.p_readout) / prob.sum()) <= 1e-5
    if i in kept:
        g = kept[i].astype(np.complex128)
        assert np.max(np.abs(g / np.linalg.norm(g) - psi / np.linalg.norm(psi))) <= 1e-5
        w = O.readout_weights_c64(kept[i])
        assert int(oc[i]) == O.trajectory_measure_weights(w, n, tb.seed, int(i), tb.thr_readout)


def test_traj_noiseless_closed_form(qc):
    tb = W.trajectory_batch(24, 6, 12, seed=4, p_gate=0.0, p_readout=0.0)
    ps, pr, oc, ne, _, _ = run_traj(qc, tb)
    for i in range(len(tb.nq)):
        n, k = int(tb.nq[i]), int(tb.iters[i])
        ref = math.sin((2 * k + 1) * math.asin(2 ** (-n / 2))) ** 2
        assert abs(ps[i] - ref) <= 1e-5
        assert abs(pr[i] - ref) <= 1e-5
        assert ne[i] == 0


@pytest.mark.parametrize("p", [1e-3, 2e-2])
def test_traj_replay_vs_oracle(qc, p):
    # the oracle replays every trajectory's Philox draws literally; each
    # outcome is replayed exactly from the kernel's own read-out weights
    tb = W.trajectory_batch(40, 5, 10, seed=17, p_gate=p, p_readout=0.05)
    ps, pr, oc, ne, info, kept = run_traj(qc, tb, autotune=1, keep=range(len(tb.nq)))
    for i in range(len(tb.nq)):
        check_instance(tb, i, ps, pr, oc, ne, kept)


@pytest.mark.parametrize("autotune", [0, 1])
def test_traj_replay_wide_states(qc, autotune):
    # 15..17 qubits: every CTA of a cluster streams several 16-byte vectors
    # per thread, and most iterations draw no error (the error-free pass)
    tb = W.trajectory_batch(6, 15, 17, seed=23, p_gate=2e-3, p_readout=0.01)
    ps, pr, oc, ne, info, kept = run_traj(qc, tb, autotune=autotune, keep=range(len(tb.nq)))
    for i in range(len(tb.nq)):
        check_instance(tb, i, ps, pr, oc, ne, kept)


def test_traj_degenerate_sizes(qc):
    # 1..4 qubits: clusters of one or two CTAs, states of 2..16 amplitudes
    # (one 16-byte vector per CTA at n = 1), noisy enough to exercise the
    # error passes
    tb = W.trajectory_batch(24, 1, 4, seed=8, p_gate=0.05, p_readout=0.05)
    ps, pr, oc, ne, info, kept = run_traj(qc, tb, autotune=1, keep=range(len(tb.nq)))
    for i in range(len(tb.nq)):
        check_instance(tb, i, ps, pr, oc, ne, kept)


def test_traj_states_output_skips_and_keeps(qc):
    # instances not asked for leave the state buffer alone; the outputs of a
    # run with kept states equal those of a plain run
    tb = W.trajectory_batch(12, 6, 9, seed=31, p_gate=1e-2, p_readout=0.02)
    a = run_traj(qc, tb, autotune=0)
    b = run_traj(qc, tb, autotune=0, keep=[2, 7])
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    assert set(b[5]) == {2, 7} and all(np.all(np.isfinite(v)) for v in b[5].values())


# ---------------------------------------------------------- torch.autograd --

def ansatz_circuit(qc, circ, dt):
    gates = []
    for g in O.ansatz_gates(circ):
        if g[0] == "cnot":
            gates.append((qc.QC_G_CNOT, g[1], g[2], 0))
        else:
            gates.append((qc.QC_G_RY if g[0] == "ry" else qc.QC_G_RZ, g[1], 0, g[2]))
    return qc.Circuit(circ.n, gates, W.ansatz_hamiltonian(circ.n), dt)


@pytest.mark.parametrize("dt", [0, 1])
def test_autograd_energy_and_grad_vs_oracle(qc, dt):
    import torch
    circs = W.ansatz(6, 4, seed=21, batch=3)
    C = ansatz_circuit(qc, circs[0], dt)
    theta = torch.tensor(np.stack([c.theta for c in circs]), dtype=torch.float64, device="cuda",
                         requires_grad=True)
    E = qc.energy(theta, C)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")  # upstream gradient
    (E * w).sum().backward()
    tol = 1e-12 if dt == 0 else 2e-5
    terms = W.ansatz_hamiltonian(6)
    for b, c in enumerate(circs):
        Er, gr = O.adjoint_gradient(c, terms)
        assert abs(float(E[b].detach()) - Er) <= tol
        assert np.max(np.abs(theta.grad[b].cpu().numpy() - w[b].item() * gr)) <= 3 * tol
    # without autograd: the forward pass and the expectations only
    with torch.no_grad():
        E2 = qc.energy(theta, C)
    assert float(torch.max(torch.abs(E2 - E.detach()))) <= tol


def test_autograd_gradcheck_finite_differences(qc):
    import torch
    circ = W.ansatz(3, 2, seed=4)[0]
    C = ansatz_circuit(qc, circ, 0)
    theta = torch.tensor(circ.theta, dtype=torch.float64, device="cuda", requires_grad=True)
    assert qc.energy(theta, C).dim() == 0  # one angle vector: a scalar energy
    assert torch.autograd.gradcheck(lambda t: qc.energy(t, C), (theta,), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_autograd_rejects_host_theta(qc):
    import torch
    circ = W.ansatz(3, 1, seed=1)[0]
    C = ansatz_circuit(qc, circ, 0)
    with pytest.raises(ValueError):
        qc.energy(torch.tensor(circ.theta), C)
    with pytest.raises(ValueError):
        qc.energy(torch.zeros(2, dtype=torch.float64, device="cuda"), C)  # fewer angles than used


def test_trajectory_plan_wrapper(qc):
    # the Python wrapper against the noiseless closed form and the raw C calls
    import torch
    tb = W.trajectory_batch(40, 6, 12, seed=77, p_gate=0.0, p_readout=0.0)
    plan = qc.TrajectoryPlan(tb.nq, tb.marked, tb.iters, tb.seed, p_gate=0.0, p_readout=0.0, autotune=False)
    out = plan.run()
    torch.cuda.synchronize()
    ps = out["p_success"].cpu().numpy()
    for i in range(len(tb.nq)):
        th = math.asin(2.0 ** (-tb.nq[i] / 2.0))
        assert abs(ps[i] - math.sin((2 * tb.iters[i] + 1) * th) ** 2) <= 1e-5
    assert int(out["n_errors"].sum()) == 0
    assert len(plan.shape) == 3
    plan.close()
    tb2 = W.trajectory_batch(24, 8, 12, seed=78, p_gate=0.01, p_readout=0.01)
    # the same (default) launch shape on both sides, so the reductions add in
    # the same order
    plan = qc.TrajectoryPlan(tb2.nq, tb2.marked, tb2.iters, tb2.seed, p_gate=0.01, p_readout=0.01,
                             autotune=False)
    got = plan.run()
    torch.cuda.synchronize()
    plan.close()
    ps, pr, oc, ne, _, _ = run_traj(qc, tb2)  # raw qc_traj_plan_* calls
    assert np.array_equal(got["n_errors"].cpu().numpy(), ne)
    assert np.array_equal(got["outcome"].cpu().numpy().astype(np.uint64), oc)
    assert np.array_equal(got["p_success"].cpu().numpy(), ps)
    assert np.array_equal(got["p_readout"].cpu().numpy(), pr)
