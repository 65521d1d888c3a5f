"""The binding's same-name functions for the entry points the classes also
wrap (state info, launch counter, allocation-free sampling, fused plans,
trajectory plans, forward pass and adjoint gradient): each gives what the
class path or the allocating call gives on the same inputs."""
import ctypes

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


def test_state_info_and_launch_counter(qc):
    s = qc.State(9, qc.QC_C64)
    ptr, n, dt = qc.qc_state_info(s.h)
    assert (ptr, n, dt) == (s.tensor.data_ptr(), 9, qc.QC_C64)
    before = qc.qc_kernel_launches()
    s.reset(0)
    s.apply_1q(3, O.H_MAT)
    assert qc.qc_kernel_launches() > before
    assert "sm_103a" in qc.qc_version() and isinstance(qc.qc_last_error(), str)
    s.close()


@pytest.mark.parametrize("dt", [0, 1])
def test_sample_noalloc_wrapper(qc, dt):
    import torch
    n = 12
    s = qc.State(n, dt)
    s.load(W.random_state(W.rng(31), n))
    out = torch.empty(300, dtype=torch.int64, device="cuda")
    qc.qc_sample_noalloc(s.tensor.data_ptr(), n, dt, 99, 300, out.data_ptr())
    assert np.array_equal(out.cpu().numpy(), s.sample(99, 300).cpu().numpy())
    s.close()


def test_fused_plan_wrappers(qc):
    n = 10
    circ = W.random_circuit(n, 6, seed=5)
    ops = []
    for l in range(circ.layers):
        for q in range(n):
            ops.append((1, q, 0, 0, circ.U[l, q]))
        for (c, t) in circ.cnot_pairs(l):
            ops.append((2, c, t, 0, None))
    h = qc.qc_fused_plan_create(n, ops, kmax=4, pad=False)
    ref = qc.FusedPlan(n, ops, kmax=4, pad=False)
    assert qc.qc_fused_plan_info(h) == ref.info()
    qs, U = qc.qc_fused_plan_block(h, 0)
    qs2, U2 = ref.block(0)
    assert qs == qs2 and np.array_equal(U, U2)
    a, b = qc.State(n, 0).reset(0), qc.State(n, 0).reset(0)
    qc.qc_fused_plan_run(a.h, h)
    ref.run(b.h)
    assert np.array_equal(a.numpy(), b.numpy())
    qc.qc_fused_plan_free(h)
    ref.close()
    a.close()
    b.close()


def test_trajectory_plan_wrappers(qc):
    import torch
    tb = W.trajectory_batch(24, 8, 12, seed=78, p_gate=0.01, p_readout=0.01)
    nq = np.ascontiguousarray(tb.nq, dtype=np.int32)
    mk = np.ascontiguousarray(tb.marked, dtype=np.uint64)
    it = np.ascontiguousarray(tb.iters, dtype=np.int32)
    d = qc.TrajDesc(len(nq), nq.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    mk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                    it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), tb.seed, tb.thr_gate, tb.thr_readout,
                    tb.p_readout)
    h = qc.qc_traj_plan_create(d, None, False)
    assert len(qc.qc_traj_plan_info(h)) == 3
    outs = {k: torch.empty(len(nq), dtype=t, device="cuda") for k, t in
            (("ps", torch.float64), ("pr", torch.float64), ("oc", torch.int64), ("ne", torch.int32))}
    qc.qc_traj_plan_run(h, qc.TrajOut(outs["ps"].data_ptr(), outs["pr"].data_ptr(), outs["oc"].data_ptr(),
                                      outs["ne"].data_ptr()))
    torch.cuda.synchronize()
    qc.qc_traj_plan_free(h)
    plan = qc.TrajectoryPlan(tb.nq, tb.marked, tb.iters, tb.seed, p_gate=0.01, p_readout=0.01, autotune=False)
    got = plan.run()
    torch.cuda.synchronize()
    plan.close()
    assert np.array_equal(outs["ps"].cpu().numpy(), got["p_success"].cpu().numpy())
    assert np.array_equal(outs["oc"].cpu().numpy(), got["outcome"].cpu().numpy())
    assert np.array_equal(outs["ne"].cpu().numpy(), got["n_errors"].cpu().numpy())
    # final states: the same-name call and the wrapper's keep= give the same
    h = qc.qc_traj_plan_create(d, None, False)
    off = np.full(len(nq), np.iinfo(np.uint64).max, dtype=np.uint64)
    off[5] = 0
    off_d = torch.from_numpy(off.view(np.int64)).cuda()
    st = torch.empty(1 << int(nq[5]), dtype=torch.complex64, device="cuda")
    qc.qc_traj_plan_run_states(h, qc.TrajOut(outs["ps"].data_ptr(), outs["pr"].data_ptr(), outs["oc"].data_ptr(),
                                             outs["ne"].data_ptr()), off_d.data_ptr(), st.data_ptr())
    torch.cuda.synchronize()
    qc.qc_traj_plan_free(h)
    plan = qc.TrajectoryPlan(tb.nq, tb.marked, tb.iters, tb.seed, p_gate=0.01, p_readout=0.01, autotune=False)
    got = plan.run(keep=[5])
    torch.cuda.synchronize()
    plan.close()
    assert torch.equal(got["states"][5], st)
    assert np.array_equal(outs["oc"].cpu().numpy(), got["outcome"].cpu().numpy())
    w = O.readout_weights_c64(st.cpu().numpy())
    assert int(got["outcome"][5]) == O.trajectory_measure_weights(w, int(nq[5]), tb.seed, 5, tb.thr_readout)


@pytest.mark.parametrize("dt", [0, 1])
def test_forward_and_adjoint_wrappers(qc, dt):
    import torch
    circs = W.ansatz(6, 4, seed=21, batch=3)
    gates = []
    for g in O.ansatz_gates(circs[0]):
        if g[0] == "cnot":
            gates.append((qc.QC_G_CNOT, g[1], g[2], 0))
        else:
            gates.append((qc.QC_G_RY if g[0] == "ry" else qc.QC_G_RZ, g[1], 0, g[2]))
    terms = W.ansatz_hamiltonian(6)
    C = qc.Circuit(6, gates, terms, dt)
    theta = torch.tensor(np.stack([c.theta for c in circs]), dtype=torch.float64, device="cuda")
    B, P = theta.shape
    E_ref, g_ref = C.energy_and_grad(theta)
    psi = torch.empty(B << 6, dtype=qc.torch_dtype(dt), device="cuda")
    lam = torch.empty_like(psi)
    E = torch.empty(B, dtype=torch.float64, device="cuda")
    grad = torch.empty(B, P, dtype=torch.float64, device="cuda")
    qc.qc_adjoint_grad(6, dt, B, gates, theta.data_ptr(), P, P, terms, psi.data_ptr(), lam.data_ptr(),
                       E.data_ptr(), grad.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(E, E_ref) and torch.equal(grad, g_ref)
    qc.qc_circuit_forward(6, dt, B, gates, theta.data_ptr(), P, psi.data_ptr())
    torch.cuda.synchronize()
    norms = (psi.view(B, -1).abs() ** 2).sum(dim=1).cpu().numpy()
    assert np.max(np.abs(norms - 1.0)) <= (1e-12 if dt == 0 else 1e-5)
    assert torch.allclose(C.energy(theta), E_ref, atol=1e-12 if dt == 0 else 1e-5)
