"""Host side of the binding: the circuit's packed gate and Pauli arrays,
its parameter count and the trajectory thresholds (no GPU)."""
import paper_0902_0699_gb300 as qc


def test_circuit_packing():
    gates = [(qc.QC_G_RY, 0, 0, 0), (qc.QC_G_CNOT, 0, 1, 0), (qc.QC_G_RZ, 2, 0, 4), (qc.QC_G_H, 1, 0, 9)]
    C = qc.Circuit(3, gates, [(0, 3, 1.0), (1, 0, 0.1)], qc.QC_C64)
    assert C.n_params == 5  # the Hadamard's param field is not an angle
    assert (C.n_gates, C.n_terms, C.dt) == (4, 2, qc.QC_C64)
    assert [(g.kind, g.q0, g.q1, g.param) for g in C.gates] == gates
    assert [(t.xmask, t.zmask, t.coeff) for t in C.terms] == [(0, 3, 1.0), (1, 0, 0.1)]
    assert qc.Circuit(2, [(qc.QC_G_CNOT, 0, 1, 0)], []).n_params == 0


def test_autograd_function_is_a_torch_function():
    import torch
    assert issubclass(qc._adjoint_function(), torch.autograd.Function)


def test_trajectory_thresholds_follow_the_descriptor_definition():
    import workloads as W
    for p in (0.0, 1e-3, 0.35, 0.5, 1.0 - 2 ** -40, 1.0):
        assert qc._threshold(p) == W.prob_threshold(p)
