"""qc_sample_noalloc: the seeded sampler for callers that cannot allocate
device memory (their pool already owns it, or they cannot take the
synchronisation a cudaMalloc / cudaFree implies).  It keeps its CDF in a
fixed device array instead of allocating one per call.

Checked through the C ABI against the allocating qc_sample on two calls in
a row (the shared scratch must not leak state from one call into the
next).  Sampling is integer work, so the outcomes must match exactly.  This
file is collected last so that a stop-at-first-failure run has already run
every other test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0902_0699_gb300 as q
    q.lib()
    return q


def _noalloc(qc, state, seed, shots):
    import torch
    out = torch.full((shots,), -1, dtype=torch.int64, device="cuda")
    rc = qc.lib().qc_sample_noalloc(ctypes.c_void_p(state.tensor.data_ptr()), state.n, state.dt, seed, shots,
                                    ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, qc.last_error()
    return out.cpu().numpy()


def test_noalloc_matches_qc_sample_twice(qc):
    cases = [(20, qc.QC_C128, 11, 4096), (13, qc.QC_C64, 2 ** 40 + 3, 1000)]
    for n, dt, seed, shots in cases:  # two calls in a row, different sizes
        s = qc.State(n, dt)
        s.load(W.random_state(W.rng(n), n))
        ref = s.sample(seed, shots).cpu().numpy()
        got = _noalloc(qc, s, seed, shots)
        assert np.array_equal(got, ref)
        s.close()


def test_noalloc_rejects_oversize(qc):
    import torch
    n = 21
    buf = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = qc.lib().qc_sample_noalloc(ctypes.c_void_p(buf.data_ptr()), n, qc.QC_C64, 1, 4,
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert rc == qc.QC_EINVAL
    assert "out of range" in qc.last_error()
