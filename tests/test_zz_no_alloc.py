"""qc_sample_noalloc: the seeded sampler for callers that cannot allocate
device memory (their pool already owns it, or they cannot take the
synchronisation a cudaMalloc / cudaFree implies).  It keeps its CDF in a
fixed device array instead of allocating one per call.

Checked through the C ABI against the allocating qc_sample on two calls in
a row (the shared scratch must not leak state from one call into the
next), on both of qc_sample's paths (more shots than 2048-amplitude blocks:
the full CDF; fewer: a per-shot bisection of the block offsets), and
against the oracle's integer-CDF sampler.  Sampling is integer work, so the
outcomes must match exactly.  A state the sampler must reject (a NaN, or
|C_i|^2 > 2) is caught on the device, and the next call still works.  This
file is collected last so that a stop-at-first-failure run has already run
every other test; it also passes on its own in a fresh process."""
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


def _noalloc_rc(qc, ptr, n, dt, seed, shots):
    import torch
    out = torch.full((max(shots, 1),), -1, dtype=torch.int64, device="cuda")
    rc = qc.lib().qc_sample_noalloc(ctypes.c_void_p(ptr), n, dt, seed, shots, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out[:shots].cpu().numpy()


def _noalloc(qc, state, seed, shots):
    rc, out = _noalloc_rc(qc, state.tensor.data_ptr(), state.n, state.dt, seed, shots)
    assert rc == 0, qc.last_error()
    return out


def _born(v):
    """Born probabilities as the library forms them: re*re + im*im in
    binary64 (complex64 squares are exact there), one rounding per step."""
    re, im = v.real.astype(np.float64), v.imag.astype(np.float64)
    return re * re + im * im


def test_noalloc_matches_qc_sample_twice(qc):
    # (n, dtype, seed, shots): more shots than blocks (2^n / 2048) takes
    # qc_sample's full-CDF path, fewer its per-shot block bisection
    cases = [(20, qc.QC_C128, 11, 4096), (13, qc.QC_C64, 2 ** 40 + 3, 1000),
             (20, qc.QC_C128, 5, 100), (20, qc.QC_C64, 6, 100), (16, qc.QC_C64, 7, 30)]
    for n, dt, seed, shots in cases:  # calls in a row, different sizes and paths
        s = qc.State(n, dt)
        s.load(W.random_state(W.rng(n + shots), n))
        ref = s.sample(seed, shots).cpu().numpy()
        got = _noalloc(qc, s, seed, shots)
        assert np.array_equal(got, ref)
        assert np.array_equal(got.astype(np.uint64), O.sample_from_probs(_born(s.numpy()), seed, shots))
        s.close()


def test_noalloc_rejects_unusable_states_on_the_device(qc):
    import torch
    n = 10
    s = qc.State(n, qc.QC_C64)
    v = W.random_state(W.rng(9), n).astype(np.complex64)
    bad = v.copy()
    bad[17] = np.nan
    s.load(bad)
    rc, _ = _noalloc_rc(qc, s.tensor.data_ptr(), n, qc.QC_C64, 1, 8)
    assert rc == qc.QC_EINVAL and "unusable" in qc.last_error()
    big = v.copy()
    big[3] = 2.0  # |C|^2 = 4 > 2
    s.load(big)
    rc, _ = _noalloc_rc(qc, s.tensor.data_ptr(), n, qc.QC_C64, 1, 8)
    assert rc == qc.QC_EINVAL
    s.load(v)  # the verdict of a rejected call does not stick
    got = _noalloc(qc, s, 21, 50)
    assert np.array_equal(got.astype(np.uint64), O.sample_from_probs(_born(s.numpy()), 21, 50))
    s.close()
    torch.cuda.synchronize()


def test_noalloc_rejects_oversize(qc):
    import torch
    n = 21
    buf = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = qc.lib().qc_sample_noalloc(ctypes.c_void_p(buf.data_ptr()), n, qc.QC_C64, 1, 4,
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert rc == qc.QC_EINVAL
    assert "out of range" in qc.last_error()
