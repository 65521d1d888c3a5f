"""Full-size parity at the benchmark configuration (30 qubits complex128,
32 qubits complex64), through the C ABI, on outputs the oracle side can
compute one by one:

* Grover with 8 seeded marked items, 100 iterations: every marked amplitude
  and a seeded sample of unmarked ones against the closed form
  sin((2k+1)theta)/sqrt(M), cos((2k+1)theta)/sqrt(N-M) (sec. 5.1);
* the QFT of that state, sampled, against its closed form
  QFT(psi)[n'] = b sqrt(N) delta_{n',0} + (a - b)/sqrt(N) sum_m e^{2 pi i m n'/N}
  (Appendix A's DFT identity applied to the Grover state);
* the gate sweep of the benchmark (H, CNOT, CPHASE at every t) followed by
  its inverse returns the sampled QFT amplitudes;
* seeded sampling of the Grover state: the state takes one value on all
  unmarked and one on all marked items, so its integer CDF has a closed
  form and the outcomes must match the Philox/bisection definition exactly.
"""
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


def closed(n, M, k):
    N = 1 << n
    th = math.asin(math.sqrt(M / N))
    return math.sin((2 * k + 1) * th) / math.sqrt(M), math.cos((2 * k + 1) * th) / math.sqrt(N - M)


def qft_closed(n, marked, a, b, idx):
    N = 1 << n
    out = np.zeros(len(idx), dtype=np.complex128)
    for i, q in enumerate(idx):
        s = 0j
        for m in marked:
            r = (int(m) * int(q)) % N
            ang = 2.0 * math.pi * r / N
            s += complex(math.cos(ang), math.sin(ang))
        out[i] = (a - b) / math.sqrt(N) * s + (b * math.sqrt(N) if q == 0 else 0.0)
    return out


def gather(st, idx):
    import torch
    t = torch.as_tensor(np.asarray(idx, dtype=np.int64), device=st.tensor.device)
    return st.tensor[t].cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("n,dt,tol,seed", [(30, 0, 1e-12, 2026), (32, 1, 1e-5, 2027)])
def test_bench_workload_full_size(qc, n, dt, tol, seed):
    import torch
    N = 1 << n
    M, iters = 8, 100
    marked = W.marked_indices(W.rng(seed), n, M)
    st = qc.State(n, dt)
    st.uniform()
    for _ in range(iters):
        st.grover_step(marked)
    a, b = closed(n, M, iters)
    g = W.rng(seed + 1)
    idx = np.unique(np.concatenate([marked.astype(np.int64), g.integers(0, N, 4000), [0, 1, N - 1]]))
    ref = np.where(np.isin(idx, marked.astype(np.int64)), a, b)
    got = gather(st, idx)
    assert np.max(np.abs(got - ref)) <= tol
    # seeded sampling of the Grover state (two distinct probabilities)
    if dt == 0:
        pv = st.probs()
        p_m = float(pv[int(marked[0])].item())
        p_u = float(pv[int(idx[~np.isin(idx, marked.astype(np.int64))][0])].item())
        assert all(float(pv[int(m)].item()) == p_m for m in marked)
        shots = st.sample(99, 1000).cpu().numpy()
        w_m, w_u = int(p_m * 2.0 ** 62), int(p_u * 2.0 ** 62)
        ms = sorted(int(m) for m in marked)

        def W_at(i):  # closed-form integer CDF
            cnt = sum(1 for m in ms if m <= i)
            return (i + 1 - cnt) * w_u + cnt * w_m
        total = W_at(N - 1)
        tg = O.sample_targets(99, 1000, total)
        for s_, t_ in zip(shots, tg):
            lo, hi = 0, N - 1
            while lo < hi:
                mid = (lo + hi) // 2
                if W_at(mid) > t_:
                    hi = mid
                else:
                    lo = mid + 1
            assert int(s_) == lo
    # QFT of the Grover state
    st.qft()
    qidx = np.unique(np.concatenate([[0, 1, 2, N - 1, N // 2], g.integers(0, N, 2000)]))
    qref = qft_closed(n, marked, a, b, qidx)
    got = gather(st, qidx)
    assert np.max(np.abs(got - qref)) <= tol
    # the benchmark sweep and its inverse
    H = O.H_MAT
    for t in range(n):
        st.apply_1q(t, H)
        st.cnot((t + 1) % n, t)
        st.cphase((t + 1) % n, t, 1)
    for t in reversed(range(n)):
        st.cphase((t + 1) % n, t, 1)  # its own inverse
        st.cnot((t + 1) % n, t)
        st.apply_1q(t, H)
    got = gather(st, qidx)
    assert np.max(np.abs(got - qref)) <= tol * 4
    nrm = st.norm()
    assert abs(nrm - 1.0) <= (1e-11 if dt == 0 else 1e-5)
    st.close()
    del st
    torch.cuda.empty_cache()
