"""GPU parity of the gate kernels against the CPU oracle, element by
element, through the C ABI.  Tolerances: max |d amp| <= 1e-12 (complex128),
<= 1e-5 (complex64); permutations (CNOT, SWAP) bit-exact."""
import math

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


def mk(qc, n, dt, vec=None, seed=0):
    s = qc.State(n, dt)
    if vec is None:
        vec = W.random_state(W.rng(seed), n)
    s.load(vec)
    return s, np.asarray(vec, dtype=np.complex128)


def as_dt(v, dt):
    return v.astype(np.complex64).astype(np.complex128) if dt == 1 else v


MATS = {
    "haar": lambda g: W.haar_u2(g, 1)[0],
    "ry": lambda g: O._mat(O.ry(g.random() * 6.3)),
    "rz": lambda g: O._mat(O.rz(g.random() * 6.3)),
    "phase": lambda g: O._mat(np.diag([1, np.exp(1j * g.random() * 6.3)])),
    "x": lambda g: O._mat(O.X_MAT),
    "y": lambda g: O._mat(O.Y_MAT),
    "h": lambda g: O._mat(O.H_MAT),
    "ident": lambda g: O._mat(np.eye(2, dtype=np.complex128)),
}


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 6, 13, 17])
@pytest.mark.parametrize("kind", list(MATS))
def test_apply_1q_all_t(qc, dt, n, kind):
    g = W.rng(hash((n, kind)) % 1000)
    s, v = mk(qc, n, dt, seed=n)
    ref = as_dt(v, dt).copy()
    for t in range(n):
        U = MATS[kind](g)
        s.apply_1q(t, U)
        O.apply_1q(ref, n, t, U)
    got = s.numpy()
    assert np.max(np.abs(got - ref)) <= TOL[dt] * max(1, n / 4)


@pytest.mark.parametrize("dt", [0, 1])
def test_ctrl_cnot_cphase_swap_all_pairs(qc, dt):
    n = 6
    g = W.rng(7)
    s, v = mk(qc, n, dt, seed=3)
    ref = as_dt(v, dt).copy()
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            U = W.haar_u2(g, 1)[0]
            s.apply_ctrl(c, t, U)
            O.apply_ctrl(ref, n, c, t, U)
            s.cphase(c, t, 1 + (c + t) % 5)
            O.cphase(ref, n, c, t, 1 + (c + t) % 5)
    got = s.numpy()
    assert np.max(np.abs(got - ref)) <= TOL[dt] * 4
    # permutations are bit-exact
    s2, v2 = mk(qc, n, dt, seed=4)
    r2 = as_dt(v2, dt).copy()
    for c in range(n):
        for t in range(n):
            if c != t:
                s2.cnot(c, t)
                O.cnot(r2, n, c, t)
                s2.swap(c, t)
                O.swap(r2, n, c, t)
    assert np.array_equal(s2.numpy(), r2)


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [12, 18])
def test_ctrl_large(qc, dt, n):
    g = W.rng(n)
    s, v = mk(qc, n, dt, seed=n)
    ref = as_dt(v, dt).copy()
    for (c, t) in [(0, n - 1), (n - 1, 0), (3, 4), (n - 2, 1), (5, n - 3)]:
        U = W.haar_u2(g, 1)[0]
        s.apply_ctrl(c, t, U)
        O.apply_ctrl(ref, n, c, t, U)
        s.cnot(t, c)
        O.cnot(ref, n, t, c)
        s.cphase(c, t, 3)
        O.cphase(ref, n, c, t, 3)
        s.swap(c, t)
        O.swap(ref, n, c, t)
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt] * 4


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [1, 4, 12, 13, 14, 17, 22])
def test_hall_and_layer(qc, dt, n):
    s, v = mk(qc, n, dt, seed=n + 1)
    ref = as_dt(v, dt).copy()
    s.hall()
    O.hall(ref, n)
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt] * max(1, n / 4)
    g = W.rng(n + 5)
    U = W.haar_u2(g, n)
    mask = (1 << n) - 1
    if n > 3:
        mask &= ~(1 << (n // 2))  # one qubit left out
    s.apply_1q_layer(U, mask)
    for q in range(n):
        if (mask >> q) & 1:
            O.apply_1q(ref, n, q, U[q])
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt] * max(1, n / 4)


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 8, 9, 10, 11, 12, 13, 16, 19])
def test_qft_vs_oracle(qc, dt, n):
    s, v = mk(qc, n, dt, seed=50 + n)
    ref = O.qft(as_dt(v, dt).copy(), n)
    s.qft()
    got = s.numpy()
    assert np.max(np.abs(got - ref)) <= TOL[dt] * max(1, n / 4)


@pytest.mark.parametrize("n", [4, 11, 20])
def test_qft_basis_state_analytic(qc, n):
    N = 1 << n
    for m in (0, 1, N // 3, N - 1):
        s = qc.State(n, 0).reset(m)
        s.qft()
        ref = np.exp(2j * np.pi * m * np.arange(N) / N) / math.sqrt(N)
        assert np.max(np.abs(s.numpy() - ref)) <= 1e-12


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n,M", [(3, 1), (8, 2), (12, 3), (16, 8), (17, 1)])
def test_grover_step_vs_literal(qc, dt, n, M):
    marked = W.marked_indices(W.rng(n * 7 + M), n, M)
    s, v = mk(qc, n, dt, seed=n)
    ref = as_dt(v, dt).copy()
    for _ in range(3):
        s.grover_step(marked)
        O.grover_step(ref, n, marked)
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt] * 4
    # a different gate in between invalidates the cached sum
    U = W.haar_u2(W.rng(1), 1)[0]
    s.apply_1q(0, U)
    O.apply_1q(ref, n, 0, U)
    s.grover_step(marked)
    O.grover_step(ref, n, marked)
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt] * 4


def grover_closed(n, marked, k):
    N, M = 2 ** n, len(marked)
    th = math.asin(math.sqrt(M / N))
    v = np.full(N, math.cos((2 * k + 1) * th) / math.sqrt(N - M), dtype=np.complex128)
    v[np.asarray(marked, dtype=np.int64)] = math.sin((2 * k + 1) * th) / math.sqrt(M)
    return v


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n,M", [(10, 1), (13, 2), (14, 8), (15, 1), (20, 8)])
def test_grover_run_closed_form(qc, dt, n, M):
    marked = W.marked_indices(W.rng(1000 + n), n, M)
    k = W.grover_iterations(n) if n <= 15 else 40
    s = qc.State(n, dt)
    s.grover_run(marked, k)
    ref = grover_closed(n, marked, k)
    assert np.max(np.abs(s.numpy() - ref)) <= TOL[dt] * (10 if dt else 1)


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [1, 5, 13, 18])
def test_reductions(qc, dt, n):
    s, v = mk(qc, n, dt, seed=n * 3)
    x = as_dt(v, dt)
    assert abs(s.norm() - O.norm(x, n)) <= 1e-12
    p = s.probs().cpu().numpy()
    pr = O.probs(x, n)
    assert np.array_equal(p, pr)  # same operations, same rounding
    for xm, zm in [(0, 0b11 & ((1 << n) - 1)), (1, 0), ((1 << n) - 1, 1), (0b101 & ((1 << n) - 1), 0b110 & ((1 << n) - 1))]:
        e = s.expect_pauli(xm, zm)
        assert abs(e - O.expect_pauli(x, n, xm, zm)) <= 1e-12


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 7, 14])
def test_expect_pauli_all_pairings(qc, dt, n):
    # x = 0 (diagonal), and x != 0 with its lowest set bit anywhere, both
    # signs of (-1)^{|x&z|} (real or imaginary pair sums), top qubit
    s, v = mk(qc, n, dt, seed=900 + n)
    x_ = as_dt(v, dt)
    g = W.rng(n)
    N = 1 << n
    cases = {(0, 0), (0, N - 1), (N - 1, 0), (N - 1, N - 1), (1 << (n - 1), 1 << (n - 1)), (1 << (n - 1), 0)}
    cases |= {(int(a), int(b)) for a, b in zip(g.integers(0, N, 12), g.integers(0, N, 12))}
    for xm, zm in sorted(cases):
        e = s.expect_pauli(xm, zm)
        ref = O.expect_pauli(x_, n, xm, zm)
        assert abs(e - ref) <= 1e-12, (xm, zm)
        assert e.imag == 0.0  # Hermitian Pauli string: exactly real


def adversarial_amplitudes(g, N, dt):
    """Amplitude bit patterns that stress p = re*re + im*im rounded in
    binary64: short significands (ties when a complex128 square is rounded,
    ties in the sum for complex64), components many binades apart, exact
    zeros, subnormal values, and complex128 values on both sides of 2^-500
    and 2^500."""
    sign = np.where(g.random((N, 2)) < 0.5, -1.0, 1.0)
    if dt == 1:
        e = g.integers(-40, 1, size=(N, 2))
        e[N // 2:] = g.integers(-149, 2, size=(N - N // 2, 2))
        x = np.ldexp(g.random((N, 2)) + 1.0, e)
        short = g.random((N, 2)) < 0.25
        x[short] = np.ldexp(g.integers(4096, 8192, size=short.sum()).astype(np.float64), -12 + e[short])
        x[g.random((N, 2)) < 0.1] = 0.0
        x[:64] = np.ldexp(g.integers(1, 1 << 20, size=(64, 2)).astype(np.float64), -149)  # subnormal
        x = (x * sign).astype(np.float32).astype(np.float64)
    else:
        e = g.integers(-60, 2, size=(N, 2))
        e[: N // 4] = g.integers(-560, 540, size=(N // 4, 2))
        x = np.ldexp(g.random((N, 2)) + 1.0, e)
        # x = M 2^-k with odd M > 2^26.5: the square's 106-bit significand
        # product rounds at an exact tie
        short = g.random((N, 2)) < 0.25
        M = 2 * g.integers(47453133, 1 << 26, size=short.sum()) + 1
        x[short] = np.ldexp(M.astype(np.float64), -27 - g.integers(0, 30, size=short.sum()))
        x[g.random((N, 2)) < 0.1] = 0.0
        x[:8] = [[2.0 ** -500, 2.0 ** -501], [2.0 ** 500, 0.0], [2.0 ** -1074, 1.0], [2.0 ** -1022, 2.0 ** -600],
                 [np.nextafter(2.0 ** -500, 0.0), 0.5], [2.0 ** 501, 0.0], [0.0, 0.0], [1.0, 1.0]]
        x = x * sign
    return x[:, 0] + 1j * x[:, 1]


@pytest.mark.parametrize("dt", [0, 1])
def test_probs_and_weights_adversarial_bits(qc, dt):
    # the probabilities are formed from the IEEE fields with integer
    # operations: every value must equal binary64 re*re + im*im bit for bit,
    # and the sampler's integer weights must follow them
    n = 14
    g = W.rng(4242 + dt)
    v = adversarial_amplitudes(g, 1 << n, dt)
    s, _ = mk(qc, n, dt, vec=v)
    p = s.probs().cpu().numpy()
    pr = O.probs(as_dt(v, dt), n)
    assert np.array_equal(p.view(np.uint64), pr.view(np.uint64))
    # a power-of-two scale keeps every significand: total probability <= 1
    q = np.where(np.abs(v) < 2.0 ** 100, v, 0.0)
    q = q * 2.0 ** -math.ceil(0.5 * math.log2(np.sum(np.abs(q) ** 2)))
    s2, _ = mk(qc, n, dt, vec=q)
    pq = O.probs(as_dt(q, dt), n)
    assert np.sum(pq) <= 1.0
    for shots in (3, 50):
        got = s2.sample(91, shots).cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, O.sample_from_probs(pq, 91, shots))


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [1, 3, 12, 15])
def test_sample_bit_exact(qc, dt, n):
    s, v = mk(qc, n, dt, seed=n + 11)
    p = s.probs().cpu().numpy()
    for seed in (0, 12345, 2 ** 40 + 7):
        got = s.sample(seed, 1000).cpu().numpy().astype(np.uint64)
        ref = O.sample_from_probs(p, seed, 1000)
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n,shots", [(12, 1), (12, 2), (12, 3), (16, 32), (16, 33), (20, 500)])
def test_sample_block_local_and_cdf_paths(qc, dt, n, shots):
    # shots <= 2^n / 2048 rescans one 2048-amplitude block per shot; more
    # shots write the full CDF: both must give the definition's outcomes
    s, v = mk(qc, n, dt, seed=n + 5 * shots)
    p = s.probs().cpu().numpy()
    for seed in (3, 2 ** 33 + 1):
        got = s.sample(seed, shots).cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, O.sample_from_probs(p, seed, shots))


@pytest.mark.parametrize("dt", [0, 1])
def test_sample_chunked_block_scan(qc, dt):
    # 2^24 amplitudes: 8192 block sums, scanned in two chunks of 4096
    n = 24
    g = W.rng(24 + dt)
    v = (g.standard_normal(1 << n) + 1j * g.standard_normal(1 << n)) * np.exp(-np.arange(1 << n) / 2.0 ** 22)
    v /= np.linalg.norm(v)
    s, _ = mk(qc, n, dt, vec=v)
    pr = O.probs(as_dt(v, dt), n)
    assert np.array_equal(s.probs().cpu().numpy(), pr)
    for shots in (5, 8193):  # block-local rescans, then the full integer CDF
        got = s.sample(2 ** 35 + 9, shots).cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, O.sample_from_probs(pr, 2 ** 35 + 9, shots))


@pytest.mark.parametrize("shots", [4, 64])
def test_sample_sparse_state(qc, shots):
    # most 2048-amplitude blocks carry zero weight: the block search must
    # skip runs of equal offsets
    n = 17
    vec = np.zeros(1 << n, dtype=complex)
    for i, a in ((5, 0.3), (40000, 0.5j), (40001, 0.1), (131071, 0.8 - 0.1j)):
        vec[i] = a
    vec /= np.linalg.norm(vec)
    s, _ = mk(qc, n, 0, vec=vec)
    p = s.probs().cpu().numpy()
    got = s.sample(77, shots).cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, O.sample_from_probs(p, 77, shots))
    assert set(got.tolist()) <= {5, 40000, 40001, 131071}


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n,shots", [(1, 5), (11, 1), (12, 3), (16, 33), (20, 1000), (24, 5), (24, 8193)])
def test_probs_sample_one_pass(qc, dt, n, shots):
    # the fused entry point writes what qc_probs writes and draws what
    # qc_sample draws: block-local rescans, the full CDF, one block (n < 11),
    # and the chunked block scan (n = 24)
    s, v = mk(qc, n, dt, seed=3 * n + shots + dt)
    pr = O.probs(as_dt(v, dt), n)
    for seed in (0, 2 ** 35 + 9):
        p, got = s.probs_sample(seed, shots)
        assert np.array_equal(p.cpu().numpy(), pr)
        got = got.cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, O.sample_from_probs(pr, seed, shots))
        assert np.array_equal(got, s.sample(seed, shots).cpu().numpy().astype(np.uint64))
    p, got = s.probs_sample(1, 0)  # no shots: probabilities only
    assert got.numel() == 0 and np.array_equal(p.cpu().numpy(), pr)


def test_probs_sample_rejects_unusable_probabilities(qc):
    n = 13
    vec = np.full(1 << n, 1.5 + 0j)
    s, _ = mk(qc, n, 0, vec=vec)
    with pytest.raises(qc.QCError) as e:
        s.probs_sample(1, 10)
    assert e.value.status == qc.QC_EINVAL


def test_sample_rejects_unusable_probabilities(qc):
    n = 13
    for vec in (np.zeros(1 << n, dtype=complex), np.full(1 << n, 1.5 + 0j), np.full(1 << n, 0.9 + 0j)):
        s, _ = mk(qc, n, 0, vec=vec)
        for shots in (1, 100):
            with pytest.raises(qc.QCError) as e:
                s.sample(1, shots)
            assert e.value.status == qc.QC_EINVAL


def test_renormalize(qc):
    n = 9
    s, v = mk(qc, n, 0, vec=W.random_state(W.rng(2), n) * 1.7)
    nrm = s.renormalize()
    assert abs(nrm - 1.7 ** 2) < 1e-12
    assert abs(s.norm() - 1.0) < 1e-14


def test_invalid_arguments(qc):
    s = qc.State(4, 0)
    bad = [lambda: s.apply_1q(4, np.eye(2, dtype=complex)), lambda: s.apply_ctrl(1, 1, np.eye(2, dtype=complex)),
           lambda: s.cphase(0, 1, 0), lambda: s.swap(2, 2), lambda: s.grover_step([16]),
           lambda: s.grover_step([1, 1]), lambda: s.apply_1q(0, [np.nan] * 8),
           lambda: s.apply_1q_layer(W.haar_u2(W.rng(0), 4), 1 << 4)]
    for f in bad:
        with pytest.raises(qc.QCError) as e:
            f()
        assert e.value.status == qc.QC_EINVAL
    with pytest.raises(qc.QCError):
        qc.qc_state_alloc(0)
    with pytest.raises(qc.QCError):
        qc.qc_state_alloc(35)
    # state unchanged by the rejected calls
    assert abs(s.numpy()[0]) >= 0
