"""Pins of the oracle's Shor steps (sec. 5.2): after preparing
2^{-n1/2} sum_j |j>|x^j mod M>, measuring register 2 with outcome k and
Fourier transforming register 1, the register-1 distribution must be the
paper's closed form (Eq. probshor)
  p(n, k) = 1/(2^{n1} D) [sin(D pi n r / 2^{n1}) / sin(pi n r / 2^{n1})]^2,
with r the period of x mod M and D the number of j with x^j = k (mod M); it
reduces to D / 2^{n1} when n r / 2^{n1} is an integer.  No GPU."""
import math

import numpy as np
import pytest

import oracle as O


def period(x, M):
    r, v = 1, x % M
    while v != 1:
        v = (v * x) % M
        r += 1
    return r


def sizes(M):
    n1 = math.ceil(math.log2(M * M))
    n2 = math.ceil(math.log2(M))
    return n1, n2


def probshor(n1, D, r):
    Q = 2 ** n1
    p = np.empty(Q)
    for nn in range(Q):
        den = math.sin(math.pi * nn * r / Q)
        if abs(den) < 1e-12:
            p[nn] = D / Q  # the integer special case
        else:
            p[nn] = (math.sin(D * math.pi * nn * r / Q) / den) ** 2 / (Q * D)
    return p


@pytest.mark.parametrize("M,x", [(15, 7), (21, 2), (15, 2)])
def test_shor_distribution_closed_form(M, x):
    n1, n2 = sizes(M)
    n = n1 + n2
    r = period(x, M)
    psi = O.shor_prepare(n, n2, x, M)
    assert abs(O.norm(psi, n) - 1.0) < 1e-13
    # register 2 outcome k = x^1 mod M (and k = 1)
    for k in (x % M, 1):
        ph = psi.copy()
        pk = O.project(ph, n, 0, n2, k)
        D = sum(1 for j in range(2 ** n1) if pow(x, j, M) == k)
        assert abs(pk - D / 2 ** n1) < 1e-13
        O.qft_range(ph, n, n2, n1)
        p = O.probs(ph, n).reshape(2 ** n1, 2 ** n2)
        assert np.max(np.abs(p[:, np.arange(2 ** n2) != k])) == 0
        ref = probshor(n1, D, r)
        assert np.max(np.abs(p[:, k] - ref)) < 1e-12


def test_qft_range_full_equals_qft():
    n = 7
    x = np.random.default_rng(3).standard_normal(1 << n) + 0j
    a = O.qft_range(x.copy(), n, 0, n)
    b = O.qft(x.copy(), n)
    assert np.max(np.abs(a - b)) < 1e-14


def test_qft_range_is_register_dft():
    # QFT on bits [2, 6) of a 6-qubit state = the DFT along that register
    n, lo, w = 6, 2, 4
    x = np.random.default_rng(4).standard_normal(1 << n) + 1j * np.random.default_rng(5).standard_normal(1 << n)
    got = O.qft_range(x.copy(), n, lo, w)
    T = x.reshape(2 ** w, 2 ** lo)
    ref = (np.fft.ifft(T, axis=0) * math.sqrt(2 ** w)).reshape(-1)
    assert np.max(np.abs(got - ref)) < 1e-13
