"""Pins of the seeded sampler: Philox4x32-10 known answers, the integer CDF on
hand-computed cases, the C (linear scan) and numpy (bisection) forms agreeing,
and a chi-squared check of the Born-rule histogram (no GPU)."""
import json
import os

import numpy as np
import scipy.stats

import oracle as O
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    kat = json.load(open(os.path.join(GOLD, "philox4x32_10_kat.json")))
    for c in kat["cases"]:
        ctr = [int(x, 16) for x in c["ctr"]]
        key = [int(x, 16) for x in c["key"]]
        assert list(O.philox4x32_10(ctr, key)) == [int(x, 16) for x in c["out"]]


def test_integer_cdf_hand_case():
    p = np.array([0.25, 0.0, 0.5, 0.25])
    cdf = O.integer_cdf(p)
    q = 1 << 62
    assert list(cdf) == [q // 4, q // 4, 3 * q // 4, q]


def test_sampler_targets_select_by_definition():
    # with p = (1/2, 1/2) the outcome is 1 exactly when r >= 2^63
    p = np.array([0.5, 0.5])
    out = O.sample_from_probs(p, seed=77, shots=200)
    key = (77, 0)
    for s in range(200):
        x = O.philox4x32_10((s, 0, 0, 0), key)
        r = (x[0] << 32) | x[1]
        assert int(out[s]) == (1 if r >= (1 << 63) else 0)


def test_c_and_numpy_sampler_agree():
    for n in (1, 4, 9):
        x = W.random_state(W.rng(n), n)
        p = O.probs(x, n)
        a = O.sample_from_probs(p, seed=1234 + n, shots=300)
        b = O.sample_from_probs_c(p, n, seed=1234 + n, shots=300)
        assert np.array_equal(a, b)


def test_zero_probability_never_sampled():
    p = np.zeros(16)
    p[[3, 11]] = 0.5
    out = O.sample_from_probs(p, seed=5, shots=2000)
    assert set(out.tolist()) <= {3, 11}


def test_chi_squared_histogram():
    n = 5
    x = W.random_state(W.rng(42), n)
    p = O.probs(x, n)
    shots = 200000
    out = O.sample_from_probs(p, seed=9, shots=shots)
    hist = np.bincount(out.astype(np.int64), minlength=1 << n)
    chi2, pval = scipy.stats.chisquare(hist, p / p.sum() * shots)
    assert pval > 1e-4
