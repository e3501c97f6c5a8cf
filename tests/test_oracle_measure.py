"""Pins of the oracle's shot sampling (CPU only): worked examples of the
inverse-CDF rule, and a chi-square test of the histogram of many samples of a
state's marginal against the exact marginal probabilities."""
import numpy as np

from paper_2409_17716_gb300 import workloads as W


def test_inverse_cdf_examples(orc):
    p = np.array([0.25, 0.75])
    assert list(orc.sample(p, [0.1, 0.3, 0.9, 0.0, 0.2499])) == [3, 2]
    p = np.array([0.0, 0.5, 0.0, 0.5])
    assert list(orc.sample(p, [0.0, 0.49, 0.5, 0.99])) == [0, 2, 0, 2]


def test_histogram_chi_square(orc):
    d, n = 3, 5
    psi = W.uniform_state(d, n, seed=4)
    m = orc.marginal(psi, d, n, [3, 1])
    shots = 200000
    u = np.random.default_rng(1).random(shots)
    h = orc.sample(m, u)
    assert h.sum() == shots
    expected = m * shots
    chi2 = float(((h - expected) ** 2 / expected).sum())
    # 8 degrees of freedom: P(chi2 > 30) < 3e-4
    assert chi2 < 30.0, chi2
