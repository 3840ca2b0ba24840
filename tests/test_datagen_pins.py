"""Pins of the synthetic-data generators against the laws they draw from.

The compound Poisson-gamma generator (the paper's Sec. 4 observation model
for powers 1 < p < 2, used for the p = 1.5 workloads) is written from its
definition: N ~ Poisson(lam), v = the sum of N Gamma(alpha, scale) draws.
Checked against what that law fixes: the mean mu, the variance phi mu^p, the
mass exp(-lam) at zero, and the whole distribution function -- the Poisson
mixture of scipy gamma CDFs -- within the sampling error of 2e5 draws.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1506_01418_gb300 import datagen


@pytest.mark.parametrize("mu,p,phi", [(2.0, 1.5, 1.3), (0.4, 1.5, 1.0), (7.0, 1.2, 0.6),
                                      (1.0, 1.8, 2.0)])
def test_compound_poisson_gamma_law(mu, p, phi):
    n = 200_000
    g = np.random.Generator(np.random.Philox(int(100 * mu + 10 * p)))
    v = datagen.compound_poisson_gamma(np.full(n, mu), p, phi, g)
    lam, alpha, scale = datagen.compound_poisson_gamma_params(mu, p, phi)
    var = phi * mu ** p
    # mean and zero mass within 4 standard errors
    assert abs(v.mean() - mu) < 4 * math.sqrt(var / n)
    p0 = math.exp(-lam)
    assert abs((v == 0).mean() - p0) < 4 * math.sqrt(p0 * (1 - p0) / n) + 1e-12
    # variance within 4 standard errors (fourth central moment from the sample)
    m4 = np.mean((v - mu) ** 4)
    assert abs(v.var() - var) < 4 * math.sqrt((m4 - var ** 2) / n)
    # the distribution function: P(v <= x) = sum_k Poisson(k; lam) GammaCDF(x; k alpha, scale)
    xs = np.quantile(v[v > 0], np.linspace(0.02, 0.98, 25))
    k = np.arange(1, 400)
    w = stats.poisson.pmf(k, lam)
    for x in xs:
        F = p0 + np.sum(w * stats.gamma.cdf(x, a=k * alpha, scale=scale))
        assert abs(np.mean(v <= x) - F) < 2.0 / math.sqrt(n), (x, F)


def test_compound_poisson_gamma_params_are_the_law_of_the_sum():
    """lam, alpha and scale reproduce mean lam alpha scale = mu and variance
    lam alpha (alpha + 1) scale^2 = phi mu^p (the compound Poisson moments)."""
    for mu, p, phi in ((2.0, 1.5, 1.3), (0.05, 1.1, 0.7), (30.0, 1.9, 3.0)):
        lam, alpha, scale = datagen.compound_poisson_gamma_params(mu, p, phi)
        assert lam * alpha * scale == pytest.approx(mu, rel=1e-12)
        assert lam * alpha * (alpha + 1) * scale ** 2 == pytest.approx(phi * mu ** p, rel=1e-12)


def test_dense_compound_poisson_has_zeros_and_the_model_mean():
    V, Wt, Ht = datagen.dense_compound_poisson(200, 150, 4, seed=5, p=1.5, phi=1.0)
    M = Wt @ Ht
    lam, _, _ = datagen.compound_poisson_gamma_params(M, 1.5, 1.0)
    zeros = (V == 0)
    assert zeros.any() and V.min() >= 0
    assert abs(zeros.mean() - np.exp(-lam).mean()) < 4 * math.sqrt(0.25 / V.size)
    # E[v - mu] = 0 and Var = phi mu^p, entry by entry: the standardised mean
    z = (V - M) / np.sqrt(M ** 1.5)
    assert abs(z.mean()) < 4 / math.sqrt(V.size)
    assert abs((z ** 2).mean() - 1.0) < 0.05
