"""Pins for the oracle's log-space Gamma / Dirichlet draws (eq. 4, eq. 19, eq. 28)."""

import numpy as np
import pytest
from scipy import stats

from oracle import philox
from oracle.dirichlet import log_dirichlet_draw, log_gamma_draw


@pytest.mark.parametrize("shape", [0.05, 0.5, 1.0, 2.5, 37.0, 1.0e3, 1.0e6])
def test_gamma_draws_follow_gamma_law(shape):
    """KS test of exp(log G) against the Gamma CDF (log scale for small shapes)."""
    n = 20000
    logg = log_gamma_draw(np.full(n, shape), 42, 0, philox.TAG_THETA, np.arange(n), 3)
    assert np.all(np.isfinite(logg))
    if shape < 1:
        # log of a Gamma(c) variate follows scipy's loggamma(c) law
        p = stats.kstest(logg, stats.loggamma(shape).cdf).pvalue
    else:
        p = stats.kstest(np.exp(logg), stats.gamma(shape).cdf).pvalue
    assert p > 1e-3


def test_dirichlet_moments_match_closed_form():
    """E[theta_u] = a_u / A and Var[theta_u] = a_u (A - a_u) / (A^2 (A + 1))."""
    conc = np.array([0.05, 0.3, 1.0, 4.0, 10.0, 0.05, 2.0])
    A = conc.sum()
    reps = 6000
    draws = np.exp(np.stack([log_dirichlet_draw(conc, 11, 0, philox.TAG_THETA, 7 * r, 0)
                             for r in range(reps)]))
    np.testing.assert_allclose(draws.sum(axis=1), 1.0, rtol=1e-12)
    mean = conc / A
    var = conc * (A - conc) / (A * A * (A + 1))
    se = np.sqrt(var / reps)
    assert np.all(np.abs(draws.mean(axis=0) - mean) < 5 * se)
    assert np.all(np.abs(draws.var(axis=0) / var - 1) < 0.15)


def test_small_shape_draws_do_not_underflow():
    conc = np.full(1000, 0.05)
    lt = log_dirichlet_draw(conc, 5, 0, philox.TAG_THETA, 0, 0)
    assert np.all(np.isfinite(lt))
    assert lt.min() < -50           # Gamma(0.05) variates this small are common
