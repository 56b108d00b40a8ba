"""Pins for the oracle's collapsed log marginal likelihood, its gradient, and ARI."""

import itertools
import math

import numpy as np

from oracle.ari import adjusted_rand_index
from oracle.logml import cluster_stats, log_ml, log_ml_grad
from oracle.model import log_crp_partition, log_marginal_cluster


def small_problem(seed=0, N=60, D=7, K=4):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 6, size=(N, D)) * (rng.random((N, D)) < 0.6)
    labels = rng.integers(0, K, size=N)
    nz = [np.nonzero(r)[0] for r in x]
    indptr = np.concatenate([[0], np.cumsum([len(z) for z in nz])])
    indices = np.concatenate(nz)
    data = np.concatenate([x[i, z] for i, z in enumerate(nz)])
    return x, labels, indptr, indices, data


def test_symmetric_beta_reduces_to_crp_times_cluster_marginals():
    """With beta_u = lambda for all u, LML = log EPPF + sum_k log f(S_k)."""
    x, labels, indptr, indices, data = small_problem()
    n, S = cluster_stats(indptr, indices, data, x.shape[0], x.shape[1], labels, 4)
    lam, alpha = 0.37, 1.9
    ref = log_crp_partition(n, alpha) + sum(log_marginal_cluster(S[k], lam) for k in range(len(n)))
    got = log_ml(n, S, math.log(alpha), np.full(x.shape[1], math.log(lam)))
    assert abs(got - ref) < 1e-9


def test_empty_clusters_are_not_counted():
    x, labels, indptr, indices, data = small_problem()
    n1, S1 = cluster_stats(indptr, indices, data, x.shape[0], x.shape[1], labels, 4)
    n2, S2 = cluster_stats(indptr, indices, data, x.shape[0], x.shape[1], labels * 2, 8)
    np.testing.assert_array_equal(n1, n2)
    np.testing.assert_array_equal(S1, S2)


def test_gradient_matches_central_finite_differences():
    x, labels, indptr, indices, data = small_problem(seed=1)
    n, S = cluster_stats(indptr, indices, data, x.shape[0], x.shape[1], labels, 4)
    rng = np.random.default_rng(2)
    la = 0.3
    lb = np.log(0.1) + 0.3 * rng.standard_normal(x.shape[1])
    ga, gb = log_ml_grad(n, S, la, lb)
    h = 1e-6
    fa = (log_ml(n, S, la + h, lb) - log_ml(n, S, la - h, lb)) / (2 * h)
    assert abs(ga - fa) < 1e-6 * max(1.0, abs(fa))
    for u in range(x.shape[1]):
        e = np.zeros_like(lb)
        e[u] = h
        fb = (log_ml(n, S, la, lb + e) - log_ml(n, S, la, lb - e)) / (2 * h)
        assert abs(gb[u] - fb) < 1e-5 * max(1.0, abs(fb))


def pair_counting_ari(a, b):
    """ARI from the four pair counts (Steinley 2004 form), by brute force over pairs."""
    n = len(a)
    s11 = s10 = s01 = s00 = 0
    for i, j in itertools.combinations(range(n), 2):
        sa, sb = a[i] == a[j], b[i] == b[j]
        s11 += sa and sb
        s10 += sa and not sb
        s01 += sb and not sa
        s00 += not sa and not sb
    den = (s11 + s10) * (s10 + s00) + (s11 + s01) * (s01 + s00)
    return 1.0 if den == 0 else 2.0 * (s11 * s00 - s10 * s01) / den


def test_ari_matches_brute_force_pair_counting():
    rng = np.random.default_rng(8)
    for _ in range(6):
        a = rng.integers(0, 4, size=60)
        b = np.where(rng.random(60) < 0.6, a, rng.integers(0, 5, size=60))
        assert abs(adjusted_rand_index(a, b) - pair_counting_ari(a, b)) < 1e-12
    assert adjusted_rand_index([0, 0, 1, 1], [5, 5, 2, 2]) == 1.0


# ---------------------------------------------------------------------------
# empirical-Bayes step (beta tied across genes)
# ---------------------------------------------------------------------------
def test_eb_step_tied_gradient_matches_finite_differences():
    """The tied log-beta move is eta times d LML / d(shared log beta), checked
    by a central difference of log_ml along the common log beta; likewise for
    log alpha."""
    from oracle.logml import eb_step
    x, labels, indptr, indices, data = small_problem(seed=3)
    n, S = cluster_stats(indptr, indices, data, x.shape[0], x.shape[1], labels, 4)
    D = x.shape[1]
    la, lb, h = 0.2, math.log(0.3), 1e-6
    lml, la2, lb2 = eb_step(n, S, la, lb, 1.0, 1.0, 1e9)
    fa = (log_ml(n, S, la + h, np.full(D, lb)) - log_ml(n, S, la - h, np.full(D, lb))) / (2 * h)
    fb = (log_ml(n, S, la, np.full(D, lb + h)) - log_ml(n, S, la, np.full(D, lb - h))) / (2 * h)
    assert abs(lml - log_ml(n, S, la, np.full(D, lb))) == 0.0
    assert abs((la2 - la) - fa) < 1e-6 * max(1.0, abs(fa))
    assert abs((lb2 - lb) - fb) < 1e-6 * max(1.0, abs(fb))


def test_eb_step_clamps_and_ascends():
    from oracle.logml import eb_step
    x, labels, indptr, indices, data = small_problem(seed=4)
    n, S = cluster_stats(indptr, indices, data, x.shape[0], x.shape[1], labels, 4)
    D = x.shape[1]
    la, lb = 1.5, math.log(3.0)
    _, la2, lb2 = eb_step(n, S, la, lb, 1e6, 1e6, 0.25)
    assert abs(abs(la2 - la) - 0.25) < 1e-15 and abs(abs(lb2 - lb) - 0.25) < 1e-15
    # small steps go uphill
    prev = log_ml(n, S, la, np.full(D, lb))
    for _ in range(20):
        _, la, lb = eb_step(n, S, la, lb, 1e-3, 1e-3, 0.1)
        cur = log_ml(n, S, la, np.full(D, lb))
        assert cur >= prev - 1e-12
        prev = cur


def test_log_ml_and_gradients_match_the_hand_derived_golden_values():
    """tests/golden/logml_small.txt: exact values derived by hand."""
    import math
    import os
    from fractions import Fraction as F
    from oracle.logml import log_ml, log_ml_grad
    path = os.path.join(os.path.dirname(__file__), "golden", "logml_small.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for case, n, S, alpha, beta, lml, ga, gb in rows:
        n = np.array([float(v) for v in n.split("|")])
        S = np.array([[float(v) for v in r.split(",")] for r in S.split("|")])
        la = math.log(float(F(alpha)))
        lb = np.log(np.array([float(F(v)) for v in beta.split(",")]))
        assert abs(log_ml(n, S, la, lb) - math.log(F(lml))) < 1e-12, case
        g_a, g_b = log_ml_grad(n, S, la, lb)
        assert abs(g_a - float(F(ga))) < 1e-12, case
        np.testing.assert_allclose(g_b, [float(F(v)) for v in gb.split(",")], atol=1e-12)
