"""Pins for the oracle's model quantities: eq. 26 scores, the collapsed cluster
marginal, the CRP partition probability and the split / merge Hastings ratios."""

import itertools
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
from scipy import stats
from scipy.special import gammaln

from oracle.model import (log_crp_partition, log_hastings_merge, log_hastings_split,
                          log_marginal_cluster, multinomial_scores)


def set_partitions(items):
    """All set partitions of a list (restricted-growth enumeration)."""
    if not items:
        yield []
        return
    first, rest = items[0], items[1:]
    for part in set_partitions(rest):
        for i in range(len(part)):
            yield part[:i] + [[first] + part[i]] + part[i + 1:]
        yield [[first]] + part


def test_scores_match_multinomial_pmf_differences():
    """s_ik - s_ik' equals log pi_k - log pi_k' + logpmf(x|theta_k) - logpmf(x|theta_k')."""
    rng = np.random.default_rng(0)
    D, K = 6, 3
    theta = rng.dirichlet(np.ones(D), size=K)
    logpi = np.log(rng.dirichlet(np.ones(K)))
    x = rng.integers(0, 5, size=(4, D))
    s = multinomial_scores(sp.csr_matrix(x.astype(float)), logpi, np.log(theta))
    for i in range(x.shape[0]):
        lp = np.array([stats.multinomial.logpmf(x[i], x[i].sum(), theta[k]) for k in range(K)])
        np.testing.assert_allclose(s[i] - s[i, 0], (logpi + lp) - (logpi[0] + lp[0]), atol=1e-10)


def polya_urn_log_marginal(S, beta):
    """Sequential Polya-urn product: draw the T counts one by one in gene order."""
    D = len(S)
    seen = [0] * D
    total = 0.0
    t = 0
    for u in range(D):
        for _ in range(int(S[u])):
            total += math.log((beta + seen[u]) / (D * beta + t))
            seen[u] += 1
            t += 1
    return total


@pytest.mark.parametrize("beta", [0.05, 0.5, 1.0, 3.0])
def test_cluster_marginal_equals_polya_urn(beta):
    rng = np.random.default_rng(1)
    for _ in range(5):
        S = rng.integers(0, 12, size=7) * (rng.random(7) < 0.7)
        assert abs(log_marginal_cluster(S, beta) - polya_urn_log_marginal(S, beta)) < 1e-10


def test_cluster_marginal_matches_dirichlet_multinomial_pmf():
    """scipy's Dirichlet-multinomial pmf = f(S) * multinomial coefficient."""
    rng = np.random.default_rng(2)
    beta = 0.3
    S = rng.integers(0, 40, size=9)
    T = S.sum()
    coef = gammaln(T + 1) - gammaln(S + 1).sum()
    ref = stats.dirichlet_multinomial.logpmf(S, np.full(9, beta), T) - coef
    assert abs(log_marginal_cluster(S, beta) - ref) < 1e-9


def test_cluster_marginal_two_genes_uniform_prior_is_beta_integral():
    """D = 2, lambda = 1: f = S0! S1! / (T + 1)! exactly."""
    for s0, s1 in [(0, 0), (3, 0), (2, 5), (17, 11)]:
        exact = Fraction(math.factorial(s0) * math.factorial(s1), math.factorial(s0 + s1 + 1))
        assert abs(log_marginal_cluster(np.array([s0, s1]), 1.0) - math.log(exact)) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("alpha", [0.3, 1.0, 2.5])
def test_crp_partition_probabilities_sum_to_one(n, alpha):
    total = sum(math.exp(log_crp_partition([len(b) for b in p], alpha))
                for p in set_partitions(list(range(n))))
    assert abs(total - 1.0) < 1e-12


def crp_sequential(blocks, alpha):
    """CRP seating probability of a labelled partition, customer by customer."""
    owner = {}
    for b, block in enumerate(blocks):
        for i in block:
            owner[i] = b
    n = len(owner)
    sizes = {}
    p = 0.0
    for i in range(n):
        b = owner[i]
        p += math.log((sizes[b] if b in sizes else alpha) / (alpha + i))
        sizes[b] = sizes.get(b, 0) + 1
    return p


def test_split_and_merge_ratios_against_exact_integrals():
    """Two genes, lambda = 1: posterior ratios from CRP seating and Beta integrals."""
    x = np.array([[3, 0], [2, 1], [0, 4], [1, 3], [4, 1]])
    A, B = [0, 1, 4], [2, 3]
    alpha = 0.7

    def log_joint(blocks):
        lp = crp_sequential(blocks, alpha)
        for blk in blocks:
            s0, s1 = x[blk].sum(axis=0)
            lp += math.log(Fraction(math.factorial(s0) * math.factorial(s1),
                                    math.factorial(s0 + s1 + 1)))
        return lp

    ratio = log_joint([A, B]) - log_joint([A + B])
    sum_logq = -1.25
    got = log_hastings_split(len(A), len(B), x[A].sum(0), x[B].sum(0), alpha, 1.0, sum_logq)
    assert abs(got - (ratio - sum_logq)) < 1e-10
    got_m = log_hastings_merge(len(A), len(B), x[A].sum(0), x[B].sum(0), alpha, 1.0)
    assert abs(got_m - (-ratio + (len(A) + len(B) - 2) * math.log(0.5))) < 1e-10


def test_merge_is_reverse_of_split_without_q():
    rng = np.random.default_rng(3)
    Sa, Sb = rng.integers(0, 50, 20), rng.integers(0, 50, 20)
    na, nb = 13, 8
    s = log_hastings_split(na, nb, Sa, Sb, 1.3, 0.1, 0.0)
    m = log_hastings_merge(na, nb, Sa, Sb, 1.3, 0.1)
    assert abs(m + s - (na + nb - 2) * math.log(0.5)) < 1e-9


# ---------------------------------------------------------------------------
# eq. 18 split ratio with theta and pi instantiated
# ---------------------------------------------------------------------------
def _tiny_split(seed=11, n=9, D=4):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 5, size=(n, D))
    side = np.arange(n) % 2
    lam = 0.7
    th = rng.dirichlet(np.full(D, 2.0), size=3)          # theta_k, theta-bar_0, theta-bar_1
    return x, side, lam, th


def test_instantiated_split_eq16_part_matches_scipy_densities():
    """The theta part of eq. 18 (eq. 16) equals the log ratio of the joint
    densities of (theta, x) written with scipy's Dirichlet and multinomial
    densities, cell by cell (an independent route: per-cell pmfs with their
    coefficients, which cancel)."""
    from scipy.stats import dirichlet, multinomial
    from oracle.model import log_hastings_split_instantiated
    x, side, lam, th = _tiny_split()
    D = x.shape[1]
    S0, S1 = x[side == 0].sum(0), x[side == 1].sum(0)
    n0, n1 = int((side == 0).sum()), int((side == 1).sum())
    # remove the eq. 14 and proposal parts: pi_k = 1 makes eq. 14 = log alpha +
    # (n0 - 1) log(n0/n) + (n1 - 1) log(n1/n)
    got = log_hastings_split_instantiated(n0, n1, S0, S1, np.log(th[0]), np.log(th[1]),
                                          np.log(th[2]), 0.0, 1.0, lam, 0.0)
    eq14 = (n0 - 1) * np.log(n0 / (n0 + n1)) + (n1 - 1) * np.log(n1 / (n0 + n1))
    def joint(theta, rows):
        return sum(multinomial.logpmf(r, r.sum(), theta) for r in rows)
    ref = (dirichlet.logpdf(th[1], np.full(D, lam)) + dirichlet.logpdf(th[2], np.full(D, lam))
           + joint(th[1], x[side == 0]) + joint(th[2], x[side == 1])
           - dirichlet.logpdf(th[0], np.full(D, lam)) - joint(th[0], x))
    assert abs((got - eq14) - ref) < 1e-9 * max(1.0, abs(ref))


def test_instantiated_split_special_cases():
    """Equal sub-cluster and cluster parameters leave one Dirichlet density and
    the eq. 14 term; the proposal term enters with a minus sign."""
    from scipy.stats import dirichlet
    from oracle.model import log_hastings_split_instantiated
    x, side, lam, th = _tiny_split(seed=12)
    D = x.shape[1]
    S0, S1 = x[side == 0].sum(0), x[side == 1].sum(0)
    n0 = n1 = 6
    lpk, alpha = np.log(0.3), 1.7
    got = log_hastings_split_instantiated(n0, n1, S0, S1, np.log(th[0]), np.log(th[0]),
                                          np.log(th[0]), lpk, alpha, lam, 0.25)
    eq14 = np.log(alpha) + 2 * (n0 - 1) * (lpk + np.log(0.5)) - (2 * n0 - 1) * lpk
    ref = eq14 + dirichlet.logpdf(th[0], np.full(D, lam)) - 0.25
    assert abs(got - ref) < 1e-10 * max(1.0, abs(ref))


def test_instantiated_split_with_posterior_proposal_densities_is_the_collapsed_ratio():
    """Eq. 16 divided by the densities of drawing theta_k, theta-bar_0 and
    theta-bar_1 from their Dirichlet posteriors (eq. 28) is the theta-integrated
    ratio, whatever the theta values: Dir(theta | beta) Mult(x | theta) /
    Dir(theta | beta + S) is the marginal likelihood of eq. 9's form.  The pi
    part is removed on both sides with the eq. 14 and CRP terms."""
    from scipy.stats import dirichlet
    from scipy.special import gammaln as lg
    from oracle.model import log_hastings_split_instantiated
    rng = np.random.default_rng(31)
    D, lam, alpha = 6, 0.4, 1.3
    S0 = rng.integers(0, 7, size=D).astype(float)
    S1 = rng.integers(0, 7, size=D).astype(float)
    S0[2] = 0.0
    n0, n1 = 5, 8
    th = [rng.dirichlet(np.full(D, 1.0)) for _ in range(3)]     # any point of the simplex
    inst = log_hastings_split_instantiated(n0, n1, S0, S1, np.log(th[0]), np.log(th[1]),
                                           np.log(th[2]), np.log(0.2), alpha, lam, 0.0)
    nk = n0 + n1
    eq14 = (np.log(alpha) + (n0 - 1) * (np.log(0.2) + np.log(n0 / nk))
            + (n1 - 1) * (np.log(0.2) + np.log(n1 / nk)) - (nk - 1) * np.log(0.2))
    q = (dirichlet.logpdf(th[1], lam + S0) + dirichlet.logpdf(th[2], lam + S1)
         - dirichlet.logpdf(th[0], lam + S0 + S1))
    crp = np.log(alpha) + lg(n0) + lg(n1) - lg(nk)
    col = log_hastings_split(n0, n1, S0, S1, alpha, lam, 0.0)
    assert abs((inst - eq14 - q) - (col - crp)) < 1e-9 * max(1.0, abs(col))


def test_hastings_ratios_match_the_hand_derived_golden_values():
    """tests/golden/hastings_small.txt: exact ratios derived by hand for tiny
    split and merge proposals (derivations in the file)."""
    import os
    from fractions import Fraction as F
    path = os.path.join(os.path.dirname(__file__), "golden", "hastings_small.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    assert len(rows) == 5
    for kind, n0, n1, s0, s1, alpha, beta, q, H in rows:
        S0 = np.array([int(v) for v in s0.split(",")], dtype=float)
        S1 = np.array([int(v) for v in s1.split(",")], dtype=float)
        a, b = float(F(alpha)), float(F(beta))
        if kind == "split":
            got = log_hastings_split(int(n0), int(n1), S0, S1, a, b, math.log(F(q)))
        else:
            got = log_hastings_merge(int(n0), int(n1), S0, S1, a, b)
        assert abs(got - math.log(F(H))) < 1e-12, (kind, n0, n1, s0, s1, got, math.log(F(H)))


@pytest.mark.parametrize("beta", [0.1, 0.5, 1.0])
def test_eq18_as_printed_favours_a_split_the_collapsed_ratio_rejects(beta):
    """Eq. 18 with the sweep-style readings (theta drawn from the eq. 28
    posteriors) against the collapsed ratio, for a fair-coin split of ONE
    generating cluster of a 4,000 x 1,000 synthetic matrix: eq. 18 is
    thousands of nats above zero (the extra Dirichlet density of the new
    theta dominates), the collapsed ratio thousands below."""
    from paper_1812_10048_gb300 import synth
    from oracle.model import log_hastings_split_instantiated
    ds = synth.make_dataset(4000, 1000, 4, seed=3)
    X = sp.csr_matrix((ds.data, ds.indices, ds.indptr), shape=(ds.N, ds.D)).toarray()
    rng = np.random.default_rng(0)
    idx = np.nonzero(ds.labels == 0)[0]
    side = rng.integers(0, 2, idx.size)
    S0, S1 = X[idx[side == 0]].sum(0), X[idx[side == 1]].sum(0)
    n0, n1 = int((side == 0).sum()), int((side == 1).sum())

    def logdir(c):
        g = np.maximum(rng.gamma(c), 1e-300)
        return np.log(g) - np.log(g.sum())

    lk, l0, l1 = logdir(beta + S0 + S1), logdir(beta + S0), logdir(beta + S1)
    D = ds.D
    dirichlet_term = gammaln(D * beta) - D * gammaln(beta) + (beta - 1) * (l0.sum() + l1.sum() - lk.sum())
    inst = log_hastings_split_instantiated(n0, n1, S0, S1, lk, l0, l1, np.log(0.25), 1.0, beta, 0.0)
    col = log_hastings_split(n0, n1, S0, S1, 1.0, beta, 0.0)
    assert dirichlet_term > 5000 and inst > 4000 and col < -2500, (dirichlet_term, inst, col)
