"""Model quantities of the Dirichlet-process mixture of multinomials (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation follows the paper: x_i^u counts of gene u in cell i (eq. 26),
symmetric Dirichlet hyper-parameter lambda (eq. 28; ``beta`` here), DP
concentration alpha, V genes (``D`` here), n_k cells and S_k gene sums of
cluster k, sub-cluster quantities with a bar.
"""

import numpy as np
from scipy.special import gammaln


def multinomial_scores(X, logpi, logtheta):
    """Eq. 4 (third line) with the eq. 26 likelihood, in log form.

    s_ik = log pi_k + sum_u x_i^u log theta_k^u, for every cell i (rows of the
    sparse count matrix X) and cluster k (rows of ``logtheta``).  The
    multinomial coefficient of eq. 26 is common to all k and is dropped.
    """
    return np.asarray(X @ logtheta.T) + logpi[None, :]


def log_marginal_cluster(S, beta):
    """Collapsed marginal log f(S) of one cluster with gene sums ``S``.

    Integrating the eq. 26 likelihood of the cluster's cells against the
    eq. 28 prior (the theta part of eq. 12) gives the Dirichlet-multinomial
    normaliser ratio
        log f(S) = lgamma(V lambda) - lgamma(V lambda + T)
                   + sum_u [lgamma(lambda + S_u) - lgamma(lambda)],
    with T = sum_u S_u (multinomial coefficients dropped).  ``S`` may carry
    leading batch axes; the gene axis is the last one.
    """
    S = np.asarray(S, dtype=np.float64)
    D = S.shape[-1]
    T = S.sum(axis=-1)
    return (gammaln(D * beta) - gammaln(D * beta + T)
            + (gammaln(beta + S) - gammaln(beta)).sum(axis=-1))


def log_crp_partition(sizes, alpha):
    """Log probability of a partition with block sizes ``sizes`` under the CRP.

    Eq. 10 integrates the mixing weights out of p(pi) p(c | pi); its printed
    form is garbled (Gamma(alpha) and the pi_{K+1} exponent), so the standard
    exchangeable partition probability function is used:
        log p(c) = K log alpha + lgamma(alpha) - lgamma(alpha + N)
                   + sum_k lgamma(n_k).
    """
    n = np.asarray(sizes, dtype=np.float64)
    N = n.sum()
    return n.size * np.log(alpha) + gammaln(alpha) - gammaln(alpha + N) + gammaln(n).sum()


def log_hastings_split(nbar0, nbar1, Sbar0, Sbar1, alpha, beta, sum_logq):
    """Log Hastings ratio of splitting cluster k into its two sub-clusters.

    Eq. 7 with the likelihood ratio of eq. 9 / eq. 14 / eq. 16 taken with
    theta and pi integrated out (the lgamma-sum form of the collapsed
    model): alpha Gamma(n0) Gamma(n1) / Gamma(n_k) * f(S0) f(S1) / f(S_k).
    The proposal ratio is q(S|S*) / q(S*|S) with q(S|S*) = 1 (the merge back
    is deterministic) and q(S*|S) the product of the eq. 8 probabilities of
    the cells' sub-labels, whose log is ``sum_logq``.
    """
    nk = nbar0 + nbar1
    Sk = np.asarray(Sbar0, dtype=np.float64) + np.asarray(Sbar1, dtype=np.float64)
    return (np.log(alpha) + gammaln(nbar0) + gammaln(nbar1) - gammaln(nk)
            + log_marginal_cluster(Sbar0, beta) + log_marginal_cluster(Sbar1, beta)
            - log_marginal_cluster(Sk, beta) - sum_logq)


def log_hastings_split_instantiated(nbar0, nbar1, Sbar0, Sbar1, logtheta_k, logtheta_0,
                                    logtheta_1, logpi_k, alpha, beta, sum_logq):
    """Log Hastings ratio of splitting cluster k with theta and pi instantiated
    (eq. 7 with the likelihood ratio of eq. 18, i.e. eq. 14 times eq. 16).

    Readings: the split clusters' parameters are the sweep's sub-cluster draws,
    theta_{k0} = theta-bar_{k,0}, theta_{k1} = theta-bar_{k,1}, and the mixing
    weights divide pi_k by the sub-cluster sizes, pi_{kr} = pi_k n-bar_r / n_k.
    Eq. 14: log alpha + (n-bar_0 - 1) log pi_{k0} + (n-bar_1 - 1) log pi_{k1}
    - (n_k - 1) log pi_k.  Eq. 16: one more Dirichlet(beta) density (its
    normaliser lgamma(D beta) - D lgamma(beta) and (beta - 1) sum_u log theta of
    each side) and the multinomial likelihoods sum_u S_u log theta_u of the
    cells of each side (multinomial coefficients cancel).  The proposal term
    is the one of the integrated form.
    """
    S0 = np.asarray(Sbar0, dtype=np.float64)
    S1 = np.asarray(Sbar1, dtype=np.float64)
    lk = np.asarray(logtheta_k, dtype=np.float64)
    l0 = np.asarray(logtheta_0, dtype=np.float64)
    l1 = np.asarray(logtheta_1, dtype=np.float64)
    D = S0.size
    nk = nbar0 + nbar1
    lp0 = logpi_k + np.log(nbar0 / nk)
    lp1 = logpi_k + np.log(nbar1 / nk)
    eq14 = np.log(alpha) + (nbar0 - 1) * lp0 + (nbar1 - 1) * lp1 - (nk - 1) * logpi_k
    prior = gammaln(D * beta) - D * gammaln(beta) + (beta - 1) * (l0.sum() + l1.sum() - lk.sum())
    lik = S0 @ l0 + S1 @ l1 - (S0 + S1) @ lk
    return eq14 + prior + lik - sum_logq


def log_hastings_merge(na, nb, Sa, Sb, alpha, beta):
    """Log Hastings ratio of merging clusters a and b (Section 2.4).

    The likelihood ratio is the inverse of the split ratio above, and eq. 23
    gives the proposal ratio of the randomised merge moves,
    q(S|S*) / q(S*|S) = (1/2)^(n_a + n_b - 2).
    """
    Sab = np.asarray(Sa, dtype=np.float64) + np.asarray(Sb, dtype=np.float64)
    return (-np.log(alpha) + gammaln(na + nb) - gammaln(na) - gammaln(nb)
            + log_marginal_cluster(Sab, beta) - log_marginal_cluster(Sa, beta)
            - log_marginal_cluster(Sb, beta) + (na + nb - 2) * np.log(0.5))
