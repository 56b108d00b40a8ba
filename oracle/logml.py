"""Collapsed log marginal likelihood and its hyper-parameter gradient (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Not a formula of the paper: it is what its appendix terms give once theta
is integrated out of eq. 12 against eq. 28 and pi out of eq. 10, with the
symmetric lambda of eq. 28 generalised to a gene-wise vector beta_u:

  LML(alpha, beta) = K log alpha + lgamma(alpha) - lgamma(alpha + N)
                     + sum_k lgamma(n_k)
                     + sum_k [ lgamma(B) - lgamma(B + T_k)
                               + sum_u (lgamma(beta_u + S_ku) - lgamma(beta_u)) ],

B = sum_u beta_u, T_k = sum_u S_ku; multinomial coefficients (constant in
labels and hyper-parameters) are dropped.  Only non-empty clusters count.
Gradients with respect to the log hyper-parameters:

  d LML / d log alpha  = K + alpha (psi(alpha) - psi(alpha + N))
  d LML / d log beta_u = beta_u sum_k [ psi(B) - psi(B + T_k)
                                        + psi(beta_u + S_ku) - psi(beta_u) ].
"""

import numpy as np
from scipy.special import digamma, gammaln

from .sampler import csr_matrix


def cluster_stats(indptr, indices, data, N, D, labels, K):
    """n_k (K,), S_ku (K, D) of the non-empty clusters among labels in [0, K)."""
    X = csr_matrix(indptr, indices, data, N, D)
    labels = np.asarray(labels, dtype=np.int64)
    n = np.bincount(labels, minlength=K)
    rows = np.repeat(np.arange(N), np.diff(X.indptr))
    S = np.bincount(labels[rows] * D + X.indices, weights=X.data.astype(np.float64),
                    minlength=K * D).reshape(K, D)
    keep = n > 0
    return n[keep].astype(np.float64), np.rint(S[keep])


def log_ml(n, S, log_alpha, log_beta):
    alpha = np.exp(log_alpha)
    beta = np.exp(np.asarray(log_beta, dtype=np.float64))
    K, N = n.size, n.sum()
    B = beta.sum()
    T = S.sum(axis=1)
    return (K * log_alpha + gammaln(alpha) - gammaln(alpha + N) + gammaln(n).sum()
            + (gammaln(B) - gammaln(B + T)).sum()
            + (gammaln(beta[None, :] + S) - gammaln(beta)[None, :]).sum())


def log_ml_grad(n, S, log_alpha, log_beta):
    """(d/d log alpha, d/d log beta) of ``log_ml``."""
    alpha = np.exp(log_alpha)
    beta = np.exp(np.asarray(log_beta, dtype=np.float64))
    K, N = n.size, n.sum()
    B = beta.sum()
    T = S.sum(axis=1)
    g_alpha = K + alpha * (digamma(alpha) - digamma(alpha + N))
    per_gene = (digamma(B) - digamma(B + T)).sum() + (digamma(beta[None, :] + S)
                                                       - digamma(beta)[None, :]).sum(axis=0)
    return g_alpha, beta * per_gene


def eb_step(n, S, log_alpha, log_beta, eta_alpha, eta_beta, max_step):
    """One empirical-Bayes step on (log alpha, log beta) with beta tied across
    genes: gradient ascent on ``log_ml`` (whose log beta is the vector of D
    equal values), each move clamped to [-max_step, max_step].  Returns (log ML
    before the step, new log alpha, new log beta).  The tied gradient is the
    sum of the gene-wise ones (chain rule for a shared log beta)."""
    D = S.shape[1]
    lb = np.full(D, float(log_beta))
    lml = log_ml(n, S, log_alpha, lb)
    g_alpha, g_beta = log_ml_grad(n, S, log_alpha, lb)
    da = min(max_step, max(-max_step, eta_alpha * g_alpha))
    db = min(max_step, max(-max_step, eta_beta * float(np.sum(g_beta))))
    return lml, log_alpha + da, float(log_beta) + db
