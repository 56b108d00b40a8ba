"""The Para-DPMM sampler, plain and slow (FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Section 2 of the paper in its order and notation:

* one sweep is the blocked iteration of eq. 4: mixing weights pi from
  p(pi | c, alpha), cluster parameters theta_k from their Dirichlet
  posteriors, sub-cluster parameters theta-bar from eq. 19, then every cell's
  label c_i from pi_k p(x_i | theta_k) (eq. 4, third line; cells are
  conditionally independent given theta and pi, Section 2.2) and its
  sub-label from eq. 8 (Section 2.3, one local Gibbs iteration);
* one ``split_merge`` call runs one of the two MH chains of Section 2.4
  (chosen by a fair coin): every cluster proposes the split given by its
  sub-labels (eq. 7 with the lgamma-sum likelihood ratio and the eq. 8
  proposal probability), or clusters are paired at random and each pair
  proposes a merge (eq. 7 with the eq. 23 proposal ratio).

Readings where the paper is silent or garbled (each one is the same on the
CUDA side):

* restricted Gibbs by default: labels range over the K existing clusters
  only; new clusters come from splits (Section 2.2-2.3).  pi_{K+1} is drawn
  but unused.  With ``open_new_cluster`` the K+1 candidate of eq. 4 is kept:
  the sweep treats it as one more cluster without cells (its theta and
  theta-bar are therefore drawn from the Dirichlet(lambda) prior and its
  weight is pi_{K+1}), all cells that choose it form one new cluster, and
  there is no candidate when K = kmax;
* eq. 8's n-bar_{r,not i} in a parallel sweep: the sweep-start sub-cluster
  count minus the indicator that cell i sat in (c_i, r) at sweep start and
  keeps its cluster; if both weights are zero they are taken as equal;
* lambda-bar = lambda;
* after the label update, empty clusters are removed with survivors keeping
  their relative order; a cluster with two or more cells and an empty
  sub-cluster redraws its cells' sub-labels as fair coins;
* ``local_iters`` local Gibbs iterations per sweep (default 1, the paper's
  choice): iterations after the first hold the labels, redraw theta-bar
  (eq. 19) and then the sub-labels (eq. 8), with their own Philox tags;
* the split proposal probability q(S*|S) is the product of the eq. 8
  probabilities of the latest local Gibbs iteration (a random re-initialisation contributes
  (1/2)^n; sub-labels set by a merge contribute 1);
* a split moves sub-cluster 1 of cluster k to the new index K + j (j-th
  accepted split, ascending k); a merge of a < b keeps index a, with the
  cells of a as sub-cluster 0 and those of b as sub-cluster 1;
* ties in a Gumbel argmax go to the lowest index; a move is accepted iff
  log u < log H.
"""

import numpy as np
import scipy.sparse as sp
from scipy.special import logsumexp

from . import philox
from .dirichlet import log_gamma_draw
from .model import log_hastings_merge, log_hastings_split, multinomial_scores

LOG_HALF = np.log(0.5)


def csr_matrix(indptr, indices, data, N, D):
    """Cells x genes sparse count matrix (integer values)."""
    return sp.csr_matrix((np.asarray(data, dtype=np.int64), np.asarray(indices, dtype=np.int64),
                          np.asarray(indptr, dtype=np.int64)), shape=(N, D))


def sufficient_stats(X, labels, sub, K):
    """n-bar[k][r] and S-bar[k][r][u] (exact integers) by direct counting."""
    N, D = X.shape
    labels = np.asarray(labels, dtype=np.int64)
    sub = np.asarray(sub, dtype=np.int64)
    nsub = np.bincount(labels * 2 + sub, minlength=2 * K).reshape(K, 2)
    rows = np.repeat(np.arange(N), np.diff(X.indptr))
    slot = (labels[rows] * 2 + sub[rows]) * D + X.indices
    Ssub = np.bincount(slot, weights=X.data.astype(np.float64), minlength=2 * K * D)
    return nsub.astype(np.int64), np.rint(Ssub).astype(np.int64).reshape(K, 2, D)


def draw_pi(nk, alpha, seed, chain_id, t):
    """Eq. 4, first line: (pi_1..pi_K, pi_{K+1}) ~ Dirichlet(n_1, .., n_K, alpha), in log."""
    shape = np.concatenate([np.asarray(nk, dtype=np.float64), [float(alpha)]])
    logg = log_gamma_draw(shape, seed, chain_id, philox.TAG_PI, np.arange(shape.size), t)
    return logg - logsumexp(logg)


def draw_theta(Ssub, beta, seed, chain_id, t):
    """Eq. 4 (second line) and eq. 19: log theta_k, log theta-bar_{k,0}, log theta-bar_{k,1}.

    Row 3k + p holds cluster k's parameters (p = 0) and its sub-clusters'
    (p = 1, 2), each drawn from Dirichlet(lambda + gene sums).
    """
    K, _, D = Ssub.shape
    conc = np.empty((3 * K, D))
    conc[0::3] = beta + Ssub[:, 0, :] + Ssub[:, 1, :]
    conc[1::3] = beta + Ssub[:, 0, :]
    conc[2::3] = beta + Ssub[:, 1, :]
    index = np.arange(3 * K * D)                      # row * D + u
    logg = log_gamma_draw(conc.ravel(), seed, chain_id, philox.TAG_THETA, index, t).reshape(3 * K, D)
    return logg - logsumexp(logg, axis=1, keepdims=True)


def label_gumbels(N, K, seed, chain_id, t):
    """Gumbel noise g_ik for the eq. 4 label draw (tag 0, word k % 4 of call k // 4)."""
    g = np.empty((N, K))
    cells = np.arange(N)
    for j in range((K + 3) // 4):
        w = philox.stream_words(seed, chain_id, philox.TAG_LABEL, cells, t, j)
        u = philox.word_to_uniform(w)
        take = min(4, K - 4 * j)
        g[:, 4 * j:4 * j + take] = philox.uniform_to_gumbel(u[:, :take])
    return g


def assign(X, logpi, logtheta, labels_old, sub_old, nsub, seed, chain_id, t):
    """Label and sub-label draw of one sweep, given pi and theta.

    Returns new labels, new sub-labels, log q_i (the log eq. 8 probability of
    each cell's drawn sub-label) and the eq. 4 scores s_ik (without noise).
    """
    N = X.shape[0]
    K = logpi.size - 1
    Xf = X.astype(np.float64)
    scores = multinomial_scores(Xf, logpi[:K], logtheta[0::3])
    labels = np.argmax(scores + label_gumbels(N, K, seed, chain_id, t), axis=1)

    # eq. 8: sub-cluster weights n-bar_{r, not i} and likelihoods under theta-bar_r
    cells = np.arange(N)
    lik = np.stack([np.asarray(Xf @ logtheta[1::3].T)[cells, labels],
                    np.asarray(Xf @ logtheta[2::3].T)[cells, labels]], axis=1)
    stays = labels == labels_old
    w = np.stack([nsub[labels, 0] - (stays & (sub_old == 0)),
                  nsub[labels, 1] - (stays & (sub_old == 1))], axis=1)
    sub, logq = eq8_draw(w, lik, seed, chain_id, philox.TAG_SUBLABEL, t)
    return labels.astype(np.int64), sub, logq, scores


def eq8_draw(w, lik, seed, chain_id, tag, t):
    """Eq. 8 by Gumbel-max: weights w[i, r] = n-bar_{r, not i} (both zero: taken
    as equal), likelihood factors lik[i, r] = log p(x_i | theta-bar_r), Gumbels
    from words 0, 1 of counter (i, t, tag, 0).  Returns the sub-labels and
    log q_i, the log eq. 8 probability of each drawn sub-label."""
    w = np.asarray(w, dtype=np.float64).copy()
    w[w.sum(axis=1) == 0] = 1.0
    with np.errstate(divide="ignore"):
        tr = np.log(w) + lik
    cells = np.arange(w.shape[0])
    words = philox.stream_words(seed, chain_id, tag, cells, t, 0)
    h = philox.uniform_to_gumbel(philox.word_to_uniform(words[:, :2]))
    sub = (tr[:, 1] + h[:, 1] > tr[:, 0] + h[:, 0]).astype(np.int64)
    logq = tr[cells, sub] - np.logaddexp(tr[:, 0], tr[:, 1])
    return sub, logq


def compact(labels, K, *per_cluster):
    """Remove empty clusters; survivors keep their relative order."""
    nk = np.bincount(labels, minlength=K)
    keep = nk > 0
    newidx = np.cumsum(keep) - 1
    return newidx[labels], int(keep.sum()), [np.asarray(a)[keep] for a in per_cluster]


def fair_coin_sublabels(cells, seed, chain_id, step, kind):
    """Random sub-labels: 1 if the tag-7 uniform is below 1/2, else 0."""
    w = philox.stream_words(seed, chain_id, philox.TAG_SUBINIT, cells, step, kind)[..., 0]
    return (philox.word_to_uniform(w) < 0.5).astype(np.int64)


class Sampler:
    """FP64 Para-DPMM chain over a cells x genes CSR count matrix."""

    def __init__(self, indptr, indices, data, N, D, alpha, beta, seed=42, chain_id=0,
                 kmax=256, split_q=True, open_new_cluster=False, local_iters=1):
        self.X = csr_matrix(indptr, indices, data, N, D)
        self.N, self.D = int(N), int(D)
        self.alpha, self.beta = float(alpha), float(beta)
        self.seed, self.chain_id, self.kmax = int(seed), int(chain_id), int(kmax)
        self.split_q = bool(split_q)
        self.open_new_cluster = bool(open_new_cluster)
        if not 1 <= int(local_iters) <= philox.LOCAL_MAX_ITERS:
            raise ValueError("local_iters must be in [1, %d]" % philox.LOCAL_MAX_ITERS)
        self.local_iters = int(local_iters)
        self.K = 1
        self.labels = np.zeros(self.N, dtype=np.int64)
        self.sub = fair_coin_sublabels(np.arange(self.N), self.seed, self.chain_id, 0,
                                       philox.SUBINIT_INIT)
        self.sumlogq = np.array([self.N * LOG_HALF])
        self.t = 0
        self.m = 0
        self.capacity_rejects = 0

    # -- state -------------------------------------------------------------
    def stats(self):
        return sufficient_stats(self.X, self.labels, self.sub, self.K)

    def set_state(self, labels, sub, K, t=None, m=None, sumlogq=None):
        self.labels = np.asarray(labels, dtype=np.int64).copy()
        self.sub = np.asarray(sub, dtype=np.int64).copy()
        self.K = int(K)
        if t is not None:
            self.t = int(t)
        if m is not None:
            self.m = int(m)
        nsub, _ = self.stats()
        self.sumlogq = (np.asarray(sumlogq, dtype=np.float64).copy() if sumlogq is not None
                        else nsub.sum(axis=1) * LOG_HALF)

    # -- one sweep (eq. 4 + eq. 8 + bookkeeping) ---------------------------
    def draw_params(self):
        """pi and theta of eq. 4 for the sweep's clusters: the K current ones,
        plus the K+1 candidate (a cluster without cells) when it is open.
        Returns log pi with one entry per cluster and a last entry for the
        unused remainder (-inf when the candidate takes pi_{K+1})."""
        nsub, Ssub = self.stats()
        logpi = draw_pi(nsub.sum(axis=1), self.alpha, self.seed, self.chain_id, self.t)
        if self.open_new_cluster and self.K < self.kmax:
            Ssub = np.concatenate([Ssub, np.zeros((1, 2, self.D), dtype=Ssub.dtype)])
            logpi = np.concatenate([logpi, [-np.inf]])
        logtheta = draw_theta(Ssub, self.beta, self.seed, self.chain_id, self.t)
        return logpi, logtheta

    def assign_and_update(self, logpi, logtheta):
        Ks = logpi.size - 1                 # the sweep's clusters (K, or K + 1 when open)
        nsub = np.zeros((Ks, 2), dtype=np.int64)
        nsub[:self.K] = self.stats()[0]
        labels, sub, logq, _ = assign(self.X, logpi, logtheta, self.labels, self.sub, nsub,
                                      self.seed, self.chain_id, self.t)
        sumlogq = np.bincount(labels, weights=logq, minlength=Ks)
        labels, self.K, (sumlogq,) = compact(labels, Ks, sumlogq)
        self.labels, self.sub, self.sumlogq = labels, sub, sumlogq
        self._reset_empty_subclusters()
        self.t += 1

    def sweep(self):
        logpi, logtheta = self.draw_params()
        self.assign_and_update(logpi, logtheta)
        for j in range(1, self.local_iters):
            self.local_gibbs(j)

    def local_gibbs(self, j):
        """Local Gibbs iteration j >= 1 after the sweep just made (Section 2.3):
        labels held, theta-bar of every sub-cluster drawn from eq. 19 given the
        current sub-labels, then every sub-label drawn from eq. 8.  A
        sub-cluster that empties stays empty until the next sweep's
        compaction; the split proposal term becomes this iteration's log q."""
        t = self.t - 1                           # the sweep's own counter
        nsub, Ssub = self.stats()
        K, D = self.K, self.D
        conc = (self.beta + Ssub).reshape(2 * K, D)           # row 2k + r
        rows = (3 * np.arange(K)[:, None] + 1 + np.arange(2)[None, :]).ravel()
        index = (rows[:, None] * D + np.arange(D)[None, :]).ravel()
        logg = log_gamma_draw(conc.ravel(), self.seed, self.chain_id, philox.tag_local_theta(j),
                              index, t).reshape(2 * K, D)
        logtb = logg - logsumexp(logg, axis=1, keepdims=True)
        Xf = self.X.astype(np.float64)
        cells = np.arange(self.N)
        lik = np.stack([np.asarray(Xf @ logtb[0::2].T)[cells, self.labels],
                        np.asarray(Xf @ logtb[1::2].T)[cells, self.labels]], axis=1)
        w = nsub[self.labels] - np.stack([self.sub == 0, self.sub == 1], axis=1)
        self.sub, logq = eq8_draw(w, lik, self.seed, self.chain_id, philox.tag_local_sub(j), t)
        self.sumlogq = np.bincount(self.labels, weights=logq, minlength=K)
        return logtb

    def _reset_empty_subclusters(self):
        nsub, _ = self.stats()
        nk = nsub.sum(axis=1)
        need = (nk >= 2) & ((nsub[:, 0] == 0) | (nsub[:, 1] == 0))
        if need.any():
            cells = np.nonzero(need[self.labels])[0]
            self.sub[cells] = fair_coin_sublabels(cells, self.seed, self.chain_id, self.t,
                                                  philox.SUBINIT_RESET)
            self.sumlogq[need] = nk[need] * LOG_HALF

    # -- split / merge (Sections 2.3-2.4) ------------------------------------
    def coin_is_split(self):
        w = philox.stream_words(self.seed, self.chain_id, philox.TAG_MOVE, 0, self.m, 0)[0]
        return bool(philox.word_to_uniform(w) < 0.5)

    def split_log_hastings(self):
        """log H for every cluster with two non-empty sub-clusters (NaN otherwise)."""
        nsub, Ssub = self.stats()
        out = np.full(self.K, np.nan)
        for k in range(self.K):
            if nsub[k, 0] >= 1 and nsub[k, 1] >= 1:
                out[k] = log_hastings_split(nsub[k, 0], nsub[k, 1], Ssub[k, 0], Ssub[k, 1],
                                            self.alpha, self.beta,
                                            self.sumlogq[k] if self.split_q else 0.0)
        return out

    def merge_pairs(self):
        w = philox.stream_words(self.seed, self.chain_id, philox.TAG_PAIR,
                                np.arange(self.K), self.m, 0)[:, 0]
        order = np.lexsort((np.arange(self.K), w))
        return [(int(min(order[2 * p], order[2 * p + 1])), int(max(order[2 * p], order[2 * p + 1])))
                for p in range(self.K // 2)]

    def merge_log_hastings(self, pairs):
        nsub, Ssub = self.stats()
        nk, S = nsub.sum(axis=1), Ssub.sum(axis=1)
        return np.array([log_hastings_merge(nk[a], nk[b], S[a], S[b], self.alpha, self.beta)
                         for a, b in pairs])

    def split_merge(self, mode=0):
        """One move of the split chain (mode 1), the merge chain (2) or a coin (0).

        Returns the number of accepted moves.
        """
        do_split = self.coin_is_split() if mode == 0 else mode == 1
        accepted = self._split() if do_split else self._merge()
        self.m += 1
        return accepted

    def _split(self):
        logH = self.split_log_hastings()
        nsub, _ = self.stats()
        acc = []
        for k in range(self.K):
            if np.isnan(logH[k]):
                continue
            w = philox.stream_words(self.seed, self.chain_id, philox.TAG_MOVE, k + 1, self.m, 0)[0]
            if np.log(philox.word_to_uniform(w)) < logH[k]:
                if self.K + len(acc) < self.kmax:
                    acc.append(k)
                else:
                    self.capacity_rejects += 1
        if not acc:
            return 0
        sumlogq = np.concatenate([self.sumlogq, np.zeros(len(acc))])
        touched = np.zeros(self.N, dtype=bool)
        for j, k in enumerate(acc):
            new = self.K + j
            in_k = self.labels == k
            touched |= in_k
            self.labels[in_k & (self.sub == 1)] = new
            sumlogq[k] = nsub[k, 0] * LOG_HALF
            sumlogq[new] = nsub[k, 1] * LOG_HALF
        cells = np.nonzero(touched)[0]
        self.sub[cells] = fair_coin_sublabels(cells, self.seed, self.chain_id, self.m,
                                              philox.SUBINIT_SPLIT)
        self.K += len(acc)
        self.sumlogq = sumlogq
        return len(acc)

    def _merge(self):
        pairs = self.merge_pairs()
        if not pairs:
            return 0
        logH = self.merge_log_hastings(pairs)
        n_acc = 0
        for (a, b), lh in zip(pairs, logH):
            w = philox.stream_words(self.seed, self.chain_id, philox.TAG_MERGE, a, self.m, 0)[0]
            if np.log(philox.word_to_uniform(w)) < lh:
                in_a, in_b = self.labels == a, self.labels == b
                self.sub[in_a] = 0
                self.sub[in_b] = 1
                self.labels[in_b] = a
                self.sumlogq[a] = 0.0
                n_acc += 1
        if n_acc:
            self.labels, self.K, (self.sumlogq,) = compact(self.labels, self.K, self.sumlogq)
        return n_acc
