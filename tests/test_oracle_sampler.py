"""Pins for the oracle sampler: the eq. 4 label draw, the eq. 8 sub-label draw,
the bookkeeping invariants, and the chain's stationary law on tiny data."""

import math

import numpy as np
import pytest
from scipy import stats
from scipy.special import logsumexp

from oracle import philox
from oracle.model import log_crp_partition, log_marginal_cluster
from oracle.sampler import Sampler, assign, csr_matrix, sufficient_stats

from .test_oracle_model import set_partitions


def replicated_rows(row, n):
    row = np.asarray(row)
    nz = np.nonzero(row)[0]
    indptr = np.arange(n + 1) * nz.size
    return indptr, np.tile(nz, n), np.tile(row[nz], n)


def test_label_draw_is_categorical_softmax():
    """Gumbel-max over s_ik + g_ik draws k with probability softmax(s_i)."""
    rng = np.random.default_rng(4)
    D, K, n = 5, 6, 30000
    row = np.array([3, 0, 1, 4, 2])
    logtheta = np.log(rng.dirichlet(np.ones(D), size=3 * K))
    logpi = np.log(rng.dirichlet(np.ones(K + 1)))
    X = csr_matrix(*replicated_rows(row, n), n, D)
    nsub = np.full((K, 2), 10)
    labels, _, _, scores = assign(X, logpi, logtheta, np.zeros(n, np.int64), np.zeros(n, np.int64),
                                  nsub, 42, 0, 9)
    p = np.exp(scores[0] - logsumexp(scores[0]))
    counts = np.bincount(labels, minlength=K)
    ok = p * n > 5
    assert ok.sum() >= 2
    obs = np.append(counts[ok], counts[~ok].sum())
    exp = np.append(p[ok] * n, p[~ok].sum() * n)
    if exp[-1] == 0:
        obs, exp = obs[:-1], exp[:-1]
    assert stats.chisquare(obs, exp).pvalue > 1e-4


def test_sublabel_draw_follows_eq8_and_logq_is_its_log_probability():
    rng = np.random.default_rng(5)
    D, K, n = 4, 2, 40000
    row = np.array([2, 1, 0, 3])
    logtheta = np.log(rng.dirichlet(np.ones(D) * 2, size=3 * K))
    logpi = np.log(np.array([0.5, 0.49, 0.01]))
    X = csr_matrix(*replicated_rows(row, n), n, D)
    nsub = np.array([[7, 3], [2, 9]])
    labels_old = np.zeros(n, np.int64)
    sub_old = (np.arange(n) % 2).astype(np.int64)
    labels, sub, logq, _ = assign(X, logpi, logtheta, labels_old, sub_old, nsub, 42, 0, 2)
    lik = np.array([[row @ logtheta[3 * k + 1], row @ logtheta[3 * k + 2]] for k in range(K)])
    for k in range(K):
        for so in (0, 1):
            sel = (labels == k) & (sub_old == so)
            if sel.sum() < 500:
                continue
            w = nsub[k].astype(float) - (np.array([0, 1]) == so) * (k == 0)
            p1 = w[1] * math.exp(lik[k, 1]) / (w[0] * math.exp(lik[k, 0]) + w[1] * math.exp(lik[k, 1]))
            m = sel.sum()
            got = sub[sel].mean()
            assert abs(got - p1) < 5 * math.sqrt(p1 * (1 - p1) / m) + 1e-9
            expect_logq = np.where(sub[sel] == 1, math.log(p1), math.log(1 - p1))
            np.testing.assert_allclose(logq[sel], expect_logq, atol=1e-9)


def test_sweep_and_moves_keep_invariants(tiny_dataset):
    ds = tiny_dataset
    s = Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, seed=3)
    colsum = np.bincount(ds.indices, weights=ds.data, minlength=ds.D)
    for it in range(12):
        s.sweep()
        s.split_merge(0)
        nsub, Ssub = s.stats()
        assert s.labels.min() >= 0 and s.labels.max() < s.K
        assert set(np.unique(s.sub)) <= {0, 1}
        assert nsub.sum() == ds.N and np.all(nsub.sum(axis=1) > 0)
        np.testing.assert_array_equal(Ssub.sum(axis=(0, 1)), colsum)
        assert s.sumlogq.shape == (s.K,) and np.all(s.sumlogq <= 0)
    assert s.t == 12 and s.m == 12


def test_forced_split_and_merge_moves():
    """Huge alpha accepts every split; tiny alpha accepts every identical-data merge."""
    rng = np.random.default_rng(6)
    n, D = 40, 3
    x = rng.integers(0, 4, size=(n, D))
    indptr = np.arange(n + 1) * D
    s = Sampler(indptr, np.tile(np.arange(D), n), x.ravel(), n, D, alpha=1e300, beta=1.0, seed=1)
    sub0 = s.sub.copy()
    assert s.split_merge(1) == 1
    assert s.K == 2
    np.testing.assert_array_equal(s.labels, sub0)        # sub-cluster 1 became cluster 1
    s.alpha = 1e-300
    assert s.split_merge(2) == 1
    assert s.K == 1 and np.all(s.labels == 0)
    np.testing.assert_array_equal(s.sub, sub0)           # a -> sub 0, b -> sub 1


def test_capacity_limit_counts_rejected_splits():
    rng = np.random.default_rng(7)
    n, D = 30, 2
    x = rng.integers(0, 4, size=(n, D))
    s = Sampler(np.arange(n + 1) * D, np.tile(np.arange(D), n), x.ravel(), n, D,
                alpha=1e300, beta=1.0, seed=1, kmax=1)
    assert s.split_merge(1) == 0 and s.K == 1 and s.capacity_rejects == 1


def exact_partition_posterior(x, alpha, beta):
    n = x.shape[0]
    parts = list(set_partitions(list(range(n))))
    logp = np.array([log_crp_partition([len(b) for b in p], alpha)
                     + sum(log_marginal_cluster(x[b].sum(axis=0), beta) for b in p) for p in parts])
    return parts, np.exp(logp - logsumexp(logp))


def canonical(labels):
    seen, out = {}, []
    for l in labels:
        out.append(seen.setdefault(int(l), len(seen)))
    return tuple(out)


def partition_key(p, n):
    lab = np.empty(n, dtype=int)
    for b, blk in enumerate(p):
        lab[blk] = b
    return canonical(lab)


TINY_X = np.array([[4, 0, 1], [3, 1, 0], [0, 3, 2], [1, 4, 1], [2, 2, 2]])
# six cells, three genes: 203 partitions, 31 of them into two blocks
SIX_X = np.array([[4, 0, 1], [3, 1, 0], [0, 3, 2], [1, 4, 1], [2, 2, 2], [0, 1, 5]])


def collapsed_gibbs_state(x, alpha, beta, iters, rng):
    """Neal (2000) Algorithm 3: textbook collapsed Gibbs from one cluster;
    returns the partition after `iters` passes (validates the enumerator)."""
    n = x.shape[0]
    lab = np.zeros(n, dtype=int)
    for _ in range(iters):
        for i in range(n):
            lab[i] = -1
            blocks = sorted(set(lab[lab >= 0]))
            lp = []
            for b in blocks:
                S = x[lab == b].sum(axis=0)
                lp.append(math.log((lab == b).sum())
                          + log_marginal_cluster(S + x[i], beta) - log_marginal_cluster(S, beta))
            lp.append(math.log(alpha) + log_marginal_cluster(x[i], beta)
                      - log_marginal_cluster(np.zeros_like(x[i]), beta))
            lp = np.array(lp)
            c = rng.choice(len(lp), p=np.exp(lp - logsumexp(lp)))
            lab[i] = blocks[c] if c < len(blocks) else (max(blocks) + 1 if blocks else 0)
    return canonical(lab)


def chi_square_against(counts, parts, post, n):
    """Pearson chi-square p-value of partition counts of independent draws
    against the enumerated probabilities (cells expecting fewer than 5 draws
    pooled into one)."""
    R = sum(counts.values())
    obs = np.array([counts.get(partition_key(p, n), 0) for p in parts], dtype=float)
    assert obs.sum() == R                 # every draw is one of the enumerated partitions
    exp = post * R
    small = exp < 5
    if small.any():
        obs = np.append(obs[~small], obs[small].sum())
        exp = np.append(exp[~small], exp[small].sum())
    return stats.chisquare(obs, exp).pvalue


def test_enumerated_posterior_matches_collapsed_gibbs_on_six_cells():
    """Independent textbook collapsed-Gibbs chains (8 passes each) on six
    cells land on the 203 partitions with the enumerated eq. 26 / eq. 28 /
    CRP posterior probabilities (chi-square)."""
    n = SIX_X.shape[0]
    parts, post = exact_partition_posterior(SIX_X, 1.0, 0.5)
    assert len(parts) == 203
    rng = np.random.default_rng(0)
    counts = {}
    for _ in range(1500):
        key = collapsed_gibbs_state(SIX_X, 1.0, 0.5, 8, rng)
        counts[key] = counts.get(key, 0) + 1
    assert chi_square_against(counts, parts, post, n) > 1e-3


def k_restricted_posterior(x, K, alpha, beta):
    parts, post = exact_partition_posterior(x, alpha, beta)
    keep = np.array([len(p) == K for p in parts])
    parts = [p for p, k in zip(parts, keep) if k]
    post = post[keep] / post[keep].sum()
    return parts, post


def fixed_k_sweeps(X, K, alpha, beta, labels, seed, sweeps):
    """The eq. 4 sweep with K held fixed (pi | c, theta | c, then all c_i | pi,
    theta in parallel): label draws that empty a cluster are redrawn with
    fresh counters, pi and theta held (rejection sampling of the restricted
    conditional).  Returns the canonical partition after `sweeps` sweeps."""
    from oracle.sampler import draw_pi, draw_theta
    n = X.shape[0]
    sub = np.zeros(n, dtype=np.int64)
    s = 0
    for t in range(sweeps):
        nsub, Ssub = sufficient_stats(X, labels, sub, K)
        logpi = draw_pi(nsub.sum(axis=1), alpha, seed, 0, t)
        logtheta = draw_theta(Ssub, beta, seed, 0, t)
        while True:
            new, _, _, _ = assign(X, logpi, logtheta, labels, sub, nsub, seed, 0, s)
            s += 1
            if np.bincount(new, minlength=K).min() > 0:
                break
        labels = new
    return canonical(labels)


@pytest.mark.parametrize("base", [100000, 200000])
def test_sweep_is_exact_gibbs_for_fixed_K_posterior_on_six_cells(base):
    """With K held fixed, the eq. 4 sweep is a Gibbs sampler for p(c | x, K
    non-empty clusters) (Section 2.2: cells are conditionally independent
    given pi and theta).  1,200 independent chains (their own Philox seeds,
    random two-block starts, 8 sweeps each) must land on the 31 two-block
    partitions of six cells with the enumerated posterior probabilities
    (chi-square, p > 0.001).  Four sweeps are measurably too few to forget
    the start; six already pass."""
    x = SIX_X
    n, D = x.shape
    K, alpha, beta = 2, 1.0, 0.5
    X = csr_matrix(np.arange(n + 1) * D, np.tile(np.arange(D), n), x.ravel(), n, D)
    parts, post = k_restricted_posterior(x, K, alpha, beta)
    assert len(parts) == 31
    rng = np.random.default_rng(base)
    counts = {}
    for r in range(1200):
        while True:
            labels = rng.integers(0, K, n)
            if np.bincount(labels, minlength=K).min() > 0:
                break
        key = fixed_k_sweeps(X, K, alpha, beta, labels, base + r, 8)
        counts[key] = counts.get(key, 0) + 1
    assert chi_square_against(counts, parts, post, n) > 1e-3


@pytest.mark.xfail(strict=True, reason=(
    "finding: the paper's chain (parallel restricted Gibbs that may empty clusters, "
    "plus separate split-only and merge-only MH chains) is not invariant for the "
    "DPMM posterior on six-cell data; it over-weights coarse partitions"))
def test_full_chain_matches_exact_partition_posterior_on_six_cells():
    """Independent full chains (sweep + coin-selected split/merge, 12 steps
    each from K = 1) against the enumerated posterior over all 203
    partitions (chi-square)."""
    x = SIX_X
    n, D = x.shape
    parts, post = exact_partition_posterior(x, 1.0, 0.5)
    counts = {}
    for r in range(500):
        s = Sampler(np.arange(n + 1) * D, np.tile(np.arange(D), n), x.ravel(), n, D, 1.0, 0.5,
                    seed=11 + r)
        for _ in range(12):
            s.sweep()
            s.split_merge(0)
        key = canonical(s.labels)
        counts[key] = counts.get(key, 0) + 1
    assert chi_square_against(counts, parts, post, n) > 1e-3


# ---------------------------------------------------------------------------
# eq. 4 with the K+1 candidate open
# ---------------------------------------------------------------------------
def _zero_rows(n, D):
    return np.zeros(n + 1, dtype=np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64)


def test_open_candidate_takes_pi_k_plus_1_on_cells_without_counts():
    """A cell without counts has p(x | theta) = 1 under every theta, so its
    label is drawn from (pi_1, .., pi_K, pi_{K+1}) alone: the fraction of cells
    that open the new cluster is pi_{K+1}, the alpha entry of eq. 4."""
    from oracle.sampler import draw_pi
    n, D, K = 20000, 4, 2
    s = Sampler(*_zero_rows(n, D), n, D, 3000.0, 0.5, seed=5, open_new_cluster=True)
    s.set_state(np.arange(n) % K, np.zeros(n, np.int64), K, t=3)
    logpi, logtheta = s.draw_params()
    assert logpi.size == K + 2 and logpi[-1] == -np.inf and logtheta.shape == (3 * (K + 1), D)
    ref = draw_pi(np.full(K, n / K), 3000.0, 5, 0, 3)
    np.testing.assert_array_equal(logpi[:K + 1], ref)
    s.assign_and_update(logpi, logtheta)
    assert s.K == K + 1                       # survivors keep their order: the new one is last
    counts = np.bincount(s.labels, minlength=K + 1)
    p = np.exp(logpi[:K + 1])
    assert p[K] > 0.05
    assert stats.chisquare(counts, p * n).pvalue > 1e-4


def test_open_candidate_theta_is_drawn_from_the_prior():
    """The candidate's theta and theta-bar rows are Dirichlet(lambda) draws
    whatever the data: mean 1/D and variance (1/D)(1 - 1/D)/(D lambda + 1)
    per gene over many sweeps."""
    n, D, lam = 6, 3, 0.7
    x = np.array([[9, 0, 1], [7, 1, 0], [8, 0, 2], [0, 5, 5], [1, 6, 4], [0, 4, 6]])
    indptr = np.arange(n + 1) * D
    s = Sampler(indptr, np.tile(np.arange(D), n), x.ravel(), n, D, 1.0, lam, seed=2,
                open_new_cluster=True)
    draws = []
    for t in range(1500):
        s.t = t
        _, logtheta = s.draw_params()
        draws.append(np.exp(logtheta[3:6]))     # K = 1: rows 3..5 are the candidate's
    th = np.concatenate(draws)                  # (3 * 1500, D) independent prior draws
    m = th.shape[0]
    var = (1 / D) * (1 - 1 / D) / (D * lam + 1)
    assert np.all(np.abs(th.mean(0) - 1 / D) < 5 * math.sqrt(var / m))
    assert np.all(np.abs(th.var(0) / var - 1) < 0.15)


def test_open_chain_with_vanishing_alpha_is_the_restricted_chain(tiny_dataset):
    """pi_{K+1} -> 0 closes the candidate: every other draw keeps its Philox
    counter, so the open chain is the restricted chain exactly."""
    ds = tiny_dataset
    a = Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1e-30, 0.5, seed=4)
    b = Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1e-30, 0.5, seed=4,
                open_new_cluster=True)
    for s in (a, b):
        s.set_state(ds.labels, np.arange(ds.N) % 2, int(ds.labels.max()) + 1)
    for _ in range(4):
        a.sweep(); b.sweep()
        a.split_merge(0); b.split_merge(0)
    assert a.K == b.K
    np.testing.assert_array_equal(a.labels, b.labels)
    np.testing.assert_array_equal(a.sub, b.sub)
    np.testing.assert_array_equal(a.sumlogq, b.sumlogq)


def test_open_candidate_absent_at_capacity():
    n, D = 8, 3
    x = np.ones((n, D), dtype=np.int64)
    s = Sampler(np.arange(n + 1) * D, np.tile(np.arange(D), n), x.ravel(), n, D, 1.0, 0.5,
                kmax=2, open_new_cluster=True)
    s.set_state(np.arange(n) % 2, np.zeros(n, np.int64), 2)
    logpi, logtheta = s.draw_params()
    assert logpi.size == 3 and logtheta.shape[0] == 6


# ---------------------------------------------------------------------------
# local Gibbs iterations after the first (Section 2.3)
# ---------------------------------------------------------------------------
def test_local_gibbs_draws_theta_bar_from_eq19_and_sublabels_from_eq8():
    """Labels held, fixed sub-label pattern on 6 identical cells (3 in each
    sub-cluster, so the n-bar_{r, not i} correction matters): over many
    steps, theta-bar has the Dirichlet(beta + S-bar_r) posterior mean, each
    cell's new sub-label is 1 with the eq. 8 probability computed from the
    returned theta-bar, and log q_i is the log of that probability."""
    n, D, lam = 6, 3, 0.5
    row = np.array([2, 1, 3])
    X = np.tile(row, (n, 1))
    s = Sampler(np.arange(n + 1) * D, np.tile(np.arange(D), n), X.ravel(), n, D, 1.0, lam,
                seed=9, local_iters=2)
    sub0 = np.array([0, 0, 0, 1, 1, 1])
    S = np.array([3 * row, 3 * row], dtype=float)             # S-bar_0, S-bar_1
    post_mean = (lam + S) / (lam * D + S.sum(axis=1, keepdims=True))
    steps = 3000
    th_sum = np.zeros((2, D))
    z_num, z_den = np.zeros(2), np.zeros(2)
    for t in range(steps):
        s.set_state(np.zeros(n, np.int64), sub0, 1, t=t + 1)
        logtb = s.local_gibbs(1)
        th_sum += np.exp(logtb)
        lik = row @ logtb.T                                   # (2,)
        for so in (0, 1):
            w = np.array([3.0, 3.0]) - (np.arange(2) == so)
            p1 = w[1] * np.exp(lik[1]) / (w[0] * np.exp(lik[0]) + w[1] * np.exp(lik[1]))
            cells = np.nonzero(sub0 == so)[0]
            got = s.sub[cells]
            z_num[so] += np.sum(got - p1)
            z_den[so] += len(cells) * p1 * (1 - p1)
    assert np.all(np.abs(z_num / np.sqrt(z_den)) < 5)
    var = post_mean * (1 - post_mean) / (lam * D + S.sum(axis=1, keepdims=True) + 1)
    assert np.all(np.abs(th_sum / steps - post_mean) < 5 * np.sqrt(var / steps))


def test_local_gibbs_log_q_is_the_log_eq8_probability():
    n, D = 7, 4
    rng = np.random.default_rng(3)
    X = rng.integers(0, 5, size=(n, D))
    s = Sampler(np.arange(n + 1) * D, np.tile(np.arange(D), n), X.ravel(), n, D, 1.0, 0.6,
                seed=4, local_iters=3)
    labels = np.array([0, 0, 0, 1, 1, 1, 1])
    sub = np.array([0, 1, 1, 0, 0, 1, 0])
    s.set_state(labels, sub, 2, t=5)
    nsub, _ = s.stats()
    logtb = s.local_gibbs(2)
    lik = np.stack([(X @ logtb[0::2].T)[np.arange(n), labels],
                    (X @ logtb[1::2].T)[np.arange(n), labels]], axis=1)
    w = nsub[labels] - np.stack([sub == 0, sub == 1], axis=1)
    with np.errstate(divide="ignore"):
        lw = np.log(w.astype(float)) + lik
    ref = lw[np.arange(n), s.sub] - np.logaddexp(lw[:, 0], lw[:, 1])
    np.testing.assert_allclose(s.sumlogq, np.bincount(labels, weights=ref), rtol=1e-12)
    np.testing.assert_array_equal(s.labels, labels)
    assert s.K == 2


def test_one_local_iteration_is_the_default_chain(tiny_dataset):
    ds = tiny_dataset
    a = Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, seed=8)
    b = Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, seed=8, local_iters=1)
    c = Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, seed=8, local_iters=3)
    for s in (a, b, c):
        s.sweep()
    np.testing.assert_array_equal(a.labels, b.labels)
    np.testing.assert_array_equal(a.sub, b.sub)
    np.testing.assert_array_equal(a.labels, c.labels)     # later iterations hold the labels
    assert not np.allclose(a.sumlogq, c.sumlogq)          # with new theta-bar draws
    with pytest.raises(ValueError):
        Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, local_iters=17)


# ---------------------------------------------------------------------------
# helpers of the sweep, pinned directly
# ---------------------------------------------------------------------------
def test_compact_keeps_survivors_in_order():
    from oracle.sampler import compact
    labels = np.array([4, 0, 4, 2, 0, 4])          # clusters 1 and 3 are empty
    per = np.array([10.0, 11.0, 12.0, 13.0, 14.0])
    new, K, (kept,) = compact(labels, 5, per)
    assert K == 3
    np.testing.assert_array_equal(new, [2, 0, 2, 1, 0, 2])
    np.testing.assert_array_equal(kept, [10.0, 12.0, 14.0])


def test_fair_coin_sublabels_are_fair_and_independent_across_kinds():
    from oracle.sampler import fair_coin_sublabels
    cells = np.arange(200000)
    a = fair_coin_sublabels(cells, 7, 0, 3, philox.SUBINIT_RESET)
    b = fair_coin_sublabels(cells, 7, 0, 3, philox.SUBINIT_SPLIT)
    c = fair_coin_sublabels(cells, 7, 0, 4, philox.SUBINIT_RESET)
    for x in (a, b, c):
        assert set(np.unique(x)) <= {0, 1}
        assert abs(x.mean() - 0.5) < 5 * np.sqrt(0.25 / cells.size)
    for x, y in ((a, b), (a, c)):
        r = np.corrcoef(x, y)[0, 1]
        assert abs(r) < 5 / np.sqrt(cells.size)


def test_label_gumbels_follow_the_gumbel_law_and_word_layout():
    from oracle.sampler import label_gumbels
    N, K = 40000, 6
    g = label_gumbels(N, K, 3, 1, 9)
    for k in range(K):
        assert stats.kstest(g[:, k], "gumbel_r").pvalue > 1e-4
    # column k is word k % 4 of call k // 4 on counter (cell, t, tag 0, k // 4)
    w = philox.stream_words(3, 1, philox.TAG_LABEL, np.arange(N), 9, 1)
    np.testing.assert_array_equal(g[:, 5], philox.uniform_to_gumbel(philox.word_to_uniform(w[:, 1])))
    assert abs(np.corrcoef(g[:, 0], g[:, 4])[0, 1]) < 5 / np.sqrt(N)
