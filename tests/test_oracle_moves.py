"""Pins for the oracle's split/merge bookkeeping (Sections 2.3-2.4): the merge
pairing, the fair coin that picks the chain, the empty-sub-cluster reset and
the sum of log q_i each move leaves behind.

The GPU parity tests compare the CUDA path with these oracle functions, so
each one is fixed here against a law or a hand value instead: the pairing is
a uniformly random set of disjoint pairs (Section 2.4, "selected randomly"),
the coin is fair, the reset fires exactly for clusters of two or more cells
with one empty sub-cluster, and the sums follow from q(S*|S) being the
product of the cells' eq. 8 probabilities (tests/golden/moves_sumlogq.txt).
"""

import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox
from oracle.sampler import Sampler, fair_coin_sublabels

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "moves_sumlogq.txt")
LOG_HALF = math.log(0.5)


def _sampler(n, D=2, alpha=1.0, beta=1.0, seed=1, kmax=256, counts=None):
    x = np.ones((n, D), dtype=np.int64) if counts is None else np.asarray(counts)
    indptr = np.arange(n + 1) * D
    return Sampler(indptr, np.tile(np.arange(D), n), x.ravel(), n, D, alpha, beta, seed=seed,
                   kmax=kmax)


# ---------------------------------------------------------------------------
# merge pairing
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 8, 9, 17])
def test_merge_pairs_are_disjoint_ordered_and_cover_all_but_one(K):
    s = _sampler(K)
    s.set_state(np.arange(K), np.zeros(K, np.int64), K)
    for m in range(200):
        s.m = m
        pairs = s.merge_pairs()
        assert len(pairs) == K // 2
        flat = [k for p in pairs for k in p]
        assert len(set(flat)) == len(flat) == 2 * (K // 2)
        assert all(0 <= a < b < K for a, b in pairs)


def _matching_key(pairs):
    return tuple(sorted(pairs))


def test_merge_pairing_is_uniform_over_perfect_matchings_of_four():
    """K = 4 has 3 perfect matchings; Section 2.4's random selection draws
    each with probability 1/3 (chi-square over 6,000 calls)."""
    s = _sampler(4)
    s.set_state(np.arange(4), np.zeros(4, np.int64), 4)
    counts = {}
    for m in range(6000):
        s.m = m
        key = _matching_key(s.merge_pairs())
        counts[key] = counts.get(key, 0) + 1
    assert set(counts) == {((0, 1), (2, 3)), ((0, 2), (1, 3)), ((0, 3), (1, 2))}
    obs = np.array(list(counts.values()))
    assert stats.chisquare(obs).pvalue > 1e-3


def test_merge_pairing_is_uniform_over_the_15_pairings_of_five():
    """K = 5: one cluster sits out and the other four form one of 3
    matchings, 15 outcomes, each with probability 1/15."""
    s = _sampler(5)
    s.set_state(np.arange(5), np.zeros(5, np.int64), 5)
    expect = set()
    for out in range(5):
        rest = [k for k in range(5) if k != out]
        a = rest[0]
        for b in rest[1:]:
            c, d = [k for k in rest[1:] if k != b]
            expect.add(_matching_key([(a, b), (c, d)]))
    assert len(expect) == 15
    counts = {}
    for m in range(9000):
        s.m = m
        key = _matching_key(s.merge_pairs())
        counts[key] = counts.get(key, 0) + 1
    assert set(counts) == expect
    assert stats.chisquare(np.array(list(counts.values()))).pvalue > 1e-3


def test_merge_pairing_does_not_favour_any_cluster_as_the_odd_one_out():
    s = _sampler(7)
    s.set_state(np.arange(7), np.zeros(7, np.int64), 7)
    out = np.zeros(7, np.int64)
    partner = np.zeros((7, 7), np.int64)
    for m in range(7000):
        s.m = m
        pairs = s.merge_pairs()
        seen = set()
        for a, b in pairs:
            partner[a, b] += 1
            seen |= {a, b}
        out[list(set(range(7)) - seen)[0]] += 1
    assert stats.chisquare(out).pvalue > 1e-3
    pair_counts = partner[np.triu_indices(7, 1)]
    assert stats.chisquare(pair_counts).pvalue > 1e-3


def test_merge_pairing_changes_with_the_call_counter_and_chain():
    s = _sampler(6)
    s.set_state(np.arange(6), np.zeros(6, np.int64), 6)
    s.m = 3
    a = s.merge_pairs()
    s.m = 4
    b = s.merge_pairs()
    t = _sampler(6)
    t.chain_id = 1
    t.set_state(np.arange(6), np.zeros(6, np.int64), 6)
    t.m = 3
    draws = [tuple(a), tuple(b), tuple(t.merge_pairs())]
    # three pairings of 6 clusters (15 possible) coincide only by chance; over
    # many counters they differ most of the time
    same = 0
    for m in range(300):
        s.m = m
        t.m = m
        same += s.merge_pairs() == t.merge_pairs()
    assert same < 60 and len(draws) == 3


# ---------------------------------------------------------------------------
# the chain coin (Section 2.4: the split or the merge chain, selected randomly)
# ---------------------------------------------------------------------------
def test_chain_coin_is_fair_and_independent_across_chains():
    s = _sampler(2)
    t = _sampler(2)
    t.chain_id = 5
    n = 20000
    a = np.empty(n, bool)
    b = np.empty(n, bool)
    for m in range(n):
        s.m = t.m = m
        a[m] = s.coin_is_split()
        b[m] = t.coin_is_split()
    for x in (a, b):
        assert stats.binomtest(int(x.sum()), n, 0.5).pvalue > 1e-3
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / math.sqrt(n)
    # successive calls are not correlated either
    assert abs(np.corrcoef(a[:-1], a[1:])[0, 1]) < 5 / math.sqrt(n)


def test_coin_mode_runs_the_chain_the_coin_names():
    """alpha = 1e300 accepts every split and rejects every merge (a merge's
    ratio carries 1/alpha), so K grows in a coin-selected call exactly when
    the coin says split."""
    n = 12
    rng = np.random.default_rng(2)
    s = _sampler(n, D=3, alpha=1e300, counts=rng.integers(0, 3, size=(n, 3)), kmax=4096)
    grew = []
    said = []
    for _ in range(40):
        s.set_state(np.zeros(n, np.int64), np.arange(n) % 2, 1)
        said.append(s.coin_is_split())
        K0 = s.K
        s.split_merge(0)
        grew.append(s.K > K0)
    assert grew == said
    assert 0 < sum(said) < 40


# ---------------------------------------------------------------------------
# the empty-sub-cluster reset at the end of a sweep
# ---------------------------------------------------------------------------
def test_reset_fires_exactly_for_clusters_of_two_or_more_cells_with_an_empty_side():
    labels = np.array([0, 0, 0, 1, 2, 2, 2, 2, 3, 3, 4])
    sub = np.array([0, 0, 0, 1, 0, 1, 0, 1, 1, 1, 0])
    K = 5
    s = _sampler(labels.size)
    for t in range(60):
        s.set_state(labels, sub, K, t=t, sumlogq=[-1.0, -2.0, -3.0, -4.0, -5.0])
        s._reset_empty_subclusters()
        # clusters 1 (one cell in sub 1), 4 (one cell in sub 0) and 2 (two and
        # two) are untouched, in sub-labels and in their sums
        keep = np.isin(labels, [1, 2, 4])
        np.testing.assert_array_equal(s.sub[keep], sub[keep])
        np.testing.assert_array_equal(s.sumlogq[[1, 2, 4]], [-2.0, -3.0, -5.0])
        # clusters 0 and 3 redraw every cell's sub-label as the tag-7 coin of
        # sweep t, and their sums become n_k log(1/2)
        redo = np.isin(labels, [0, 3])
        cells = np.nonzero(redo)[0]
        np.testing.assert_array_equal(
            s.sub[cells], fair_coin_sublabels(cells, s.seed, s.chain_id, t, philox.SUBINIT_RESET))
        np.testing.assert_allclose(s.sumlogq[[0, 3]], [3 * LOG_HALF, 2 * LOG_HALF], rtol=0,
                                   atol=1e-15)
        np.testing.assert_array_equal(s.labels, labels)


def test_reset_coins_are_fair():
    n = 4000
    s = _sampler(n)
    ones = 0
    for t in range(10):
        s.set_state(np.zeros(n, np.int64), np.zeros(n, np.int64), 1, t=t)
        s._reset_empty_subclusters()
        ones += int(s.sub.sum())
    assert stats.binomtest(ones, 10 * n, 0.5).pvalue > 1e-3


def test_sweep_calls_the_reset_after_the_compaction():
    """A sweep whose draw leaves a cluster with an empty side ends with that
    cluster's sub-labels redrawn: after any sweep every cluster of two or
    more cells has both sub-clusters occupied or was just reset (its sum is
    then exactly n_k log(1/2))."""
    rng = np.random.default_rng(8)
    n, D = 30, 4
    s = _sampler(n, D=D, counts=rng.integers(0, 6, size=(n, D)), seed=4)
    reset_seen = 0
    for _ in range(40):
        s.sweep()
        nsub, _ = s.stats()
        nk = nsub.sum(axis=1)
        for k in range(s.K):
            if nk[k] >= 2 and (nsub[k] == 0).any():
                # a reset's coins may land on one side again; its sum says so
                assert s.sumlogq[k] == nk[k] * LOG_HALF
        reset_seen += int(np.any(np.isclose(s.sumlogq, nk * LOG_HALF)))
    assert reset_seen > 0


# ---------------------------------------------------------------------------
# sum of log q_i after each kind of step, against hand values
# ---------------------------------------------------------------------------
def _golden_cases():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, step, K, labels, sub, before, after = line.split()
            rows.append((name, step, int(K), [int(v) for v in labels.split(",")],
                         [int(v) for v in sub.split(",")],
                         [float(v) for v in before.split(",")],
                         [float(v) for v in after.split(",")]))
    return rows


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c[0])
def test_sum_log_q_after_moves_and_resets_matches_hand_values(case):
    name, step, K, labels, sub, before, after = case
    n = len(labels)
    alpha = {"split": 1e300, "merge": 1e-300, "reset": 1.0}[step]
    s = _sampler(n, D=2, alpha=alpha, beta=1.0, seed=3)
    s.set_state(labels, sub, K, t=2, m=5, sumlogq=before)
    if step == "split":
        s.split_merge(1)
    elif step == "merge":
        s.split_merge(2)
    else:
        s._reset_empty_subclusters()
    assert s.K == len(after)
    np.testing.assert_allclose(s.sumlogq, after, rtol=0, atol=1e-15)


def test_split_moves_sub_cluster_one_to_new_indices_in_ascending_order():
    s = _sampler(9, alpha=1e300, seed=3)
    labels = [0, 0, 0, 0, 0, 1, 1, 1, 1]
    sub = [0, 1, 1, 0, 1, 0, 0, 1, 1]
    s.set_state(labels, sub, 2, m=5)
    assert s.split_merge(1) == 2
    np.testing.assert_array_equal(s.labels, [0, 2, 2, 0, 2, 1, 1, 3, 3])
    # every touched cell draws a fresh tag-7 coin of call m (kind 2)
    np.testing.assert_array_equal(
        s.sub, fair_coin_sublabels(np.arange(9), s.seed, s.chain_id, 5, philox.SUBINIT_SPLIT))
    assert s.m == 6


def test_merge_keeps_the_lower_index_with_cells_of_a_as_sub_zero():
    s = _sampler(7, alpha=1e-300, seed=3)
    labels = np.array([2, 0, 1, 2, 1, 0, 2])
    s.set_state(labels, [1, 1, 0, 0, 1, 0, 1], 3, m=7)
    pairs = s.merge_pairs()
    assert len(pairs) == 1
    a, b = pairs[0]
    out = ({0, 1, 2} - {a, b}).pop()
    assert s.split_merge(2) == 1 and s.K == 2
    # survivors keep their order: the merged cluster a and the one left out
    new_a, new_out = (0, 1) if a < out else (1, 0)
    np.testing.assert_array_equal(s.labels[labels == a], new_a)
    np.testing.assert_array_equal(s.labels[labels == b], new_a)
    np.testing.assert_array_equal(s.labels[labels == out], new_out)
    np.testing.assert_array_equal(s.sub[labels == a], 0)
    np.testing.assert_array_equal(s.sub[labels == b], 1)
    assert s.sumlogq[new_a] == 0.0


def test_merge_of_three_clusters_leaves_each_one_out_over_the_calls():
    """A merge pass over three clusters pairs two and leaves one out; over the
    call counters each of the three is left out at some call."""
    s = _sampler(6, alpha=1e-300, seed=9)
    outs = set()
    for m in range(60):
        s.set_state([0, 0, 1, 1, 2, 2], [0, 1, 0, 1, 0, 1], 3, m=m)
        (a, b), = s.merge_pairs()
        outs.add(({0, 1, 2} - {a, b}).pop())
    assert outs == {0, 1, 2}
