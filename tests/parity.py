"""Shared checks of the GPU label step against FP64 decisions (test helper).

Given the parameters the GPU used (FP32 values, read back and widened to
FP64), the FP64 oracle arithmetic fixes every cell's eq. 4 label and eq. 8
sub-label from the same Philox words.  The GPU's FP32 (or BF16 hi/lo)
contraction may decide differently only where the two competing perturbed
values lie closer than the contraction's error bound; every other cell must
agree exactly, and the per-cluster sum of log q_i must agree within the sum
of the per-cell bounds.
"""

import numpy as np

from oracle import philox

# FP32 logarithms and the final log-sum-exp of log q_i carry a few ulps
LOGQ_RTOL, LOGQ_ATOL = 1e-6, 1e-6


def fp32_bound(X, logtheta):
    """Per (cell, row of logtheta) bound of the FP32 CSR contraction:
    1e-5 sum_u x_u |log theta_u| + 1e-5 |score| + 1e-4."""
    ax = abs(X)
    sc = np.asarray(X @ logtheta.T)
    return 1e-5 * np.asarray(ax @ np.abs(logtheta).T) + 1e-5 * np.abs(sc) + 1e-4


def bf16_bound(X, logtheta):
    """Per (cell, row) bound of the BF16 hi/lo tensor-core contraction: the
    hi/lo representation error 2^-16 |d| of each centred value d = log theta -
    m_u (twice, for safety), plus FP32 accumulation."""
    m = logtheta.mean(axis=0)
    d = logtheta - m[None, :]
    ax = abs(X)
    sc = np.asarray(X @ d.T)
    return 2 * 2.0 ** -16 * np.asarray(ax @ np.abs(d).T) + 1e-5 * np.abs(sc) + 1e-3


def fp64_decisions(X, cells, logpi, logtheta, labels0, sub0, nsub0, K, seed, chain_id, t,
                   bound_rows):
    """FP64 eq. 4 labels and eq. 8 sub-labels of `cells` (X holds their rows)
    from the given parameters, with the near-tie masks of each decision.

    logtheta: (3K, D), row 3k cluster k, rows 3k + 1 + r its sub-clusters.
    bound_rows: (n, 3K) error bound of each contraction the GPU forms.
    Returns a dict: lab, near_lab, sub, near_sub, logq, logq_tol (sub-label
    quantities assume the cell takes the FP64 label)."""
    n = cells.size
    sc = np.asarray(X @ logtheta.T)                         # (n, 3K)
    g = np.empty((n, K))
    for j in range((K + 3) // 4):
        w = philox.stream_words(seed, chain_id, philox.TAG_LABEL, cells, t, j)
        take = min(4, K - 4 * j)
        g[:, 4 * j:4 * j + take] = philox.uniform_to_gumbel(philox.word_to_uniform(w[:, :take]))
    v = sc[:, 0::3] + logpi[None, :K] + g
    order = np.argsort(-v, axis=1, kind="stable")
    lab = order[:, 0]
    rows = np.arange(n)
    if K > 1:
        gap = v[rows, order[:, 0]] - v[rows, order[:, 1]]
        near_lab = gap < 2 * bound_rows[:, 0::3].max(axis=1)
    else:
        near_lab = np.zeros(n, bool)
    lik = np.stack([sc[rows, 3 * lab + 1], sc[rows, 3 * lab + 2]], axis=1)
    b = np.stack([bound_rows[rows, 3 * lab + 1], bound_rows[rows, 3 * lab + 2]], axis=1)
    stays = labels0 == lab
    w = np.stack([nsub0[lab, 0] - (stays & (sub0 == 0)), nsub0[lab, 1] - (stays & (sub0 == 1))],
                 axis=1).astype(np.float64)
    w[w.sum(axis=1) == 0] = 1.0
    with np.errstate(divide="ignore"):
        tr = np.log(w) + lik
    h = philox.uniform_to_gumbel(philox.word_to_uniform(
        philox.stream_words(seed, chain_id, philox.TAG_SUBLABEL, cells, t, 0)[:, :2]))
    a, c = tr[:, 1] + h[:, 1], tr[:, 0] + h[:, 0]
    sub = (a > c).astype(np.int64)
    both = np.isfinite(tr).all(axis=1)
    near_sub = both & (np.abs(a - c) < b.sum(axis=1) + 1e-5)
    logq = tr[rows, sub] - np.logaddexp(tr[:, 0], tr[:, 1])
    logq_tol = np.where(both, b.sum(axis=1), 0.0) + LOGQ_RTOL * np.abs(logq) + LOGQ_ATOL
    return dict(lab=lab, near_lab=near_lab, sub=sub, near_sub=near_sub, logq=logq,
                logq_tol=logq_tol)


def assert_decisions(ref, lab, sub):
    """Labels equal the FP64 ones except near-ties; where the label agrees,
    sub-labels equal the FP64 ones except eq. 8 near-ties.  Returns the mask of
    cells whose label and sub-label both agree."""
    mism = lab != ref["lab"]
    assert np.all(ref["near_lab"][mism]), \
        f"{mism.sum()} label mismatches, {ref['near_lab'].sum()} near-ties"
    ok = ~mism
    mism_s = ok & (sub != ref["sub"])
    assert np.all(ref["near_sub"][mism_s]), \
        f"{mism_s.sum()} sub-label mismatches, {ref['near_sub'].sum()} near-ties"
    return ok & ~mism_s


def check_assign(ref, K, K_gpu, lab_gpu, sub_gpu, sumlogq_gpu, seed, chain_id, t):
    """The GPU state after a label step (labels, sub-labels, compaction and
    sub-cluster resets; all N cells) against the FP64 decisions `ref`:

    * the compaction keeps the clusters the FP64 labels keep (same K), so the
      GPU's labels map back to pre-compaction indices;
    * labels and eq. 8 sub-labels as in assert_decisions;
    * clusters of two or more cells with an empty sub-cluster redraw their
      sub-labels as the tag-7 coins of sweep t, with sum log q = n log(1/2);
    * every other cluster's sum log q within the summed per-cell bound.
    Returns (clusters checked for sum log q, label near-tie flips)."""
    from oracle.sampler import fair_coin_sublabels
    lab_ref = ref["lab"]
    keep = np.bincount(lab_ref, minlength=K) > 0
    Kc = int(keep.sum())
    assert K_gpu == Kc, (K_gpu, Kc)
    sumlogq_gpu = np.asarray(sumlogq_gpu)
    assert sumlogq_gpu.shape[0] >= Kc
    inv = np.nonzero(keep)[0]
    assert int(lab_gpu.max()) < Kc, "the GPU kept a cluster the FP64 labels empty"
    lab_pre = inv[lab_gpu]
    mism = lab_pre != lab_ref
    assert np.all(ref["near_lab"][mism]), \
        f"{mism.sum()} label mismatches, {ref['near_lab'].sum()} near-ties"
    # sub-cluster resets decided from the FP64 decisions
    n0 = np.bincount(lab_ref[ref["sub"] == 0], minlength=K)
    n1 = np.bincount(lab_ref[ref["sub"] == 1], minlength=K)
    reset = (n0 + n1 >= 2) & ((n0 == 0) | (n1 == 0))
    in_reset = reset[lab_ref] & ~mism
    cells = np.nonzero(in_reset)[0]
    if cells.size:
        coins = fair_coin_sublabels(cells, seed, chain_id, t, 1)
        np.testing.assert_array_equal(sub_gpu[cells], coins)
        for k in np.nonzero(reset)[0]:
            if not mism[lab_ref == k].any():
                j = int(np.searchsorted(inv, k))
                np.testing.assert_allclose(sumlogq_gpu[j], (n0[k] + n1[k]) * np.log(0.5),
                                           rtol=1e-12)
    ok = ~mism & ~in_reset
    mism_s = ok & (sub_gpu != ref["sub"])
    assert np.all(ref["near_sub"][mism_s]), \
        f"{mism_s.sum()} sub-label mismatches, {ref['near_sub'].sum()} near-ties"
    agree = ok & ~mism_s
    # a cluster gaining or losing a near-tie cell has another sum
    dirty = (np.bincount(lab_ref[~agree], minlength=K) > 0) | \
        (np.bincount(lab_pre[~agree], minlength=K) > 0)
    exp = np.bincount(lab_ref, weights=ref["logq"], minlength=K)
    tol = np.bincount(lab_ref, weights=ref["logq_tol"], minlength=K)
    sel = keep & ~dirty & ~reset
    got = sumlogq_gpu[np.searchsorted(inv, np.nonzero(sel)[0])]
    err = np.abs(got - exp[sel])
    assert np.all(err <= tol[sel]), (err, tol[sel])
    return int(sel.sum()), int(mism.sum())


def decisions_from_oracle(o, logpi, logtheta, bound_rows):
    """FP64 decisions for all cells of oracle chain `o` (before its update)
    with the given parameters, cross-checked against the oracle's own eq. 4
    / eq. 8 draw (oracle.sampler.assign): the same labels, sub-labels and
    log q_i."""
    from oracle.sampler import assign
    K = o.K
    nsub0, _ = o.stats()
    X = o.X.astype(np.float64)
    cells = np.arange(o.N)
    ref = fp64_decisions(X, cells, logpi, logtheta, o.labels, o.sub, nsub0, K, o.seed,
                         o.chain_id, o.t, bound_rows)
    lab, sub, logq, _ = assign(o.X, np.asarray(logpi)[:K + 1], logtheta, o.labels,
                               o.sub, nsub0, o.seed, o.chain_id, o.t)
    np.testing.assert_array_equal(lab, ref["lab"])
    np.testing.assert_array_equal(sub, ref["sub"])
    np.testing.assert_allclose(logq, ref["logq"], rtol=1e-12, atol=1e-12)
    return ref
