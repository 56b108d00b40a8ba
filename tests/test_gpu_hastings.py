"""Split proposals scored with the sweep's parameters instantiated (eq. 18:
eq. 14 times eq. 16) against the FP64 oracle, on both engines."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1812_10048_gb300 import build
    build.build()
    import paper_1812_10048_gb300 as P
    return P


@pytest.fixture(scope="module")
def data():
    from paper_1812_10048_gb300 import synth
    return synth.make_dataset(900, 400, 4, seed=21)


def _merged_start(P, ds, engine, seed):
    """Two clusters, each the union of two generating clusters, random sub-labels."""
    eng = P.ENGINE_AUTO if engine == "auto" else P.ENGINE_CSR_FP32
    s = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, seed=seed,
                  engine=eng, hastings="instantiated")
    rng = np.random.default_rng(seed)
    labels = (ds.labels // 2).astype(np.int32)
    sub = rng.integers(0, 2, size=ds.N).astype(np.uint8)
    s.set_state(labels, sub, 2)
    return s


def _expected(P, s, D, alpha, beta):
    from oracle.model import log_hastings_split_instantiated
    _, _, K, _, _ = s.get_state()
    logpi, logtheta = P.dpmm_get_params(s.ctx, K, D)
    nsub, Ssub, sumlogq = s.stats()
    ref = np.full(K, np.nan)
    for k in range(K):
        n0, n1 = int(nsub[k, 0]), int(nsub[k, 1])
        if n0 < 1 or n1 < 1:
            continue
        ref[k] = log_hastings_split_instantiated(
            n0, n1, Ssub[k, 0], Ssub[k, 1], logtheta[3 * k], logtheta[3 * k + 1],
            logtheta[3 * k + 2], float(logpi[k]), alpha, beta, float(sumlogq[k]))
    return K, ref, (nsub, Ssub, sumlogq)


@pytest.mark.parametrize("engine", ["auto", "csr"])
def test_instantiated_split_ratio_matches_oracle(P, data, engine):
    s = _merged_start(P, data, engine, seed=4)
    s.sweep(6)                   # sub-clusters settle on the generating clusters
    K, ref, _ = _expected(P, s, data.D, 1.0, 0.5)
    assert K == 2                # no cluster emptied: rows of the draw = clusters
    n_acc = s.split_merge(1)
    chain, log_h, _ = P.dpmm_debug_moves(s.ctx, s.kmax)
    assert chain == 1
    assert np.array_equal(np.isnan(log_h), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert ok.all()
    np.testing.assert_allclose(log_h[ok], ref[ok], rtol=1e-10, atol=1e-7)
    # separated generating clusters: both splits are strongly favoured
    assert (ref > 50).all() and n_acc == 2
    _, K2 = s.labels()
    assert K2 == 4
    # the move consumed the sweep's draws: a second proposal round has none
    assert s.split_merge(1) == 0
    _, log_h2, _ = P.dpmm_debug_moves(s.ctx, s.kmax)
    assert np.isnan(log_h2).all()


def test_instantiated_ratio_on_unsplittable_clusters(P, data):
    """Each cluster one generating cluster: the instantiated ratio is finite and
    matches the oracle, and it lies far above the collapsed ratio of the same
    sub-clusters (eq. 16 carries one more Dirichlet density and no density for
    drawing the new theta, which favours every split)."""
    s = P.Sampler(data.indptr, data.indices, data.data, data.N, data.D, 1.0, 0.5, seed=9,
                  hastings="instantiated")
    rng = np.random.default_rng(9)
    s.set_state(data.labels.astype(np.int32), rng.integers(0, 2, size=data.N).astype(np.uint8), 4)
    s.sweep(3)
    K, ref, (nsub, Ssub, sumlogq) = _expected(P, s, data.D, 1.0, 0.5)
    assert K == 4
    s.split_merge(1)
    _, log_h, _ = P.dpmm_debug_moves(s.ctx, s.kmax)
    ok = ~np.isnan(ref)
    assert np.array_equal(np.isnan(log_h), ~ok)
    np.testing.assert_allclose(log_h[ok], ref[ok], rtol=1e-10, atol=1e-7)
    from oracle.model import log_hastings_split
    for k in np.where(ok)[0]:
        col = log_hastings_split(int(nsub[k, 0]), int(nsub[k, 1]), Ssub[k, 0], Ssub[k, 1],
                                 1.0, 0.5, float(sumlogq[k]))
        assert log_h[k] > col + 100.0


def test_instantiated_needs_a_sweep_first(P, data):
    """After set_state no sweep's parameters belong to the clusters: no split
    is proposed (NaN ratios), merges still run."""
    s = _merged_start(P, data, "auto", seed=5)
    assert s.split_merge(1) == 0
    chain, log_h, _ = P.dpmm_debug_moves(s.ctx, s.kmax)
    assert chain == 1 and log_h.size == 2 and np.isnan(log_h).all()
    s.split_merge(2)
    chain, log_h, _ = P.dpmm_debug_moves(s.ctx, s.kmax)
    assert chain == 2 and np.isfinite(log_h).all()


def test_instantiated_chain_keeps_statistics_exact(P, data):
    """Graph-stepped chain with instantiated splits: the statistics kept by the
    sweeps and moves equal a recount from the labels."""
    from oracle.logml import cluster_stats
    s = P.Sampler(data.indptr, data.indices, data.data, data.N, data.D, 1.0, 0.5, seed=12,
                  hastings="instantiated")
    s.step(25)
    labels, K = s.labels()
    _, sub, _, _, _ = s.get_state()
    n, S = cluster_stats(data.indptr, data.indices, data.data, data.N, data.D, labels, K)
    nsub, Ssub, _ = s.stats()
    np.testing.assert_array_equal(nsub.sum(1), n)
    np.testing.assert_array_equal(Ssub.sum(1), S)
    for k in range(K):
        for r in range(2):
            assert nsub[k, r] == np.sum((labels == k) & (sub == r))
    assert K >= 3                # the generating clusters get separated
