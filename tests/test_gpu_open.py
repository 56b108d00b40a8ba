"""Eq. 4 with the K+1 candidate open (opts.open_new_cluster) against the FP64
oracle: the appended cluster's draws, the label draw that may choose it, and
the chain's bookkeeping."""

import numpy as np
import pytest

from .test_gpu_parity import SCORE_ATOL, SCORE_RTOL

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
def padded():
    """The tiny workload plus 300 cells without counts (their label is drawn
    from pi alone, so some of them open the candidate when alpha is large)."""
    from paper_1812_10048_gb300 import synth
    ds = synth.tiny()
    extra = 300
    indptr = np.concatenate([ds.indptr, np.full(extra, ds.indptr[-1], ds.indptr.dtype)])
    labels = np.concatenate([ds.labels, np.zeros(extra, ds.labels.dtype)])
    return synth.Dataset(indptr=indptr, indices=ds.indices, data=ds.data, N=ds.N + extra,
                         D=ds.D, labels=labels)


def _pair(P, ds, alpha, seed, engine="csr"):
    from oracle.sampler import Sampler as OracleSampler
    eng = P.ENGINE_CSR_FP32 if engine == "csr" else P.ENGINE_AUTO
    g = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, alpha, 0.5, seed=seed, kmax=64,
                  engine=eng, open_new_cluster=True)
    o = OracleSampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, alpha, 0.5, seed=seed, kmax=64,
                      open_new_cluster=True)
    K = int(ds.labels.max()) + 1
    sub = (np.arange(ds.N) % 2).astype(np.int64)
    o.set_state(ds.labels, sub, K, t=5)
    P.dpmm_set_state(g.ctx, o.labels, o.sub, o.K, o.t, o.m, o.sumlogq)
    return g, o


def test_open_draw_appends_the_candidate_and_matches_oracle(P, padded):
    g, o = _pair(P, padded, 500.0, seed=3)
    K0 = o.K
    P.dpmm_draw_params(g.ctx)
    _, _, K, _, _ = g.get_state()
    assert K == K0 + 1
    logpi, logtheta = P.dpmm_get_params(g.ctx, K, padded.D)
    ref_pi, ref_th = o.draw_params()
    assert ref_pi.size == logpi.size == K0 + 2
    assert logpi[-1] == -np.inf and ref_pi[-1] == -np.inf
    np.testing.assert_allclose(logpi[:-1], ref_pi[:-1], rtol=1e-5, atol=1e-4)
    assert logtheta.shape == ref_th.shape == (3 * (K0 + 1), padded.D)
    # the candidate's rows are prior draws (gene sums zero), the others as in
    # the restricted draw; a rare Gamma flip moves a row's normaliser
    far = np.abs(logtheta - ref_th) > 1e-2
    assert far.sum() <= max(2, 1e-3 * ref_th.size)
    rows = np.setdiff1d(np.arange(ref_th.shape[0]), np.unique(np.nonzero(far)[0]))
    np.testing.assert_allclose(logtheta[rows], ref_th[rows], rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("engine", ["csr", "auto"])
def test_open_label_draw_with_injected_params_matches_oracle(P, padded, engine):
    from oracle.sampler import label_gumbels, sufficient_stats
    from oracle.model import multinomial_scores
    g, o = _pair(P, padded, 500.0, seed=8, engine=engine)
    K0 = o.K
    P.dpmm_draw_params(g.ctx)
    logpi32, logtheta32 = P.dpmm_get_params(g.ctx, K0 + 1, padded.D)
    P.dpmm_set_params(g.ctx, logpi32, logtheta32)
    logpi, logtheta = logpi32.astype(np.float64), logtheta32.astype(np.float64)
    gum = label_gumbels(o.N, K0 + 1, o.seed, o.chain_id, o.t)
    if engine == "csr":
        s = multinomial_scores(o.X.astype(np.float64), logpi[:K0 + 1], logtheta[0::3])
        srt = np.sort(s + gum, axis=1)
        near = srt[:, -1] - srt[:, -2] < SCORE_RTOL * np.abs(s).max(axis=1) + SCORE_ATOL
    else:                                        # BF16 hi/lo contraction and its bound
        from .test_gpu_tile import centred_reference
        ref, bound = centred_reference(o, logtheta)
        srt = np.sort(ref[:, :K0 + 1] + logpi[None, :K0 + 1] + gum, axis=1)
        near = srt[:, -1] - srt[:, -2] < 2 * bound[:, :K0 + 1].max(axis=1)
    o.assign_and_update(logpi, logtheta)
    P.dpmm_assign(g.ctx)
    labels, sub, K, t, _ = g.get_state()
    assert t == o.t
    assert o.K == K0 + 1 and K == o.K            # the candidate was chosen and kept
    mism = labels != o.labels
    assert np.all(near[mism]), f"{mism.sum()} label mismatches, {near.sum()} near-ties"
    new = labels == K0
    assert new.sum() > 20
    nsub, Ssub, _ = g.stats()
    on, oS = sufficient_stats(o.X, labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)


def test_open_chain_with_vanishing_alpha_is_the_restricted_chain(P):
    """pi_{K+1} -> 0: the open chain keeps every Philox counter of the
    restricted one, so on the FP32 CSR engine the two chains are identical."""
    from paper_1812_10048_gb300 import synth
    ds = synth.tiny()
    kw = dict(seed=6, kmax=64, engine=P.ENGINE_CSR_FP32)
    a = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1e-30, 0.5, **kw)
    b = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1e-30, 0.5,
                  open_new_cluster=True, **kw)
    K = int(ds.labels.max()) + 1
    sub = (np.arange(ds.N) % 2).astype(np.uint8)
    for s in (a, b):
        s.set_state(ds.labels.astype(np.int32), sub, K)
    a.step(10)
    b.step(10)
    sa, sb = a.get_state(), b.get_state()
    for x, y in zip(sa, sb):
        np.testing.assert_array_equal(x, y)
    na, Sa, qa = a.stats()
    nb, Sb, qb = b.stats()
    np.testing.assert_array_equal(na, nb)
    np.testing.assert_array_equal(Sa, Sb)
    np.testing.assert_array_equal(qa, qb)


def test_open_chain_keeps_statistics_exact(P, padded):
    from oracle.sampler import sufficient_stats
    g = P.Sampler(padded.indptr, padded.indices, padded.data, padded.N, padded.D, 200.0, 0.5,
                  seed=14, open_new_cluster=True)
    opened = 0
    for _ in range(12):
        _, K0 = g.labels()
        g.sweep(1)
        _, K1 = g.labels()
        opened += K1 > K0
        g.split_merge(0)
    assert opened > 0
    labels, sub, K, _, _ = g.get_state()
    nsub, Ssub, _ = g.stats()
    on, oS = sufficient_stats(g_X(padded), labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
    assert (nsub.sum(1) > 0).all()


def g_X(ds):
    from oracle.sampler import csr_matrix
    return csr_matrix(ds.indptr, ds.indices, ds.data, ds.N, ds.D)


def test_open_candidate_absent_at_capacity(P):
    n, D = 40, 3
    rng = np.random.default_rng(2)
    x = rng.integers(1, 4, size=(n, D))
    indptr = (np.arange(n + 1) * D).astype(np.int32)
    g = P.Sampler(indptr, np.tile(np.arange(D), n).astype(np.int32), x.ravel(), n, D, 1e6, 1.0,
                  kmax=2, seed=1, open_new_cluster=True)
    g.set_state((np.arange(n) % 2).astype(np.int32), np.zeros(n, np.uint8), 2)
    P.dpmm_draw_params(g.ctx)
    _, _, K, _, _ = g.get_state()
    assert K == 2
    g.step(5)
    _, K = g.labels()
    assert K <= 2
