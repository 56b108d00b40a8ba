"""Parity at the benchmark sizes, in the configurations bench.py times.

The oracle cannot run whole sweeps at these sizes, so each test checks what it
can compute one by one on sampled outputs (labels and eq. 8 sub-labels of
sampled cells, decided in FP64 from the GPU's own parameters; split and merge
ratios from the GPU's exact statistics; the parameter draw from the same
Philox counters) and properties that hold at any size (statistics equal to a
recount from the labels)."""

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TWO_M16 = 2.0 ** -16


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1812_10048_gb300 import build
    build.build()
    import paper_1812_10048_gb300 as P
    return P


def csr(ds):
    from oracle.sampler import csr_matrix
    return csr_matrix(ds.indptr, ds.indices, ds.data, ds.N, ds.D)


def library_sizes(ds):
    """Total count of every cell (int64; empty rows give 0)."""
    starts = np.minimum(ds.indptr[:-1].astype(np.int64), max(0, ds.data.size - 1))
    lib = np.add.reduceat(ds.data, starts, dtype=np.int64) if ds.data.size else np.zeros(ds.N, np.int64)
    lib[np.diff(ds.indptr) == 0] = 0
    return lib


def check_stats_properties(ds, labels, sub, K, nsub, Ssub, genes):
    """n-bar exact; per-(k, r) totals equal the library sizes of the member
    cells; S-bar exact on the sampled genes (entries gathered from the CSR)."""
    lab = labels.astype(np.int64)
    slot = 2 * lab + sub.astype(np.int64)
    np.testing.assert_array_equal(nsub.reshape(-1), np.bincount(slot, minlength=2 * K))
    tot = np.bincount(slot, weights=library_sizes(ds), minlength=2 * K)
    np.testing.assert_array_equal(Ssub.reshape(2 * K, ds.D).sum(axis=1, dtype=np.int64),
                                  np.rint(tot).astype(np.int64))
    pos = np.nonzero(np.isin(ds.indices, genes))[0]
    rows = np.searchsorted(ds.indptr, pos, side="right") - 1
    for u in genes:
        sel = ds.indices[pos] == u
        ref = np.bincount(slot[rows[sel]], weights=ds.data[pos[sel]].astype(np.float64),
                          minlength=2 * K)
        np.testing.assert_array_equal(Ssub.reshape(2 * K, ds.D)[:, u].astype(np.int64),
                                      np.rint(ref).astype(np.int64))


def check_draw(P, g, ds, alpha, beta, seed):
    """dpmm_draw_params against the oracle's Dirichlet draws from the GPU's
    exact statistics (same Philox counters); returns the FP32 parameters."""
    from oracle.sampler import draw_pi, draw_theta
    labels, sub, K, t, _ = g.get_state()
    nsub, Ssub, _ = g.stats()
    P.dpmm_draw_params(g.ctx)
    logpi, logtheta = P.dpmm_get_params(g.ctx, K, ds.D)
    ref_pi = draw_pi(nsub.sum(axis=1).astype(np.float64), alpha, seed, 0, t)
    ref_th = draw_theta(Ssub.astype(np.int64), beta, seed, 0, t)
    np.testing.assert_allclose(logpi, ref_pi, rtol=1e-5, atol=1e-4)
    far = np.abs(logtheta - ref_th) > 1e-2
    assert far.sum() <= max(2, 1e-4 * far.size), far.sum()
    rows = np.setdiff1d(np.arange(ref_th.shape[0]), np.unique(np.nonzero(far)[0]))
    np.testing.assert_allclose(logtheta[rows], ref_th[rows], rtol=1e-5, atol=1e-4)
    return labels, sub, nsub, K, t, logpi.astype(np.float64), logtheta.astype(np.float64)


def check_sampled_labels(P, g, ds, cells, before, seed, bf16):
    """After dpmm_assign with the drawn parameters: each sampled cell's label
    (eq. 4 Gumbel-max) and eq. 8 sub-label equal the FP64 decision from the
    same parameters and Philox words, except where the top two perturbed
    values are closer than the contraction's error bound."""
    from oracle import philox
    labels0, sub0, nsub0, K, t, logpi, logtheta = before
    P.dpmm_assign(g.ctx)
    labels, sub, K1, _, _ = g.get_state()
    X = csr(ds)[cells].astype(np.float64)
    if bf16:
        m = logtheta.mean(axis=0)
        d = logtheta - m[None, :]
        bound_rows = 2 * TWO_M16 * np.asarray(abs(X) @ np.abs(d).T)
    else:
        bound_rows = 1e-5 * np.asarray(abs(X) @ np.abs(logtheta).T)
    sc = np.asarray(X @ logtheta.T)                  # (n, 3K): row 3k + p
    bound_rows = bound_rows + 1e-5 * np.abs(sc) + 1e-3
    g_lab = np.empty((cells.size, K))
    for j in range((K + 3) // 4):
        w = philox.stream_words(seed, 0, philox.TAG_LABEL, cells, t, j)
        take = min(4, K - 4 * j)
        g_lab[:, 4 * j:4 * j + take] = philox.uniform_to_gumbel(philox.word_to_uniform(w[:, :take]))
    v = sc[:, 0::3] + logpi[None, :K] + g_lab
    order = np.argsort(-v, axis=1)
    exp_lab = order[:, 0]
    gap = v[np.arange(cells.size), order[:, 0]] - v[np.arange(cells.size), order[:, 1]]
    near = gap < 2 * bound_rows[:, 0::3].max(axis=1)
    # no cluster empties at these sizes, so the compaction keeps the labels
    assert K1 == K
    mism = labels[cells] != exp_lab
    assert np.all(near[mism]), f"{mism.sum()} label mismatches, {near.sum()} near-ties"
    # eq. 8 for the cells whose label agrees
    ok = ~mism
    c = exp_lab[ok]
    lik = np.stack([sc[ok][np.arange(ok.sum()), 3 * c + 1], sc[ok][np.arange(ok.sum()), 3 * c + 2]], axis=1)
    stays = labels0[cells][ok] == c
    so = sub0[cells][ok]
    w = np.stack([nsub0[c, 0] - (stays & (so == 0)), nsub0[c, 1] - (stays & (so == 1))],
                 axis=1).astype(np.float64)
    w[w.sum(axis=1) == 0] = 1.0
    with np.errstate(divide="ignore"):
        tr = np.log(w) + lik
    h = philox.uniform_to_gumbel(philox.word_to_uniform(
        philox.stream_words(seed, 0, philox.TAG_SUBLABEL, cells[ok], t, 0)[:, :2]))
    exp_sub = (tr[:, 1] + h[:, 1] > tr[:, 0] + h[:, 0]).astype(np.int64)
    b_sub = bound_rows[ok][np.arange(ok.sum()), 3 * c + 1] + bound_rows[ok][np.arange(ok.sum()), 3 * c + 2]
    near_s = np.abs((tr[:, 1] + h[:, 1]) - (tr[:, 0] + h[:, 0])) < b_sub
    mism_s = sub[cells][ok] != exp_sub
    assert np.all(near_s[mism_s]), f"{mism_s.sum()} sub-label mismatches, {near_s.sum()} near-ties"
    return int(ok.sum()), int(mism.sum()), int(mism_s.sum())


def check_moves(P, g, alpha, beta):
    """Split and merge log H against the oracle from the GPU's exact statistics."""
    from oracle.model import log_hastings_merge, log_hastings_split
    nsub, Ssub, sumlogq = g.stats()
    K = nsub.shape[0]
    g.split_merge(1)
    chain, log_h, _ = P.dpmm_debug_moves(g.ctx, g.kmax)
    assert chain == 1 and log_h.size == K
    for k in range(K):
        n0, n1 = int(nsub[k, 0]), int(nsub[k, 1])
        if n0 < 1 or n1 < 1:
            assert np.isnan(log_h[k])
            continue
        ref = log_hastings_split(n0, n1, Ssub[k, 0], Ssub[k, 1], alpha, beta, float(sumlogq[k]))
        assert abs(log_h[k] - ref) <= 1e-10 * abs(ref) + 1e-6, (k, log_h[k], ref)
    nsub, Ssub, _ = g.stats()
    g.split_merge(2)
    chain, log_h, pairs = P.dpmm_debug_moves(g.ctx, g.kmax)
    assert chain == 2
    nk, S = nsub.sum(axis=1), Ssub.sum(axis=1)
    for (a, b), lh in zip(pairs, log_h):
        ref = log_hastings_merge(int(nk[a]), int(nk[b]), S[a], S[b], alpha, beta)
        assert abs(lh - ref) <= 1e-10 * abs(ref) + 1e-6, (a, b, lh, ref)


def test_pbmc68k_bench_configuration(P):
    """68,000 x 1,000, the bench's main configuration (dense-tile BF16 engine,
    alpha 1, beta 0.1, kmax 256, seed 42)."""
    from paper_1812_10048_gb300 import synth
    ds = synth.pbmc68k()
    g = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.1, kmax=256, seed=42,
                  engine=P.ENGINE_AUTO)
    g.step(6)
    labels, sub, K, _, _ = g.get_state()
    nsub, Ssub, _ = g.stats()
    rng = np.random.default_rng(68)
    check_stats_properties(ds, labels, sub, K, nsub, Ssub, rng.choice(ds.D, 24, replace=False))
    from oracle.sampler import sufficient_stats
    on, oS = sufficient_stats(csr(ds), labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
    before = check_draw(P, g, ds, 1.0, 0.1, 42)
    cells = np.sort(rng.choice(ds.N, 3000, replace=False))
    n_ok, _, _ = check_sampled_labels(P, g, ds, cells, before, 42, bf16=True)
    assert n_ok >= cells.size - 10
    check_moves(P, g, 1.0, 0.1)
    g.close()


def test_pbmc68k_fp32_engine(P):
    from paper_1812_10048_gb300 import synth
    ds = synth.pbmc68k()
    g = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.1, kmax=256, seed=42,
                  engine=P.ENGINE_CSR_FP32)
    g.step(4)
    before = check_draw(P, g, ds, 1.0, 0.1, 42)
    rng = np.random.default_rng(69)
    cells = np.sort(rng.choice(ds.N, 3000, replace=False))
    n_ok, _, _ = check_sampled_labels(P, g, ds, cells, before, 42, bf16=False)
    assert n_ok >= cells.size - 10
    labels, sub, K, _, _ = g.get_state()
    nsub, Ssub, _ = g.stats()
    check_stats_properties(ds, labels, sub, K, nsub, Ssub, rng.choice(ds.D, 24, replace=False))
    g.close()


def test_large_bench_configuration(P):
    """1.3 M x 2,000 with 2% deep cells (counts above 255: the BF16 hi pass)."""
    from paper_1812_10048_gb300 import synth
    ds = synth.large(workers=os.cpu_count())
    g = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.1, kmax=256, seed=42,
                  engine=P.ENGINE_AUTO)
    g.step(3)
    labels, sub, K, _, _ = g.get_state()
    nsub, Ssub, _ = g.stats()
    rng = np.random.default_rng(13)
    check_stats_properties(ds, labels, sub, K, nsub, Ssub, rng.choice(ds.D, 8, replace=False))
    before = check_draw(P, g, ds, 1.0, 0.1, 42)
    deep = np.nonzero(library_sizes(ds) > 5000)[0]
    cells = np.sort(np.concatenate([rng.choice(ds.N, 1500, replace=False),
                                    rng.choice(deep, 500, replace=False)]))
    cells = np.unique(cells)
    n_ok, _, _ = check_sampled_labels(P, g, ds, cells, before, 42, bf16=True)
    assert n_ok >= cells.size - 10
    check_moves(P, g, 1.0, 0.1)
    g.close()


def test_batched_bench_configuration(P):
    """64 datasets (1,000 to 50,000 cells each) in one batch, as bench.py times
    it: every chain's statistics equal a recount from its labels, and two
    chains evolve exactly as they do alone."""
    from paper_1812_10048_gb300 import synth
    dss = synth.batched(workers=os.cpu_count())
    data = [(d.indptr, d.indices, d.data, d.N) for d in dss]
    bs = P.BatchSampler(data, 1000, 1.0, 0.5, kmax=64, seed=42, engine=P.ENGINE_AUTO)
    bs.step(3)
    rng = np.random.default_rng(64)
    for b in range(len(dss)):
        v = bs.chain(b)
        labels, sub, K, _, _ = v.get_state()
        nsub, Ssub, _ = v.stats()
        check_stats_properties(dss[b], labels, sub, K, nsub, Ssub,
                               rng.choice(1000, 4, replace=False))
    for b in (0, 37):
        d = dss[b]
        s = P.Sampler(d.indptr, d.indices, d.data, d.N, 1000, 1.0, 0.5, kmax=64, seed=42,
                      chain_id=b, engine=P.ENGINE_AUTO)
        s.step(3)
        for x, y in zip(bs.chain(b).get_state(), s.get_state()):
            np.testing.assert_array_equal(x, y)
        s.close()
    bs.close()


def test_logml_grad_bench_configuration(P):
    """100,000 x 2,000, K = 25 generating labels: forward log ML and its
    gradients against the FP64 oracle (the grad bench's inputs)."""
    import torch
    from oracle.logml import cluster_stats, log_ml, log_ml_grad
    from paper_1812_10048_gb300 import synth
    ds = synth.grad_workload()
    K = int(ds.labels.max()) + 1
    rng = np.random.default_rng(1005)
    lb = (np.log(0.1) + 0.1 * rng.standard_normal(ds.D)).astype(np.float32)
    la = 0.0
    h = P.LogML(ds.indptr, ds.indices, ds.data, ds.N, ds.D, ds.labels, K)
    n, S = cluster_stats(ds.indptr, ds.indices, ds.data, ds.N, ds.D, ds.labels, K)
    ref = log_ml(n, S, la, lb.astype(np.float64))
    got = h.forward(la, torch.from_numpy(lb).cuda())
    assert abs(got - ref) <= 1e-10 * abs(ref)
    ga_ref, gb_ref = log_ml_grad(n, S, la, lb.astype(np.float64))
    gb = torch.empty(ds.D, dtype=torch.float32, device="cuda")
    ga = h.backward(la, torch.from_numpy(lb).cuda(), gb)
    torch.cuda.synchronize()
    assert abs(ga - ga_ref) <= 1e-9 * max(1.0, abs(ga_ref))
    np.testing.assert_allclose(gb.cpu().numpy(), gb_ref, rtol=2e-4, atol=1e-2)
