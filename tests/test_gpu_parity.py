"""GPU path vs FP64 oracle, through the C ABI (libdpmm.so).

Tolerances (derived from the arithmetic):
* generator words, labels given identical perturbed-score order, integer
  statistics: bit-exact;
* FP32 scores: |s_gpu - s_oracle| <= 1e-5 |s| + 1e-4 (eq. 4 / eq. 26 sums of
  up to a few thousand FP32 products);
* labels: identical except cells whose top-two perturbed scores differ by
  less than that bound (near-ties);
* log theta draws: rtol 1e-5, atol 1e-4, except rare Marsaglia-Tsang
  accept/reject flips where FP32 and FP64 land on opposite sides of the
  acceptance boundary (counted, at most 0.1% of the draws);
* FP64 Hastings ratios: rtol 1e-10.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SCORE_RTOL, SCORE_ATOL = 1e-5, 1e-4


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1812_10048_gb300 import build
    build.build()
    import paper_1812_10048_gb300 as P
    torch.cuda.init()
    return P


@pytest.fixture(scope="module")
def tiny():
    from paper_1812_10048_gb300 import synth
    return synth.tiny()


def make_pair(P, ds, alpha=1.0, beta=0.5, seed=42, kmax=64, **kw):
    """A GPU chain on the FP32 CSR engine (the FP32 tolerances of this file) and an
    oracle chain with the same seed."""
    from oracle.sampler import Sampler as OracleSampler
    kw.setdefault("engine", P.ENGINE_CSR_FP32)
    g = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, alpha, beta, kmax=kmax, seed=seed, **kw)
    o = OracleSampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, alpha, beta, seed=seed, kmax=kmax)
    return g, o


def oracle_warm_state(ds, n_steps=4, alpha=1.0, beta=0.5, seed=7):
    from oracle.sampler import Sampler as OracleSampler
    o = OracleSampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, alpha, beta, seed=seed)
    for _ in range(n_steps):
        o.sweep()
        o.split_merge(0)
    return o


def test_device_philox_matches_oracle(P):
    from oracle import philox
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    seed = 0x1234567890ABCDEF
    got = P.dpmm_debug_philox(ctr, seed)
    ref = philox.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], seed & 0xFFFFFFFF, seed >> 32)
    np.testing.assert_array_equal(got, ref)


def test_curand_philox_reference_matches_oracle(P):
    """cuRAND's Philox4_32_10: consecutive outputs of curand_init(seed, 0, 0)."""
    from oracle import philox
    seed = 987654321
    got = P.dpmm_debug_curand_philox(seed, 8)
    ref = philox.philox4x32_10(np.arange(8), 0, 0, 0, seed & 0xFFFFFFFF, seed >> 32)
    np.testing.assert_array_equal(got, ref)


def test_init_state_and_stats_match_oracle(P, tiny):
    g, o = make_pair(P, tiny)
    labels, sub, K, t, m = g.get_state()
    assert K == 1 and t == 0 and m == 0
    np.testing.assert_array_equal(labels, o.labels)
    np.testing.assert_array_equal(sub, o.sub)
    nsub, Ssub, sumlogq = g.stats()
    on, oS = o.stats()
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
    np.testing.assert_allclose(sumlogq, o.sumlogq, rtol=1e-12)


def inject(P, g, o):
    P.dpmm_set_state(g.ctx, o.labels, o.sub, o.K, o.t, o.m, o.sumlogq)


def test_set_state_roundtrip_and_stats_exact(P, tiny):
    o = oracle_warm_state(tiny)
    g, _ = make_pair(P, tiny)
    inject(P, g, o)
    labels, sub, K, t, m = g.get_state()
    np.testing.assert_array_equal(labels, o.labels)
    np.testing.assert_array_equal(sub, o.sub)
    assert (K, t, m) == (o.K, o.t, o.m)
    nsub, Ssub, _ = g.stats()
    on, oS = o.stats()
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)


def test_draw_params_match_oracle(P, tiny):
    from oracle.sampler import draw_pi, draw_theta
    o = oracle_warm_state(tiny)
    g, _ = make_pair(P, tiny, seed=7)
    inject(P, g, o)
    P.dpmm_draw_params(g.ctx)
    logpi, logtheta = P.dpmm_get_params(g.ctx, o.K, tiny.D)
    nsub, Ssub = o.stats()
    ref_pi = draw_pi(nsub.sum(axis=1), o.alpha, o.seed, o.chain_id, o.t)
    ref_th = draw_theta(Ssub, o.beta, o.seed, o.chain_id, o.t)
    bad_pi = ~np.isclose(logpi, ref_pi, rtol=1e-5, atol=1e-4)
    assert bad_pi.sum() == 0, (logpi, ref_pi)
    bad = ~np.isclose(logtheta, ref_th, rtol=1e-5, atol=1e-4)
    # a flip changes one Gamma variate, which shifts the whole row's normaliser slightly;
    # count flips as elements far outside tolerance
    flips = (np.abs(logtheta - ref_th) > 1e-2).sum()
    assert flips <= max(2, 1e-3 * ref_th.size), flips
    rows_with_flip = np.unique(np.nonzero(np.abs(logtheta - ref_th) > 1e-2)[0])
    clean = np.setdiff1d(np.arange(ref_th.shape[0]), rows_with_flip)
    assert bad[clean].sum() == 0


def oracle_perturbed(o, logpi, logtheta):
    """Oracle perturbed scores (FP64) for the injected parameters."""
    from oracle.sampler import label_gumbels
    from oracle.model import multinomial_scores
    X = o.X.astype(np.float64)
    s = multinomial_scores(X, logpi[:o.K], logtheta[0::3])
    return s, s + label_gumbels(o.N, o.K, o.seed, o.chain_id, o.t)


def test_assign_with_injected_params_matches_oracle(P, tiny):
    """Labels, sub-labels, compaction, resets and sum log q of one label step
    from the oracle's state and the GPU's drawn parameters: every cell's
    decision equals the FP64 one except near-ties of the FP32 contraction."""
    from .parity import check_assign, decisions_from_oracle, fp32_bound
    o = oracle_warm_state(tiny)
    g, _ = make_pair(P, tiny, seed=7)
    inject(P, g, o)
    P.dpmm_draw_params(g.ctx)
    logpi32, logtheta32 = P.dpmm_get_params(g.ctx, o.K, tiny.D)
    P.dpmm_set_params(g.ctx, logpi32, logtheta32)
    logpi, logtheta = logpi32.astype(np.float64), logtheta32.astype(np.float64)
    ref = decisions_from_oracle(o, logpi, logtheta, fp32_bound(o.X.astype(np.float64), logtheta))
    K0, t0 = o.K, o.t
    o.assign_and_update(logpi, logtheta)
    P.dpmm_assign(g.ctx)
    labels, sub, K, t, m = g.get_state()
    assert t == o.t and K == o.K
    nsub, Ssub, sq = g.stats()
    checked, _ = check_assign(ref, K0, K, labels, sub, sq, o.seed, o.chain_id, t0)
    assert checked >= 1
    # statistics are exact for the GPU's own labels
    from oracle.sampler import sufficient_stats
    on, oS = sufficient_stats(o.X, labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)


def test_scores_match_oracle_fp64(P, tiny):
    o = oracle_warm_state(tiny)
    g, _ = make_pair(P, tiny, seed=7)
    inject(P, g, o)
    P.dpmm_draw_params(g.ctx)
    logpi32, logtheta32 = P.dpmm_get_params(g.ctx, o.K, tiny.D)
    cells = np.arange(0, tiny.N, 7)
    got = P.dpmm_debug_scores(g.ctx, cells, o.K)
    X = o.X[cells].astype(np.float64)
    lt = logtheta32.astype(np.float64)
    ref_c = np.asarray(X @ lt[0::3].T) + logpi32[:o.K].astype(np.float64)
    ref_s = np.stack([np.asarray(X @ lt[1::3].T), np.asarray(X @ lt[2::3].T)], axis=2).reshape(len(cells), -1)
    ref = np.concatenate([ref_c, ref_s], axis=1)
    np.testing.assert_allclose(got, ref, rtol=SCORE_RTOL, atol=SCORE_ATOL)


def test_one_full_sweep_agrees_with_oracle(P, tiny):
    """One whole sweep (the GPU draws its own FP32 parameters): the draws
    agree with the oracle's FP64 ones (test_draw_params_match_oracle), and the
    labels, sub-labels and sums of log q are the FP64 decisions from the
    parameters the GPU drew, except near-ties."""
    from .parity import check_assign, decisions_from_oracle, fp32_bound
    o = oracle_warm_state(tiny)
    g, _ = make_pair(P, tiny, seed=7)
    inject(P, g, o)
    K0, t0 = o.K, o.t
    g.sweep(1)
    labels, sub, K, t, m = g.get_state()
    assert t == t0 + 1
    _, _, sq = g.stats()
    # the sweep's own draws (rows of the pre-compaction clusters)
    logpi32, logtheta32 = P.dpmm_get_params(g.ctx, K0, tiny.D)
    logpi, logtheta = logpi32.astype(np.float64), logtheta32.astype(np.float64)
    ref = decisions_from_oracle(o, logpi, logtheta, fp32_bound(o.X.astype(np.float64), logtheta))
    check_assign(ref, K0, K, labels, sub, sq, o.seed, o.chain_id, t0)
    # the oracle's own sweep (its FP64 draws): the same decisions except where
    # the difference of the two draws, bounded per cell and column, or the
    # contraction's error can move them
    lp_o, lt_o = o.draw_params()
    X = o.X.astype(np.float64)
    dpar = np.abs(np.asarray(X @ (logtheta - lt_o).T))
    dpar[:, 0::3] += np.abs(logpi[:K0] - lp_o[:K0])[None, :]
    ref_o = decisions_from_oracle(o, lp_o, lt_o, fp32_bound(X, logtheta) + dpar)
    check_assign(ref_o, K0, K, labels, sub, sq, o.seed, o.chain_id, t0)


@pytest.mark.parametrize("mode", [1, 2])
def test_split_merge_matches_oracle(P, tiny, mode):
    o = oracle_warm_state(tiny, n_steps=3)
    g, _ = make_pair(P, tiny, seed=7)
    inject(P, g, o)
    n_acc = g.split_merge(mode)
    chain, log_h, pair_ab = P.dpmm_debug_moves(g.ctx, g.kmax)
    assert chain == mode
    if mode == 1:
        ref = o.split_log_hastings()
        assert np.array_equal(np.isnan(log_h), np.isnan(ref))
        ok = ~np.isnan(ref)
        np.testing.assert_allclose(log_h[ok], ref[ok], rtol=1e-10, atol=1e-8)
    else:
        pairs = o.merge_pairs()
        np.testing.assert_array_equal(pair_ab, np.array(pairs, dtype=np.int32).reshape(-1, 2))
        ref = o.merge_log_hastings(pairs)
        np.testing.assert_allclose(log_h, ref, rtol=1e-10, atol=1e-8)
    ref_acc = o.split_merge(mode)
    assert n_acc == ref_acc
    labels, sub, K, t, m = g.get_state()
    assert (K, m) == (o.K, o.m)
    np.testing.assert_array_equal(labels, o.labels)
    np.testing.assert_array_equal(sub, o.sub)
    nsub, Ssub, sumlogq = g.stats()
    on, oS = o.stats()
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
    np.testing.assert_allclose(sumlogq, o.sumlogq, rtol=1e-6, atol=1e-6)


def test_forced_split_then_merge_and_capacity(P):
    rng = np.random.default_rng(6)
    n, D = 40, 3
    x = rng.integers(1, 4, size=(n, D))
    indptr = (np.arange(n + 1) * D).astype(np.int32)
    indices = np.tile(np.arange(D), n).astype(np.int32)
    g = P.Sampler(indptr, indices, x.ravel(), n, D, 1e300, 1.0, kmax=2, seed=1)
    _, sub0, _, _, _ = g.get_state()
    assert g.split_merge(1) == 1
    labels, _, K, _, _ = g.get_state()
    assert K == 2
    np.testing.assert_array_equal(labels, sub0)
    assert g.split_merge(1) == 0          # capacity: kmax = 2
    g2 = P.Sampler(indptr, indices, x.ravel(), n, D, 1e-300, 1.0, kmax=4, seed=1)
    P.dpmm_set_state(g2.ctx, sub0, np.zeros(n, np.uint8), 2)
    assert g2.split_merge(2) == 1
    labels, sub, K, _, _ = g2.get_state()
    assert K == 1 and np.all(labels == 0)
    np.testing.assert_array_equal(sub, sub0)


def test_graph_step_equals_eager_calls(P, tiny):
    g1, _ = make_pair(P, tiny, seed=11)
    g2, _ = make_pair(P, tiny, seed=11)
    for _ in range(5):
        g1.sweep(1)
        P.dpmm_split_merge(g1.ctx, 0, want_count=False)
    g2.step(5)
    a, b = g1.get_state(), g2.get_state()
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[2:] == b[2:]


def test_chain_invariants_and_recovery(P, tiny):
    from oracle.ari import adjusted_rand_index
    from oracle.sampler import sufficient_stats, csr_matrix
    g = P.Sampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5, seed=3)
    g.step(40)
    labels, sub, K, t, m = g.get_state()
    assert (t, m) == (40, 40)
    assert labels.min() >= 0 and labels.max() < K
    nsub, Ssub, _ = g.stats()
    X = csr_matrix(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D)
    on, oS = sufficient_stats(X, labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
    assert np.all(nsub.sum(axis=1) > 0)
    assert adjusted_rand_index(labels, tiny.labels) > 0.95


def test_resume_is_bit_identical(P, tiny):
    g1, _ = make_pair(P, tiny, seed=5)
    g1.step(6)
    labels, sub, K, t, m = g1.get_state()
    _, _, sq = g1.stats()
    g2, _ = make_pair(P, tiny, seed=5)
    P.dpmm_set_state(g2.ctx, labels, sub, K, t, m, sq)
    g1.step(4)
    g2.step(4)
    a, b = g1.get_state(), g2.get_state()
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_edge_cases_empty_rows_wide_counts_single_cell(P):
    from oracle.sampler import sufficient_stats, csr_matrix
    rng = np.random.default_rng(9)
    # empty rows and counts above 65535 (unpacked storage path)
    N, D = 300, 17
    dense = rng.integers(0, 5, size=(N, D)) * (rng.random((N, D)) < 0.3)
    dense[::10] = 0
    dense[3, 2] = 70000
    r, c = np.nonzero(dense)
    indptr = np.concatenate([[0], np.cumsum(np.count_nonzero(dense, axis=1))]).astype(np.int32)
    g = P.Sampler(indptr, c.astype(np.int32), dense[r, c].astype(np.int32), N, D, 1.0, 0.3, seed=2)
    g.step(10)
    labels, sub, K, _, _ = g.get_state()
    nsub, Ssub, _ = g.stats()
    on, oS = sufficient_stats(csr_matrix(indptr, c, dense[r, c], N, D), labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
    # a single cell, a single gene
    g1 = P.Sampler(np.array([0, 1], np.int32), np.array([0], np.int32), np.array([5], np.int32),
                   1, 1, 1.0, 1.0, seed=1)
    g1.step(3)
    labels, _, K, _, _ = g1.get_state()
    assert K == 1 and labels[0] == 0


def test_no_cells_or_no_genes_are_rejected(P):
    empty = np.zeros(0, np.int32)
    with pytest.raises(P.DpmmError, match="EINVAL"):
        P.Sampler(np.zeros(1, np.int32), empty, empty, 0, 5, 1.0, 1.0)
    with pytest.raises(P.DpmmError, match="EINVAL"):
        P.Sampler(np.zeros(3, np.int32), empty, empty, 2, 0, 1.0, 1.0)


@pytest.mark.parametrize("engine", ["csr_fp32", "tile_bf16"])
def test_matrix_without_counts(P, engine):
    """No cell has a count: eq. 4 labels come from log pi and the Gumbels
    alone and eq. 8 sub-labels from the n-bar weights.  One label step from an
    injected K = 4 state agrees with the FP64 decisions on the same Philox
    words; a chain keeps valid labels and exact (all-zero) S-bar."""
    from types import SimpleNamespace
    from oracle.sampler import Sampler as OracleSampler, sufficient_stats
    from .parity import bf16_bound, check_assign, decisions_from_oracle, fp32_bound
    N, D = 700, 40
    empty = np.zeros(0, np.int32)
    ds = SimpleNamespace(indptr=np.zeros(N + 1, np.int32), indices=empty, data=empty, N=N, D=D)
    eng = P.ENGINE_CSR_FP32 if engine == "csr_fp32" else P.ENGINE_TILE_BF16
    rng = np.random.default_rng(17)
    labels0 = rng.permutation(np.arange(N) % 4)
    sub0 = rng.integers(0, 2, size=N)
    o = OracleSampler(ds.indptr, ds.indices, ds.data, N, D, 1.0, 0.5, seed=7)
    n0 = np.bincount(labels0, minlength=4)
    o.set_state(labels0, sub0, 4, t=3, m=3, sumlogq=n0 * np.log(0.5))
    g, _ = make_pair(P, ds, seed=7, engine=eng)
    inject(P, g, o)
    P.dpmm_draw_params(g.ctx)
    logpi32, logtheta32 = P.dpmm_get_params(g.ctx, o.K, D)
    P.dpmm_set_params(g.ctx, logpi32, logtheta32)
    logpi, logtheta = logpi32.astype(np.float64), logtheta32.astype(np.float64)
    bound = (fp32_bound if engine == "csr_fp32" else bf16_bound)(o.X.astype(np.float64), logtheta)
    ref = decisions_from_oracle(o, logpi, logtheta, bound)
    K0, t0 = o.K, o.t
    o.assign_and_update(logpi, logtheta)
    P.dpmm_assign(g.ctx)
    assert P.dpmm_debug_engine(g.ctx) == (1 if engine == "tile_bf16" else 0)
    labels, sub, K, t, m = g.get_state()
    assert t == o.t and K == o.K
    nsub, Ssub, sq = g.stats()
    checked, _ = check_assign(ref, K0, K, labels, sub, sq, o.seed, o.chain_id, t0)
    assert checked >= 1
    # a chain of sweeps and moves on the empty matrix
    g.step(20)
    labels, sub, K, _, _ = g.get_state()
    assert 1 <= K and labels.min() >= 0 and labels.max() < K
    nsub, Ssub, _ = g.stats()
    on, oS = sufficient_stats(o.X, labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
    assert not np.any(Ssub)


def _wide_matrix(D, big, seed=23):
    """260 cells (two full 128-cell tiles and a ragged one) over D genes, about
    30 genes a cell, the last gene used, counts of 255, 256-999 and `big`."""
    from types import SimpleNamespace
    rng = np.random.default_rng(seed)
    N = 260
    cols_l, x_l = [], []
    for i in range(N):
        cols = np.unique(rng.integers(0, D, size=30))
        if i % 7 == 0:
            cols = np.unique(np.append(cols, D - 1))
        x = rng.integers(1, 6, size=cols.size)
        if i % 11 == 0:
            x[0] = big
        if i % 5 == 0:
            x[-1] = rng.integers(256, 1000)
        if i % 13 == 0:
            x[rng.integers(0, cols.size)] = 255
        cols_l.append(cols.astype(np.int32))
        x_l.append(x.astype(np.int32))
    indptr = np.concatenate([[0], np.cumsum([c.size for c in cols_l])]).astype(np.int32)
    return SimpleNamespace(indptr=indptr, indices=np.concatenate(cols_l),
                           data=np.concatenate(x_l), N=N, D=D)


def _one_label_step_against_fp64(P, ds, engine, bound_fn):
    """One label step of a GPU chain from an injected K = 3 state, checked
    against the FP64 decisions from the parameters the GPU drew; statistics
    exact.  Returns the GPU chain."""
    from oracle.sampler import Sampler as OracleSampler, sufficient_stats
    from .parity import check_assign, decisions_from_oracle
    rng = np.random.default_rng(29)
    labels0 = rng.permutation(np.arange(ds.N) % 3)
    sub0 = rng.integers(0, 2, size=ds.N)
    o = OracleSampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, seed=5)
    o.set_state(labels0, sub0, 3, t=2, m=2,
                sumlogq=np.bincount(labels0, minlength=3) * np.log(0.5))
    g, _ = make_pair(P, ds, seed=5, engine=engine)
    inject(P, g, o)
    P.dpmm_draw_params(g.ctx)
    logpi32, logtheta32 = P.dpmm_get_params(g.ctx, o.K, ds.D)
    P.dpmm_set_params(g.ctx, logpi32, logtheta32)
    logpi, logtheta = logpi32.astype(np.float64), logtheta32.astype(np.float64)
    ref = decisions_from_oracle(o, logpi, logtheta, bound_fn(o.X.astype(np.float64), logtheta))
    K0, t0 = o.K, o.t
    o.assign_and_update(logpi, logtheta)
    P.dpmm_assign(g.ctx)
    labels, sub, K, t, m = g.get_state()
    assert t == o.t and K == o.K
    nsub, Ssub, sq = g.stats()
    checked, _ = check_assign(ref, K0, K, labels, sub, sq, o.seed, o.chain_id, t0)
    assert checked >= 1
    on, oS = sufficient_stats(o.X, labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
    return g


@pytest.mark.parametrize("engine", ["csr_fp32", "tile_bf16"])
def test_widest_packed_matrix(P, engine):
    """The packed form's limits: 65,536 genes (the last one used) and counts
    up to 65,535, with high bytes for the tensor-core form's second plane."""
    from .parity import bf16_bound, fp32_bound
    from .test_gpu_tile import blocked_reference
    ds = _wide_matrix(65536, 65535)
    tile = engine == "tile_bf16"
    g = _one_label_step_against_fp64(P, ds, P.ENGINE_TILE_BF16 if tile else P.ENGINE_CSR_FP32,
                                     bf16_bound if tile else fp32_bound)
    assert P.dpmm_debug_engine(g.ctx) == (1 if tile else 0)
    if tile:
        T, C, tptr, tent = P.dpmm_debug_tile_layout(g.ctx)
        rT, rC, rptr, rent = blocked_reference(ds.indptr, ds.indices, ds.data, ds.N, ds.D)
        assert (T, C) == (rT, rC) == (3, 1024)
        np.testing.assert_array_equal(tptr, rptr)
        np.testing.assert_array_equal(tent, rent)


@pytest.mark.parametrize("D, big", [(65537, 65535), (1000, 65536)])
def test_tile_engine_on_unpackable_counts_runs_the_csr_engine(P, D, big):
    """One gene too many or one count too large for the packed entries: a
    chain that asks for the tensor-core engine is labelled by the FP32 CSR
    engine, with the FP32 decisions."""
    from .parity import fp32_bound
    ds = _wide_matrix(D, big)
    g = _one_label_step_against_fp64(P, ds, P.ENGINE_TILE_BF16, fp32_bound)
    assert P.dpmm_debug_engine(g.ctx) == 0


def test_invalid_inputs_raise(P):
    ok_ptr = np.array([0, 1, 2], np.int32)
    with pytest.raises(P.DpmmError, match="EINVAL"):
        P.Sampler(ok_ptr, np.array([0, 5], np.int32), np.array([1, 1], np.int32), 2, 3, 1.0, 1.0)
    with pytest.raises(P.DpmmError, match="EINVAL"):
        P.Sampler(np.array([0, 2, 1], np.int32), np.array([0, 1], np.int32),
                  np.array([1, 1], np.int32), 2, 3, 1.0, 1.0)
    with pytest.raises(P.DpmmError, match="EINVAL"):
        P.Sampler(ok_ptr, np.array([0, 1], np.int32), np.array([1, -1], np.int32), 2, 3, 1.0, 1.0)
    with pytest.raises(P.DpmmError, match="EINVAL"):
        P.Sampler(ok_ptr, np.array([0, 1], np.int32), np.array([1, 1], np.int32), 2, 3, 0.0, 1.0)
    with pytest.raises(P.DpmmError, match="EINVAL"):
        P.Sampler(ok_ptr, np.array([0, 1], np.int32), np.array([1, 1], np.int32), 2, 3, 1.0, 1.0,
                  kmax=0)
    with pytest.raises(P.DpmmError, match="EOVERFLOW"):
        big = np.full(70000, 65535, np.int32)
        P.Sampler(np.arange(70001, dtype=np.int32), np.zeros(70000, np.int32), big, 70000, 1, 1.0, 1.0)


def test_phase_timing_events_in_graph(P, tiny):
    g, _ = make_pair(P, tiny, seed=13)
    P.dpmm_profile(g.ctx, True)
    g.step(3)
    ms = P.dpmm_phase_times(g.ctx, 5)
    assert np.all(ms > 0) and np.all(ms < 1000)
    g.sweep(1)                      # eager calls record the same events
    ms2 = P.dpmm_phase_times(g.ctx, 4)
    assert np.all(ms2 > 0)


@pytest.mark.parametrize("K", [2, 4, 8, 14, 16, 24, 32, 40, 120])
def test_assign_parity_across_kernel_variants(P, tiny, K):
    """Every label-kernel variant (lanes per column P = 4..32 with and without spare
    lanes, fused and separate statistics, shared-memory and global tables for K > 32)
    against the oracle from an injected state and injected parameters."""
    _assign_parity(P, tiny, K, P.ENGINE_CSR_FP32)


@pytest.mark.parametrize("K", [41, 57, 120])
def test_tile_configuration_above_40_clusters(P, tiny, K):
    """With the dense-tile engine built but K > 40, the CSR kernel labels the cells
    and the tile statistics kernel counts them from the blocked copy through its
    global-memory partial slots: labels as in the CSR configuration, statistics
    exact."""
    _assign_parity(P, tiny, K, P.ENGINE_AUTO)


def _assign_parity(P, tiny, K, engine):
    from oracle.sampler import Sampler as OracleSampler, sufficient_stats
    rng = np.random.default_rng(K)
    labels = rng.integers(0, K, size=tiny.N)
    labels[:K] = np.arange(K)
    sub = rng.integers(0, 2, size=tiny.N)
    o = OracleSampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5, seed=17,
                      kmax=128)
    o.set_state(labels, sub, K, t=5, m=2)
    g = P.Sampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5, kmax=128, seed=17,
                  engine=engine)
    P.dpmm_set_state(g.ctx, o.labels, o.sub, o.K, o.t, o.m, o.sumlogq)
    P.dpmm_draw_params(g.ctx)
    logpi32, logtheta32 = P.dpmm_get_params(g.ctx, K, tiny.D)
    P.dpmm_set_params(g.ctx, logpi32, logtheta32)
    logpi, logtheta = logpi32.astype(np.float64), logtheta32.astype(np.float64)
    s, _ = oracle_perturbed(o, logpi, logtheta)
    cells = np.arange(0, tiny.N, 37)
    got = P.dpmm_debug_scores(g.ctx, cells, K)
    np.testing.assert_allclose(got[:, :K], s[cells], rtol=SCORE_RTOL, atol=SCORE_ATOL)
    from .parity import check_assign, decisions_from_oracle, fp32_bound
    ref = decisions_from_oracle(o, logpi, logtheta, fp32_bound(o.X.astype(np.float64), logtheta))
    t0 = o.t
    o.assign_and_update(logpi, logtheta)
    P.dpmm_assign(g.ctx)
    lab, sb, Kg, t, m = g.get_state()
    assert t == o.t and Kg == o.K
    nsub, Ssub, sq = g.stats()
    check_assign(ref, K, Kg, lab, sb, sq, o.seed, o.chain_id, t0)
    on, oS = sufficient_stats(o.X, lab, sb, Kg)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)


def test_init_from_device_and_pinned_arrays(P, tiny):
    """dpmm_init takes host, pinned host or device arrays: the chains are
    identical, and a bad entry in device memory is reported as from the host."""
    import torch
    args = (tiny.N, tiny.D, 1.0, 0.5)
    kw = dict(seed=5, kmax=32)
    a = P.Sampler(tiny.indptr, tiny.indices, tiny.data, *args, **kw)
    dev = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32)).cuda()
           for x in (tiny.indptr, tiny.indices, tiny.data)]
    pin = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32)).pin_memory()
           for x in (tiny.indptr, tiny.indices, tiny.data)]
    torch.cuda.synchronize()
    b = P.Sampler(dev[0], dev[1], dev[2], *args, **kw)
    c = P.Sampler(pin[0], pin[1], pin[2], *args, **kw)
    for s in (a, b, c):
        s.step(6)
    for x, y, z in zip(a.get_state(), b.get_state(), c.get_state()):
        np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(x, z)
    bad = dev[1].clone()
    bad[17] = tiny.D
    torch.cuda.synchronize()
    with pytest.raises(P.DpmmError, match="column index .* at entry 17"):
        P.Sampler(dev[0], bad, dev[2], *args, **kw)
    badv = dev[2].clone()
    badv[3] = -2
    torch.cuda.synchronize()
    with pytest.raises(P.DpmmError, match="negative count -2 at entry 3"):
        P.Sampler(dev[0], dev[1], badv, *args, **kw)


@pytest.mark.parametrize("engine", ["tile", "csr", "csr_large_k"])
def test_sum_log_q_is_bit_identical_between_runs(P, tiny, engine):
    """The per-cluster sums of log q are exact integer sums of 2^-32 units, so
    the same label step run twice from the same state gives the same bits,
    whatever order the atomics took; two chains with the same seed stay
    bit-identical in every output over whole steps (split decisions read
    these sums)."""
    eng = P.ENGINE_TILE_BF16 if engine == "tile" else P.ENGINE_CSR_FP32
    K = 48 if engine == "csr_large_k" else 6
    rng = np.random.default_rng(31)
    labels = rng.integers(0, K, size=tiny.N)
    labels[:K] = np.arange(K)
    sub = rng.integers(0, 2, size=tiny.N).astype(np.uint8)
    g = P.Sampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5, kmax=64,
                  seed=3, engine=eng)
    outs = []
    for _ in range(3):
        P.dpmm_set_state(g.ctx, labels, sub, K, 4, 1)
        g.sweep(1)
        outs.append((g.get_state(), g.stats()))
    for (st, sts) in outs[1:]:
        for x, y in zip(st, outs[0][0]):
            np.testing.assert_array_equal(x, y)
        for x, y in zip(sts, outs[0][1]):
            np.testing.assert_array_equal(x, y)
    a = P.Sampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5, kmax=64,
                  seed=8, engine=eng)
    b = P.Sampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5, kmax=64,
                  seed=8, engine=eng)
    a.step(12)
    b.step(12)
    for x, y in zip(a.get_state(), b.get_state()):
        np.testing.assert_array_equal(x, y)
    for x, y in zip(a.stats(), b.stats()):
        np.testing.assert_array_equal(x, y)
