"""Tensor-core engine: the tcgen05 self-test against numpy, then the dense-tile
label engine against the FP64 oracle."""

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


def to_bf16_bits(x):
    """Round-toward-zero float32 -> bf16 bit patterns, and their exact values."""
    b = (np.ascontiguousarray(x, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)
    v = (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return b, v


@pytest.mark.parametrize("Kd,N", [(64, 16), (64, 64), (128, 96), (192, 128), (256, 256)])
def test_tcgen05_gemm_matches_numpy(P, Kd, N):
    rng = np.random.default_rng(Kd + N)
    A, Av = to_bf16_bits(rng.integers(0, 256, size=(128, Kd)).astype(np.float32))
    B, Bv = to_bf16_bits(rng.standard_normal((N, Kd)).astype(np.float32) * 3)
    C = P.dpmm_debug_tc_gemm(A, B)
    ref = Av @ Bv.T
    np.testing.assert_allclose(C, ref, rtol=2e-6, atol=1e-3 * np.abs(ref).max() * 1e-3 + 1e-4)


# ---------------------------------------------------------------------------
# dense-tile label engine
# ---------------------------------------------------------------------------
TWO_M16 = 2.0 ** -16


@pytest.fixture(scope="module")
def tiny():
    from paper_1812_10048_gb300 import synth
    return synth.tiny()


def injected(P, ds, K, seed, engine=None, kmax=128):
    """GPU chain (dense-tile engine) and oracle chain in the same random state with
    K clusters, with parameters drawn on the GPU and injected back (FP32)."""
    from oracle.sampler import Sampler as OracleSampler
    rng = np.random.default_rng(seed)
    labels = rng.integers(0, K, size=ds.N)
    labels[:K] = np.arange(K)
    sub = rng.integers(0, 2, size=ds.N)
    o = OracleSampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, seed=seed, kmax=kmax)
    o.set_state(labels, sub, K, t=3, m=1)
    g = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, kmax=kmax, seed=seed,
                  engine=P.ENGINE_TILE_BF16 if engine is None else engine)
    P.dpmm_set_state(g.ctx, o.labels, o.sub, o.K, o.t, o.m, o.sumlogq)
    P.dpmm_draw_params(g.ctx)
    logpi, logtheta = P.dpmm_get_params(g.ctx, K, ds.D)
    P.dpmm_set_params(g.ctx, logpi, logtheta)
    return g, o, logpi.astype(np.float64), logtheta.astype(np.float64)


def centred_reference(o, logtheta):
    """FP64 centred scores and the BF16 hi/lo error bound of each (cell, column)."""
    X = o.X.astype(np.float64)
    m = logtheta.mean(axis=0)
    d = logtheta - m[None, :]
    K = logtheta.shape[0] // 3
    order = np.concatenate([np.arange(0, 3 * K, 3),
                            np.stack([np.arange(1, 3 * K, 3), np.arange(2, 3 * K, 3)], 1).ravel()])
    dd = d[order]
    ref = np.asarray(X @ dd.T)
    bound = 2 * TWO_M16 * np.asarray(X @ np.abs(dd).T) + 1e-5 * np.abs(ref) + 1e-3
    return ref, bound


@pytest.mark.parametrize("K", [1, 2, 5, 10, 16, 23, 40])
def test_tile_scores_within_bf16_bound(P, tiny, K):
    g, o, logpi, logtheta = injected(P, tiny, K, seed=100 + K)
    got = P.dpmm_debug_tile_scores(g.ctx, tiny.N, K)
    ref, bound = centred_reference(o, logtheta)
    err = np.abs(got - ref)
    assert np.all(err <= bound), (err.max(), (err / bound).max())


@pytest.mark.parametrize("K", [2, 7, 10, 40])
def test_tile_assign_matches_oracle_except_near_ties(P, tiny, K):
    """The dense-tile label step from an injected state and parameters: every
    label, sub-label, reset and sum of log q equals the FP64 oracle's except
    near-ties within the BF16 hi/lo bound; statistics exact."""
    from oracle.sampler import sufficient_stats
    from .parity import bf16_bound, check_assign, decisions_from_oracle
    g, o, logpi, logtheta = injected(P, tiny, K, seed=200 + K)
    ref = decisions_from_oracle(o, logpi, logtheta, bf16_bound(o.X.astype(np.float64), logtheta))
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


def test_tile_chain_invariants_and_recovery(P, tiny):
    from oracle.ari import adjusted_rand_index
    from oracle.sampler import csr_matrix, sufficient_stats
    g = P.Sampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5, seed=3,
                  engine=P.ENGINE_TILE_BF16)
    g.step(40)
    labels, sub, K, t, m = g.get_state()
    nsub, Ssub, _ = g.stats()
    on, oS = sufficient_stats(csr_matrix(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D),
                              labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
    assert adjusted_rand_index(labels, tiny.labels) > 0.95


def test_tile_engine_small_shapes(P):
    """One partial tile (N < 128), one partial chunk (D < 64), counts above 255."""
    from oracle.sampler import csr_matrix, sufficient_stats
    rng = np.random.default_rng(5)
    N, D = 77, 23
    dense = rng.integers(0, 6, size=(N, D)) * (rng.random((N, D)) < 0.5)
    dense[5, 3] = 1000
    dense[9] = 0
    r, c = np.nonzero(dense)
    indptr = np.concatenate([[0], np.cumsum(np.count_nonzero(dense, axis=1))]).astype(np.int32)
    g = P.Sampler(indptr, c.astype(np.int32), dense[r, c].astype(np.int32), N, D, 1.0, 0.5, seed=4,
                  engine=P.ENGINE_TILE_BF16)
    g.step(8)
    labels, sub, K, _, _ = g.get_state()
    nsub, Ssub, _ = g.stats()
    on, oS = sufficient_stats(csr_matrix(indptr, c, dense[r, c], N, D), labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)


# ---------------------------------------------------------------------------
# blocked copy built on the device by dpmm_init
# ---------------------------------------------------------------------------
def blocked_reference(indptr, indices, data, N, D):
    """The blocked copy from its definition: entries stably ordered by bucket
    (tile * C + chunk, quarter), each segment padded to a multiple of 4."""
    indptr = np.asarray(indptr, np.int64)
    indices = np.asarray(indices, np.int64)
    data = np.asarray(data, np.int64)
    T, C = (N + 127) // 128, (D + 63) // 64
    rows = np.repeat(np.arange(N), np.diff(indptr))
    key = 4 * ((rows // 128) * C + indices // 64) + (rows // 32) % 4
    order = np.argsort(key, kind="stable")
    counts = np.bincount(key, minlength=4 * T * C).reshape(T * C, 4)
    padded = (counts.sum(axis=1) + 3) // 4 * 4
    seg0 = np.concatenate([[0], np.cumsum(padded)[:-1]])
    tptr = np.empty(4 * T * C + 1, np.int64)
    tptr[:-1] = (seg0[:, None] + np.concatenate([np.zeros((T * C, 1), np.int64),
                                                 np.cumsum(counts, axis=1)[:, :3]], axis=1)).ravel()
    tptr[-1] = padded.sum()
    tent = np.zeros(int(padded.sum()), np.uint64)
    ks = key[order]
    first = np.searchsorted(ks, ks, side="left")
    pos = tptr[ks] + (np.arange(ks.size) - first)
    val = ((rows[order] % 128) << 22) | ((indices[order] % 64) << 16) | data[order]
    tent[pos] = val
    return T, C, tptr, tent.astype(np.uint32)


def _layout_case(P, indptr, indices, data, N, D):
    g = P.Sampler(indptr, indices, data, N, D, 1.0, 0.5, kmax=16, seed=1,
                  engine=P.ENGINE_TILE_BF16)
    T, C, tptr, tent = P.dpmm_debug_tile_layout(g.ctx)
    rT, rC, rptr, rent = blocked_reference(indptr, indices, data, N, D)
    assert (T, C) == (rT, rC)
    np.testing.assert_array_equal(tptr, rptr)
    np.testing.assert_array_equal(tent, rent)
    g.close()


def test_blocked_copy_matches_its_definition(P, tiny):
    _layout_case(P, tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D)
    # ragged: N not a multiple of 128 (a partial last quarter), D not a
    # multiple of 64, empty rows, zero counts, a dense row
    rng = np.random.default_rng(21)
    N, D = 301, 70
    dense = rng.integers(0, 4, size=(N, D)) * (rng.random((N, D)) < 0.2)
    dense[::7] = 0
    dense[5] = rng.integers(1, 300, size=D)
    r, c = np.nonzero(dense)
    indptr = np.concatenate([[0], np.cumsum(np.count_nonzero(dense, axis=1))]).astype(np.int32)
    idx, val = c.astype(np.int32), dense[r, c].astype(np.int32)
    val[3] = 0                                      # an explicit zero count
    _layout_case(P, indptr, idx, val, N, D)


def test_blocked_copy_at_the_bench_size(P):
    from paper_1812_10048_gb300 import synth
    ds = synth.pbmc68k()
    _layout_case(P, ds.indptr, ds.indices, ds.data, ds.N, ds.D)


def _engine_after_sweep(P, ds, K, engine):
    rng = np.random.default_rng(K)
    labels = rng.integers(0, K, size=ds.N)
    labels[:K] = np.arange(K)
    sub = rng.integers(0, 2, size=ds.N).astype(np.uint8)
    g = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, kmax=64, seed=5,
                  engine=engine)
    P.dpmm_set_state(g.ctx, labels, sub, K, 3, 0)
    g.sweep(1)
    used = P.dpmm_debug_engine(g.ctx)
    g.close()
    return used


def test_engine_choice_follows_the_measured_density_rule(P):
    """Automatic engine: the tensor-core engine for 3 <= K <= 40 at any density
    and for K <= 2 below 12% density; the CSR engine for K <= 2 at 12% or more
    (where it was measured faster) and for K > 40.  A forced tile engine labels
    every 1 <= K <= 40."""
    from paper_1812_10048_gb300 import synth
    dense = synth.tiny()                                     # ~29% of entries non-zero
    sparse = synth.make_dataset(2000, 500, 4, gamma=0.05, lib_mu=np.log(40.0), lib_sigma=0.3,
                                seed=77)
    assert dense.density >= 0.12 and sparse.density < 0.12, (dense.density, sparse.density)
    assert _engine_after_sweep(P, dense, 2, P.ENGINE_AUTO) == 0
    assert _engine_after_sweep(P, dense, 3, P.ENGINE_AUTO) == 1
    assert _engine_after_sweep(P, dense, 40, P.ENGINE_AUTO) == 1
    assert _engine_after_sweep(P, dense, 41, P.ENGINE_AUTO) == 0
    assert _engine_after_sweep(P, sparse, 2, P.ENGINE_AUTO) == 1
    assert _engine_after_sweep(P, dense, 2, P.ENGINE_TILE_BF16) == 1
    assert _engine_after_sweep(P, dense, 2, P.ENGINE_CSR_FP32) == 0


def test_auto_engine_below_the_cut_matches_the_oracle(P, tiny):
    """K = 2 on the dense tiny workload takes the CSR engine under AUTO: labels,
    sub-labels and sums of log q are the FP64 decisions except near-ties of the
    FP32 contraction; statistics exact."""
    from oracle.sampler import sufficient_stats
    from .parity import check_assign, decisions_from_oracle, fp32_bound
    g, o, logpi, logtheta = injected(P, tiny, 2, seed=311, engine=P.ENGINE_AUTO)
    ref = decisions_from_oracle(o, logpi, logtheta, fp32_bound(o.X.astype(np.float64), logtheta))
    t0 = o.t
    o.assign_and_update(logpi, logtheta)
    P.dpmm_assign(g.ctx)
    assert P.dpmm_debug_engine(g.ctx) == 0
    lab, sb, Kg, t, m = g.get_state()
    assert t == o.t and Kg == o.K
    nsub, Ssub, sq = g.stats()
    check_assign(ref, 2, Kg, lab, sb, sq, o.seed, o.chain_id, t0)
    on, oS = sufficient_stats(o.X, lab, sb, Kg)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
