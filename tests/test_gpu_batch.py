"""Batched chains (dpmm_init_batch): one launch per kernel over all chains.

Each chain of a batch must evolve exactly as the single chain with the same
data, seed and chain id: identical labels, sub-labels, K, counters, integer
statistics and per-cluster sums of log q (accumulated as exact integers of
2^-32, so the order of the additions does not matter).  Two chains of a
batch are also checked against the FP64 oracle directly.
"""

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


def datasets(big_count=False):
    from paper_1812_10048_gb300 import synth
    shapes = [(1500, 3), (3100, 6), (700, 4), (2200, 5)]
    out = []
    for b, (N, K) in enumerate(shapes):
        ds = synth.make_dataset(N, 300, K, gamma=0.1, lib_mu=np.log(900.0), lib_sigma=0.5,
                                seed=3000 + b)
        data = ds.data.copy()
        if big_count and b == 1:
            data[5] = 70000   # no packed copy for this chain: CSR engine only
        out.append((ds.indptr, ds.indices, data, ds.N))
    return out


def compare(P, batch, singles, D):
    for b, s in enumerate(singles):
        v = batch.chain(b)
        lb, sb, Kb, tb, mb = v.get_state()
        ls, ss, Ks, ts, ms = s.get_state()
        assert (Kb, tb, mb) == (Ks, ts, ms), b
        np.testing.assert_array_equal(lb, ls)
        np.testing.assert_array_equal(sb, ss)
        nb, Sb, qb = v.stats()
        ns, Ss, qs = s.stats()
        np.testing.assert_array_equal(nb, ns)
        np.testing.assert_array_equal(Sb, Ss)
        np.testing.assert_array_equal(qb, qs)


@pytest.mark.parametrize("engine", ["auto", "csr"])
def test_batch_chains_evolve_as_single_chains(P, engine):
    eng = {"auto": P.ENGINE_AUTO, "csr": P.ENGINE_CSR_FP32}[engine]
    ds = datasets()
    batch = P.BatchSampler(ds, 300, 1.0, 0.5, kmax=32, seed=9, chain_id=4, engine=eng)
    singles = [P.Sampler(d[0], d[1], d[2], d[3], 300, 1.0, 0.5, kmax=32, seed=9, chain_id=4 + b,
                         engine=eng) for b, d in enumerate(ds)]
    batch.sweep(2)
    for s in singles:
        s.sweep(2)
    compare(P, batch, singles, 300)
    batch.split_merge(1)
    for s in singles:
        s.split_merge(1)
    compare(P, batch, singles, 300)
    batch.step(4)
    for s in singles:
        s.step(4)
    compare(P, batch, singles, 300)
    assert batch.plans_applied() == sum(s.plans_applied() for s in singles)
    for s in singles:
        s.close()
    batch.close()


def test_batch_mixing_tile_and_csr_chains(P):
    """A chain whose counts exceed 65,535 has no packed or blocked copy: in a batch
    with dense-tile chains it is labelled and counted by the CSR kernels."""
    ds = datasets(big_count=True)
    batch = P.BatchSampler(ds, 300, 1.0, 0.5, kmax=32, seed=2, engine=P.ENGINE_AUTO)
    singles = [P.Sampler(d[0], d[1], d[2], d[3], 300, 1.0, 0.5, kmax=32, seed=2, chain_id=b,
                         engine=P.ENGINE_AUTO) for b, d in enumerate(ds)]
    batch.step(5)
    for s in singles:
        s.step(5)
    compare(P, batch, singles, 300)
    batch.close()
    for s in singles:
        s.close()


def test_large_batch_of_small_chains(P):
    """600 chains (more than the draw kernel reads side by side, so its
    per-chain loop and the engine-selection kernel's per-chain noise split
    run): three of them against their single-chain runs, bit for bit."""
    from paper_1812_10048_gb300 import synth
    ds = []
    for b in range(600):
        d = synth.make_dataset(40 + (b * 7) % 160, 64, 2 + b % 3, gamma=0.2,
                               lib_mu=np.log(300.0), lib_sigma=0.4, seed=7000 + b)
        ds.append((d.indptr, d.indices, d.data, d.N))
    batch = P.BatchSampler(ds, 64, 1.0, 0.5, kmax=8, seed=13, chain_id=0)
    picks = [0, 311, 599]
    singles = [P.Sampler(ds[b][0], ds[b][1], ds[b][2], ds[b][3], 64, 1.0, 0.5, kmax=8, seed=13,
                         chain_id=b) for b in picks]
    batch.step(4)
    for s in singles:
        s.step(4)
    for b, s in zip(picks, singles):
        v = batch.chain(b)
        got, ref = v.get_state(), s.get_state()
        assert got[2:] == ref[2:], b
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_array_equal(got[1], ref[1])
        for x, y in zip(v.stats(), s.stats()):
            np.testing.assert_array_equal(x, y)
        s.close()
    batch.close()


@pytest.mark.parametrize("engine", ["auto", "tile"])
def test_batch_of_degenerate_and_tile_boundary_chains(P, engine):
    """A batch holding a one-cell chain, chains of 127, 128 and 129 cells (the
    128-cell tile boundary), a chain without any count and a larger one: every
    chain equals its single-chain run bit for bit, and its statistics equal a
    recount of its own labels."""
    from paper_1812_10048_gb300 import synth
    from oracle.sampler import csr_matrix, sufficient_stats
    D = 64
    ds = []
    for b, N in enumerate((1, 127, 128, 129, 500)):
        d = synth.make_dataset(N, D, min(3, N), gamma=0.2, lib_mu=np.log(300.0), lib_sigma=0.4,
                               seed=7700 + b)
        ds.append((d.indptr, d.indices, d.data, d.N))
    empty = np.zeros(0, np.int32)
    ds.insert(3, (np.zeros(301, np.int32), empty, empty, 300))
    eng = {"auto": P.ENGINE_AUTO, "tile": P.ENGINE_TILE_BF16}[engine]
    batch = P.BatchSampler(ds, D, 1.0, 0.5, kmax=16, seed=21, chain_id=0, engine=eng)
    singles = [P.Sampler(d[0], d[1], d[2], d[3], D, 1.0, 0.5, kmax=16, seed=21, chain_id=b,
                         engine=eng) for b, d in enumerate(ds)]
    batch.step(6)
    for s in singles:
        s.step(6)
    compare(P, batch, singles, D)
    for b, (ip, ix, dt, N) in enumerate(ds):
        labels, sub, K, _, _ = batch.chain(b).get_state()
        nsub, Ssub, _ = batch.chain(b).stats()
        on, oS = sufficient_stats(csr_matrix(ip, ix, dt, N, D), labels, sub, K)
        np.testing.assert_array_equal(nsub, on)
        np.testing.assert_array_equal(Ssub, oS)
    for s in singles:
        s.close()
    batch.close()


def test_batch_context_rejects_per_chain_calls(P):
    ds = datasets()[:2]
    batch = P.BatchSampler(ds, 300, kmax=16)
    with pytest.raises(P.DpmmError, match="dpmm_chain"):
        P.dpmm_labels(batch.ctx, ds[0][3])
    with pytest.raises(P.DpmmError, match="outside"):
        P.dpmm_chain(batch.ctx, 2)
    v = batch.chain(1)
    v.close()                      # a view: the batch keeps the chain
    labels, K = batch.chain(1).labels()
    assert labels.shape == (ds[1][3],) and K >= 1
    batch.close()


@pytest.mark.parametrize("engine", ["auto", "csr"])
def test_two_batch_chains_match_the_oracle(P, engine):
    """Chains 0 and 2 of a four-chain batch, started from oracle states: one
    batched sweep gives every cell the FP64 oracle's label and sub-label from
    the parameters the batch drew (except near-ties), with exact statistics;
    one batched split and one merge move from the GPU's state give the
    oracle's log H (FP64, 1e-10) and the oracle's moves exactly."""
    from oracle.sampler import Sampler as OracleSampler, sufficient_stats
    from .parity import bf16_bound, check_assign, decisions_from_oracle, fp32_bound
    eng = {"auto": P.ENGINE_AUTO, "csr": P.ENGINE_CSR_FP32}[engine]
    ds = datasets()
    D = 300
    batch = P.BatchSampler(ds, D, 1.0, 0.5, kmax=32, seed=21, chain_id=0, engine=eng)
    oracles = {}
    for b in (0, 2):
        ip, ix, dt, N = ds[b]
        o = OracleSampler(ip, ix, dt, N, D, 1.0, 0.5, seed=21, chain_id=b, kmax=32)
        for _ in range(3):
            o.sweep()
            o.split_merge(0)
        P.dpmm_set_state(batch.chain(b).ctx, o.labels, o.sub, o.K, o.t, o.m, o.sumlogq)
        oracles[b] = o
    batch.sweep(1)
    for b, o in oracles.items():
        v = batch.chain(b)
        K0, t0 = o.K, o.t
        labels, sub, K, t, m = v.get_state()
        assert t == t0 + 1
        logpi32, logtheta32 = P.dpmm_get_params(v.ctx, K0, D)
        logpi, logtheta = logpi32.astype(np.float64), logtheta32.astype(np.float64)
        X = o.X.astype(np.float64)
        bound = bf16_bound(X, logtheta) if engine == "auto" else fp32_bound(X, logtheta)
        ref = decisions_from_oracle(o, logpi, logtheta, bound)
        nsub, Ssub, sq = v.stats()
        check_assign(ref, K0, K, labels, sub, sq, o.seed, o.chain_id, t0)
        on, oS = sufficient_stats(o.X, labels, sub, K)
        np.testing.assert_array_equal(nsub, on)
        np.testing.assert_array_equal(Ssub, oS)
        o.set_state(labels, sub, K, t, m, sq)
    for mode in (1, 2):
        P.dpmm_split_merge(batch.ctx, mode, want_count=False)
        for b, o in oracles.items():
            v = batch.chain(b)
            chain, log_h, pair_ab = P.dpmm_debug_moves(v.ctx, 32)
            assert chain == mode
            if mode == 1:
                ref = o.split_log_hastings()
                assert np.array_equal(np.isnan(log_h), np.isnan(ref))
                ok = ~np.isnan(ref)
                np.testing.assert_allclose(log_h[ok], ref[ok], rtol=1e-10, atol=1e-8)
            else:
                pairs = o.merge_pairs()
                np.testing.assert_array_equal(pair_ab,
                                              np.array(pairs, dtype=np.int32).reshape(-1, 2))
                np.testing.assert_allclose(log_h, o.merge_log_hastings(pairs), rtol=1e-10,
                                           atol=1e-8)
            o.split_merge(mode)
            labels, sub, K, t, m = v.get_state()
            assert (K, m) == (o.K, o.m)
            np.testing.assert_array_equal(labels, o.labels)
            np.testing.assert_array_equal(sub, o.sub)
            nsub, Ssub, sq = v.stats()
            on, oS = o.stats()
            np.testing.assert_array_equal(nsub, on)
            np.testing.assert_array_equal(Ssub, oS)
            np.testing.assert_allclose(sq, o.sumlogq, rtol=1e-9, atol=1e-9)
    batch.close()
