"""Batched chains (dpmm_init_batch): one launch per kernel over all chains.

Each chain of a batch must evolve exactly as the single chain with the same
data, seed and chain id: identical labels, sub-labels, K, counters and
(integer) statistics.  The per-cluster sum of log q is an FP64 sum of FP32
atomics whose order is not fixed, so it is compared within rounding.
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
        np.testing.assert_allclose(qb, qs, rtol=1e-5, atol=1e-3)


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
