"""Local Gibbs iterations after the first (opts.local_iters, Section 2.3)
against the FP64 oracle: one iteration in isolation (eq. 19 draws, eq. 8
sub-labels, recounted statistics), chains, batches and argument checks."""

import numpy as np
import pytest

from .test_gpu_batch import compare, datasets
from .test_gpu_parity import oracle_warm_state

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
def tiny():
    from paper_1812_10048_gb300 import synth
    return synth.tiny()


@pytest.mark.parametrize("engine", ["csr", "auto"])
@pytest.mark.parametrize("j", [1, 5])
def test_one_local_iteration_matches_oracle(P, tiny, engine, j):
    from oracle import philox
    from oracle.sampler import eq8_draw, sufficient_stats
    o = oracle_warm_state(tiny, n_steps=3, seed=11)
    o.local_iters = 6
    eng = P.ENGINE_CSR_FP32 if engine == "csr" else P.ENGINE_AUTO
    g = P.Sampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, o.alpha, o.beta,
                  seed=o.seed, kmax=64, engine=eng, local_iters=6)
    P.dpmm_set_state(g.ctx, o.labels, o.sub, o.K, o.t, o.m, o.sumlogq)
    nsub0, _ = o.stats()
    sub0 = o.sub.copy()
    P.dpmm_local_gibbs(g.ctx, j)
    ref_tb = o.local_gibbs(j)                       # (2K, D), row 2k + r
    K, D = o.K, tiny.D
    _, logtheta = P.dpmm_get_params(g.ctx, K, D)
    got_tb = np.empty((2 * K, D))
    got_tb[0::2], got_tb[1::2] = logtheta[1::3], logtheta[2::3]
    # eq. 19 draws: as the sweep's draws, a rare Gamma flip moves one row's normaliser
    far = np.abs(got_tb - ref_tb) > 1e-2
    assert far.sum() <= max(2, 1e-3 * far.size)
    rows = np.setdiff1d(np.arange(2 * K), np.unique(np.nonzero(far)[0]))
    np.testing.assert_allclose(got_tb[rows], ref_tb[rows], rtol=1e-5, atol=1e-4)
    # eq. 8 under the GPU's own theta-bar, decided in FP64: equal but for near-ties
    labels, sub, Kg, t, _ = g.get_state()
    assert Kg == K and t == o.t
    np.testing.assert_array_equal(labels, o.labels)
    X = o.X.astype(np.float64)
    cells = np.arange(o.N)
    lik = np.stack([np.asarray(X @ got_tb[0::2].T)[cells, labels],
                    np.asarray(X @ got_tb[1::2].T)[cells, labels]], axis=1)
    w = nsub0[labels] - np.stack([sub0 == 0, sub0 == 1], axis=1)
    exp_sub, exp_logq = eq8_draw(w, lik, o.seed, o.chain_id, philox.tag_local_sub(j), o.t - 1)
    words = philox.stream_words(o.seed, o.chain_id, philox.tag_local_sub(j), cells, o.t - 1, 0)
    h = philox.uniform_to_gumbel(philox.word_to_uniform(words[:, :2]))
    ww = w.astype(np.float64)
    ww[ww.sum(axis=1) == 0] = 1.0
    with np.errstate(divide="ignore"):
        tr = np.log(ww) + lik
    margin = np.abs((tr[:, 1] + h[:, 1]) - (tr[:, 0] + h[:, 0]))
    near = margin < 1e-5 * np.abs(lik).max(axis=1) + 1e-3
    mism = sub != exp_sub
    assert np.all(near[mism]), f"{mism.sum()} sub-label mismatches, {near.sum()} near-ties"
    # statistics of the GPU's own state, exact; sum log q within FP32 rounding
    nsub, Ssub, sumlogq = g.stats()
    on, oS = sufficient_stats(o.X, labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
    # per cluster without a near-tie flip: the FP64 sum within the summed
    # per-cell bound of the FP32 sub-scores and logarithms
    tol_i = 1e-5 * np.abs(lik).max(axis=1) + 1e-3 + 1e-6 * np.abs(exp_logq) + 1e-6
    dirty = np.bincount(labels[mism], minlength=K) > 0
    ref_q = np.bincount(labels, weights=exp_logq, minlength=K)
    tol = np.bincount(labels, weights=tol_i, minlength=K)
    err = np.abs(sumlogq - ref_q)
    assert np.all(err[~dirty] <= tol[~dirty]), (err[~dirty], tol[~dirty])
    assert (~dirty).sum() >= 1


def test_local_iterations_chain_keeps_statistics_exact(P, tiny):
    from oracle.sampler import sufficient_stats
    g = P.Sampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5, seed=3,
                  kmax=64, local_iters=4)
    g.step(15)
    labels, sub, K, t, _ = g.get_state()
    assert t == 15
    nsub, Ssub, sumlogq = g.stats()
    on, oS = sufficient_stats(g_oracle_X(tiny), labels, sub, K)
    np.testing.assert_array_equal(nsub, on)
    np.testing.assert_array_equal(Ssub, oS)
    assert np.isfinite(sumlogq).all() and (sumlogq <= 0).all()


def g_oracle_X(ds):
    from oracle.sampler import csr_matrix
    return csr_matrix(ds.indptr, ds.indices, ds.data, ds.N, ds.D)


def test_one_local_iteration_is_the_default_chain(P, tiny):
    a = P.Sampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5, seed=5)
    b = P.Sampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5, seed=5,
                  local_iters=1)
    a.step(8)
    b.step(8)
    for x, y in zip(a.get_state(), b.get_state()):
        np.testing.assert_array_equal(x, y)


def test_batched_local_iterations_equal_single_chains(P):
    ds = datasets()
    batch = P.BatchSampler(ds, 300, 1.0, 0.5, kmax=32, seed=9, chain_id=4, local_iters=3)
    singles = [P.Sampler(d[0], d[1], d[2], d[3], 300, 1.0, 0.5, kmax=32, seed=9, chain_id=4 + b,
                         local_iters=3) for b, d in enumerate(ds)]
    batch.step(4)
    for s in singles:
        s.step(4)
    compare(P, batch, singles, 300)
    batch.close()
    for s in singles:
        s.close()


FORMS = [{"local_lanes": v} for v in (4, 8, 16, 32)] + [{"local_stream": 1}]


def same_chain(x, y, what):
    (sx, tx), (sy, ty) = x, y
    assert sx[2:] == sy[2:], what
    for a, c in zip(sx[:2] + tuple(tx), sy[:2] + tuple(ty)):
        np.testing.assert_array_equal(a, c, err_msg=what)


@pytest.mark.parametrize("engine", ["auto", "csr"])
def test_local_forms_give_identical_chains(P, tiny, engine):
    """The contraction's FP32 order is fixed, so the streamed form and the
    group form with any lanes per cell give bit-identical chains (single and
    batched, the batch with one chain lacking the packed rows)."""
    eng = {"auto": P.ENGINE_AUTO, "csr": P.ENGINE_CSR_FP32}[engine]

    def single(tu):
        s = P.Sampler(tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5, kmax=32,
                      seed=21, engine=eng, local_iters=3)
        if tu:
            P.dpmm_set_tuning(s.ctx, **tu)
        s.step(6)
        out = (s.get_state(), s.stats())
        s.close()
        return out

    def batched(tu, big):
        b = P.BatchSampler(datasets(big_count=big), 300, 1.0, 0.5, kmax=32, seed=9, chain_id=4,
                           engine=eng, local_iters=3)
        if tu:
            P.dpmm_set_tuning(b.ctx, **tu)
        b.step(4)
        out = [(b.chain(i).get_state(), b.chain(i).stats()) for i in range(b.B)]
        b.close()
        return out

    ref = single(None)
    brefs = {big: batched(None, big) for big in (False, True)}
    for tu in FORMS:
        same_chain(single(tu), ref, str(tu))
        for big in (False, True):
            for i, (x, y) in enumerate(zip(batched(tu, big), brefs[big])):
                same_chain(x, y, f"{tu} big={big} chain {i}")


def test_local_streamed_form_rows_longer_than_a_slot(P):
    """Rows of more than 10,234 entries (a ring slot less the alignment
    margin) go around the ring (read from global memory) and give the same
    sub-labels as the group form; so does a block range longer than the
    producer's 1,024-cell window."""
    rng = np.random.default_rng(77)
    N, D = 160_000, 12_000
    lens = rng.integers(1, 60, size=N)
    lens[[3, 250, 251, 252, 700, 159_999]] = [8700, 10234, 10235, 12_000, 11_000, 7200]
    indptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    # distinct columns per row: (7 row + 131 j) mod D, j < n (131 is prime to D), sorted
    row = np.repeat(np.arange(N), lens)
    j = np.arange(indptr[-1]) - np.repeat(indptr[:-1], lens)
    cols = (7 * row + 131 * j) % D
    order = np.lexsort((cols, row))
    indices = cols[order]
    data = rng.integers(1, 30, size=indptr[-1])

    def run(tu):
        s = P.Sampler(indptr, indices.astype(np.int32), data.astype(np.int32), N, D, 1.0, 0.5,
                      kmax=8, seed=4, engine=P.ENGINE_CSR_FP32, local_iters=2)
        if tu:
            P.dpmm_set_tuning(s.ctx, **tu)
        s.sweep(1)                        # K = 1: the table (96 KB) leaves room for two ring slots
        P.dpmm_local_gibbs(s.ctx, 1)
        out = (s.get_state(), s.stats())
        s.close()
        return out

    ref = run(None)
    assert ref[0][2] == 1
    for tu in FORMS:
        same_chain(run(tu), ref, str(tu))


def test_local_iteration_arguments(P, tiny):
    args = (tiny.indptr, tiny.indices, tiny.data, tiny.N, tiny.D, 1.0, 0.5)
    with pytest.raises(P.DpmmError):
        P.Sampler(*args, local_iters=17)
    plain = P.Sampler(*args)
    plain.sweep(1)
    with pytest.raises(P.DpmmError, match="local_iters > 1"):
        P.dpmm_local_gibbs(plain.ctx, 1)
    with pytest.raises(P.DpmmError):
        P.Sampler(*args, local_iters=2, hastings="instantiated")
    g = P.Sampler(*args, local_iters=2)
    with pytest.raises(P.DpmmError, match="t = 0"):
        P.dpmm_local_gibbs(g.ctx, 1)
    g.sweep(1)
    with pytest.raises(P.DpmmError):
        P.dpmm_local_gibbs(g.ctx, 0)
    with pytest.raises(P.DpmmError):
        P.dpmm_local_gibbs(g.ctx, 16)
    P.dpmm_local_gibbs(g.ctx, 3)
