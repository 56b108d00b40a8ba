"""Launch tuning (dpmm_set_tuning) and the autotuner.

No launch setting may change a result: a chain stepped under any tuning must
end bit-identical to the same chain under the defaults (labels, sub-labels,
K, counters, integer statistics, sums of log q).  The autotuner must leave
the chain's state as it found it and reuse its cached choice.
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


@pytest.fixture(scope="module")
def dense():
    """4,000 x 512 at ~2,000 counts per cell, 6 clusters: dense enough for the
    tile engine at every K >= 1 under the automatic rule's K >= 3."""
    from paper_1812_10048_gb300 import synth
    return synth.make_dataset(4000, 512, 6, gamma=0.1, lib_mu=np.log(2000.0), lib_sigma=0.4,
                              seed=4101)


def batch_data():
    from paper_1812_10048_gb300 import synth
    out = []
    for b, (N, K) in enumerate([(1500, 3), (2600, 6), (900, 4)]):
        ds = synth.make_dataset(N, 320, K, gamma=0.1, lib_mu=np.log(1200.0), lib_sigma=0.5,
                                seed=4200 + b)
        out.append((ds.indptr, ds.indices, ds.data, ds.N))
    return out


def snapshot(s):
    lab, sub, K, t, m = s.get_state()
    n, S, q = s.stats()
    return lab, sub, K, t, m, n, S, q


def assert_same(a, b, what=""):
    assert a[2:5] == b[2:5], what
    for x, y in zip(a[:2] + a[5:], b[:2] + b[5:]):
        np.testing.assert_array_equal(x, y, err_msg=what)


TUNINGS = (
    [{"stats_blocks_per_sm": v} for v in (1, 2, 8)]
    + [{"tile_stages": 2}, {"tile_stages": 4}]
    + [{"tile_scatter": v} for v in (8, 16)]
    + [{"draw_blocks_per_sm": 1}]
    + [{"stats_blocks_per_sm": 1, "tile_stages": 2, "tile_scatter": 16, "draw_blocks_per_sm": 1}]
)


def run_single(P, ds, tuning, steps=8):
    s = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, kmax=32, seed=77)
    if tuning:
        P.dpmm_set_tuning(s.ctx, **tuning)
    s.step(steps)
    snap = snapshot(s)
    tile = P.dpmm_debug_engine(s.ctx)
    s.close()
    return snap, tile


def lanes_for(nnz, N):
    """Default lanes per cell of the local sub-label kernel for a mean row."""
    mean = nnz // N
    return 4 if mean < 64 else 8 if mean < 128 else 16 if mean < 256 else 32


def test_defaults_reported(P, dense):
    s = P.Sampler(dense.indptr, dense.indices, dense.data, dense.N, dense.D, 1.0, 0.5, kmax=32)
    lanes = lanes_for(int(dense.indptr[-1]), dense.N)
    assert P.dpmm_get_tuning(s.ctx) == {"stats_blocks_per_sm": 4, "tile_stages": 4,
                                        "tile_scatter": 12, "draw_blocks_per_sm": 2,
                                        "local_lanes": lanes, "local_stream": 0}
    P.dpmm_set_tuning(s.ctx, tile_stages=2, tile_scatter=16, local_lanes=32)
    assert P.dpmm_get_tuning(s.ctx) == {"stats_blocks_per_sm": 4, "tile_stages": 2,
                                        "tile_scatter": 16, "draw_blocks_per_sm": 2,
                                        "local_lanes": 32, "local_stream": 0}
    P.dpmm_set_tuning(s.ctx)                     # all zero: back to the defaults
    assert P.dpmm_get_tuning(s.ctx)["tile_stages"] == 4
    assert P.dpmm_get_tuning(s.ctx)["local_lanes"] == lanes
    s.close()
    data = batch_data()
    b = P.BatchSampler(data, 320, kmax=16)
    blanes = lanes_for(sum(int(d[0][-1]) for d in data), sum(d[3] for d in data))
    assert P.dpmm_get_tuning(b.ctx) == {"stats_blocks_per_sm": 2, "tile_stages": 2,
                                        "tile_scatter": 12, "draw_blocks_per_sm": 2,
                                        "local_lanes": blanes, "local_stream": 0}
    b.close()


@pytest.mark.parametrize("bad", [{"stats_blocks_per_sm": 3}, {"tile_stages": 3},
                                 {"tile_scatter": 10}, {"draw_blocks_per_sm": 4},
                                 {"tile_stages": -1}, {"local_lanes": 2}, {"local_lanes": 64},
                                 {"local_stream": 2}])
def test_invalid_tuning_rejected(P, dense, bad):
    s = P.Sampler(dense.indptr, dense.indices, dense.data, dense.N, dense.D, 1.0, 0.5, kmax=32)
    before = P.dpmm_get_tuning(s.ctx)
    with pytest.raises(P.DpmmError):
        P.dpmm_set_tuning(s.ctx, **bad)
    assert P.dpmm_get_tuning(s.ctx) == before
    with pytest.raises(ValueError):
        P.dpmm_set_tuning(s.ctx, no_such_field=1)
    s.close()


def test_every_tuning_gives_identical_chains(P, dense):
    ref, tile = run_single(P, dense, None)
    assert tile == 1 and ref[2] >= 3
    for tu in TUNINGS:
        got, tile = run_single(P, dense, tu)
        assert tile == 1
        assert_same(got, ref, str(tu))


def test_every_tuning_gives_identical_batches(P):
    data = batch_data()

    def run(tu):
        b = P.BatchSampler(data, 320, kmax=16, seed=31, chain_id=2)
        if tu:
            P.dpmm_set_tuning(b.ctx, **tu)
        b.step(6)
        snaps = [snapshot(b.chain(i)) for i in range(b.B)]
        b.close()
        return snaps

    ref = run(None)
    for tu in TUNINGS:
        for i, (g, r) in enumerate(zip(run(tu), ref)):
            assert_same(g, r, f"{tu} chain {i}")


def test_retuning_between_steps(P, dense):
    """A tuning change between steps (the step graph is rebuilt) continues the
    chain exactly."""
    ref, _ = run_single(P, dense, None, steps=9)
    s = P.Sampler(dense.indptr, dense.indices, dense.data, dense.N, dense.D, 1.0, 0.5, kmax=32,
                  seed=77)
    s.step(3)
    P.dpmm_set_tuning(s.ctx, tile_scatter=8, stats_blocks_per_sm=8)
    s.step(3)
    P.dpmm_set_tuning(s.ctx, tile_stages=2, draw_blocks_per_sm=1)
    s.step(3)
    assert_same(snapshot(s), ref)
    s.close()


def test_autotune_keeps_state_and_uses_cache(P, dense, tmp_path):
    from paper_1812_10048_gb300 import autotune as A
    path = str(tmp_path / "tuning.json")
    s = P.Sampler(dense.indptr, dense.indices, dense.data, dense.N, dense.D, 1.0, 0.5, kmax=32,
                  seed=77)
    s.step(5)
    before = snapshot(s)
    rec = A.autotune(s, [dense.indptr], trial_steps=3, repeats=1, path=path)
    assert rec["source"] == "measured" and rec["measurements"] >= 8
    assert set(rec["tuning"]) == set(P.TUNING_FIELDS)
    assert P.dpmm_get_tuning(s.ctx) == rec["tuning"]
    assert_same(snapshot(s), before, "state after autotune")
    s.step(4)                                     # continues as an untuned chain would
    ref, _ = run_single(P, dense, None, steps=9)
    assert_same(snapshot(s), ref, "continuation after autotune")
    rec2 = A.autotune(s, [dense.indptr], trial_steps=3, repeats=1, path=path)
    assert rec2["source"] == "cache" and rec2["tuning"] == rec["tuning"]
    assert rec2["key"] == rec["key"]
    s.close()


def test_autotune_batch_keeps_state(P, tmp_path):
    from paper_1812_10048_gb300 import autotune as A
    data = batch_data()
    b = P.BatchSampler(data, 320, kmax=16, seed=31, chain_id=2)
    b.step(3)
    before = [snapshot(b.chain(i)) for i in range(b.B)]
    rec = A.autotune(b, [d[0] for d in data], trial_steps=2, repeats=1,
                     path=str(tmp_path / "t.json"))
    assert rec["source"] == "measured" and rec["key"].endswith("chains<=4")
    for i in range(b.B):
        assert_same(snapshot(b.chain(i)), before[i], f"chain {i}")
    b.step(3)
    r = P.BatchSampler(data, 320, kmax=16, seed=31, chain_id=2)
    r.step(6)
    for i in range(b.B):
        assert_same(snapshot(b.chain(i)), snapshot(r.chain(i)), f"chain {i}")
    b.close()
    r.close()
