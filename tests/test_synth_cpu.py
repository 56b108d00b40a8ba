"""The seeded synthetic inputs (the stand-ins for the paper's UMI datasets):
valid CSR, the documented shapes and densities, cluster sizes and library
sizes as the recipe states, and block-parallel generation independent of the
number of workers.  No GPU."""

import numpy as np
import pytest

from paper_1812_10048_gb300 import synth


def _check_csr(ds):
    ip, ix, dt = ds.indptr, ds.indices, ds.data
    assert ip.dtype == np.int32 and ix.dtype == np.int32 and dt.dtype == np.int32
    assert ip.shape == (ds.N + 1,) and ip[0] == 0 and ip[-1] == ix.size == dt.size
    assert np.all(np.diff(ip) >= 0)
    assert ix.min() >= 0 and ix.max() < ds.D
    assert dt.min() >= 1                      # only non-zero counts are stored
    # columns strictly increasing inside every row
    step = np.diff(ix.astype(np.int64))
    row_start = np.zeros(ix.size, dtype=bool)
    row_start[ip[:-1][np.diff(ip) > 0]] = True
    assert np.all(step[~row_start[1:]] > 0)


def _row_sums(ds):
    return np.add.reduceat(ds.data.astype(np.int64), ds.indptr[:-1]) * (np.diff(ds.indptr) > 0)


def test_cluster_sizes_sum_to_N_and_follow_the_weights():
    for N, K, s in ((2000, 5, None), (68000, 10, 1.2), (1001, 7, 1.0), (5, 7, None)):
        sizes = synth.cluster_sizes(N, K, s)
        assert sizes.sum() == N and sizes.shape == (K,)
        w = np.ones(K) if s is None else np.arange(1, K + 1, dtype=np.float64) ** (-s)
        assert np.all(np.abs(sizes - N * w / w.sum()) < 1.0)
    assert list(synth.cluster_sizes(2000, 5)) == [400] * 5
    z = synth.cluster_sizes(68000, 10, 1.2)
    assert np.all(np.diff(z) <= 0)            # Zipf: non-increasing in k


def test_tiny_workload_recipe():
    ds = synth.tiny()
    _check_csr(ds)
    assert (ds.N, ds.D) == (2000, 500)
    assert list(np.bincount(ds.labels)) == [400] * 5
    assert ds.data.size == 290976             # 29.1% density for this seed
    lib = _row_sums(ds)
    assert lib.min() >= 1
    # LogNormal(log 1500, 0.5) library sizes
    assert abs(np.mean(np.log(lib)) - np.log(1500.0)) < 0.05
    assert abs(np.std(np.log(lib)) - 0.5) < 0.05


def test_tiny_is_reproducible_and_seeded():
    a, b, c = synth.tiny(), synth.tiny(), synth.tiny(seed=7)
    assert np.array_equal(a.indptr, b.indptr) and np.array_equal(a.data, b.data)
    assert np.array_equal(a.indices, b.indices) and np.array_equal(a.labels, b.labels)
    assert not (a.data.size == c.data.size and np.array_equal(a.data, c.data))


def test_pbmc68k_workload_recipe():
    ds = synth.pbmc68k()
    _check_csr(ds)
    assert (ds.N, ds.D) == (68000, 1000)
    assert ds.data.size == 9777098            # the measured density, 14.4%
    assert round(ds.density, 4) == 0.1438
    assert np.array_equal(np.bincount(ds.labels, minlength=10), synth.cluster_sizes(68000, 10, 1.2))
    lib = _row_sums(ds)
    assert abs(np.mean(np.log(lib)) - np.log(1000.0)) < 0.02
    assert abs(np.std(np.log(lib)) - 0.6) < 0.02


def test_deep_cells_reach_the_stated_range():
    ds = synth.make_dataset(3000, 200, 3, gamma=0.05, lib_mu=np.log(1000.0), lib_sigma=0.6,
                            deep_frac=0.05, seed=11)
    _check_csr(ds)
    lib = _row_sums(ds)
    deep = lib >= 5000
    assert 0.02 < deep.mean() < 0.09
    assert lib.max() <= 60000


@pytest.mark.parametrize("workers", [1, 2])
def test_block_generation_does_not_depend_on_the_workers(workers):
    kw = dict(gamma=0.05, lib_mu=np.log(1000.0), lib_sigma=0.6, zipf=1.0, deep_frac=0.02,
              seed=1003, block=1000)
    ref = synth.make_dataset_blocks(3500, 300, 4, workers=1, **kw)
    ds = synth.make_dataset_blocks(3500, 300, 4, workers=workers, **kw)
    _check_csr(ds)
    for name in ("indptr", "indices", "data", "labels"):
        assert np.array_equal(getattr(ds, name), getattr(ref, name))
