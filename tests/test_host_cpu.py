"""Host-side helpers of the studies: the close-cell-type generator and the
cluster matching used for per-cell stability."""

import numpy as np


def test_similar_types_depth_changes_only_the_library_sizes():
    from paper_1812_10048_gb300 import synth
    a = synth.similar_types(600, 200, 3, 300)
    b = synth.similar_types(600, 200, 3, 30000)
    np.testing.assert_array_equal(a.labels, b.labels)       # same cells, same types
    for ds, depth in ((a, 300), (b, 30000)):
        lib = np.add.reduceat(ds.data.astype(np.int64), ds.indptr[:-1].astype(np.int64))
        assert abs(np.median(lib) / depth - 1) < 0.1
        assert ds.indices.max() < ds.D and ds.data.min() >= 1
    # the types differ only slightly: per-type gene frequencies at depth 30000
    # agree to within a few percent of the profile scale
    freq = np.zeros((3, b.D))
    rows = np.repeat(np.arange(b.N), np.diff(b.indptr))
    np.add.at(freq, (b.labels[rows], b.indices), b.data)
    freq /= freq.sum(axis=1, keepdims=True)
    top = np.argsort(-freq.mean(axis=0))[:20]
    ratio = freq[:, top] / freq[:, top].mean(axis=0)
    assert np.all(np.abs(np.log(ratio)) < 0.3) and np.any(np.abs(np.log(ratio)) > 0.01)


def test_matched_labels_map_found_clusters_to_generating_ones():
    import bench
    truth = np.array([0, 0, 1, 1, 2, 2, 2])
    found = np.array([5, 5, 0, 0, 3, 3, 3])          # a relabelling
    np.testing.assert_array_equal(bench._matched_labels(found, truth), truth)
    split = np.array([0, 1, 2, 2, 3, 3, 4])          # an over-split partition
    np.testing.assert_array_equal(bench._matched_labels(split, truth), truth)
