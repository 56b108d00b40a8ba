"""Host logic of the launch autotuner: workload keys, the coordinate descent,
the on-disk cache (no GPU needed)."""

import json

import pytest

from paper_1812_10048_gb300 import autotune as A


def test_workload_key_buckets():
    k = A.workload_key("GB300", 1000, 10, 0.1438, 68000, 1)
    assert k == "GB300|D=1000|K<=10|density~0.15|cells<=131072|chains<=1"
    assert A.workload_key("GB300", 1000, 7, 0.14, 70000, 1) == k
    assert A.workload_key("GB300", 1000, 11, 0.14, 68000, 1) != k
    assert A.workload_key("GB300", 1000, 10, 0.14, 68000, 64).endswith("chains<=64")
    assert "|" not in A.workload_key("GB300", 1000, 10, 0.14, 68000, 1).split("|")[0]


def test_coordinate_descent_finds_the_separable_optimum():
    # cost separable in the settings: the optimum is each setting's best value
    best_of = {"stats_blocks_per_sm": 8, "tile_stages": 2, "tile_scatter": 16,
               "draw_blocks_per_sm": 1}
    calls = []

    def measure(s):
        calls.append(dict(s))
        return 1.0 + sum(0.1 * (s[k] != v) for k, v in best_of.items())

    best, t, n = A.coordinate_descent(measure, start={"stats_blocks_per_sm": 4,
                                                      "tile_stages": 4, "tile_scatter": 12,
                                                      "draw_blocks_per_sm": 2})
    assert best == best_of and t == pytest.approx(1.0)
    assert n == len(calls) == 1 + 3 + 1 + 2 + 1       # one baseline, then each alternative


def test_coordinate_descent_keeps_the_incumbent_within_the_margin():
    def measure(s):
        return 1.0 - 0.01 * (s["tile_scatter"] == 16)      # 1% better: below the 2% margin
    best, _, _ = A.coordinate_descent(measure, start={"tile_scatter": 12})
    assert best["tile_scatter"] == 12


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tuning.json")
    assert A.load_cache(p) == {}
    A.store_cache("k1", {"tuning": {"tile_scatter": 8}, "ms_per_step": 0.1}, p)
    A.store_cache("k2", {"tuning": {"tile_scatter": 16}, "ms_per_step": 0.2}, p)
    c = A.load_cache(p)
    assert c["k1"]["tuning"]["tile_scatter"] == 8 and c["k2"]["ms_per_step"] == 0.2
    with open(p) as f:
        assert set(json.load(f)) == {"k1", "k2"}


def test_cache_path_from_environment(monkeypatch, tmp_path):
    monkeypatch.setenv(A.CACHE_ENV, str(tmp_path / "x.json"))
    assert A.cache_path() == str(tmp_path / "x.json")
    assert A.cache_path("/explicit.json") == "/explicit.json"
