"""Host logic of bench.py, without a GPU: the algorithmic bytes behind the
roofline line, the DRAM-traffic record's source check, the measured-peak
lookup and the clock summary taken from nvidia-smi samples."""

import hashlib
import json
import types

import bench


def _pbmc68k_sizes():
    return types.SimpleNamespace(N=68000, D=1000, nnz=9777098)


def test_label_kernel_bytes_per_launch():
    # indptr 4 (N + 1), packed entries 4 nnz, cell state read and written
    # 8 N, the 3K log theta rows 4 * 3 K D and log pi 4 (K + 1)
    ds = _pbmc68k_sizes()
    assert bench.assign_algorithmic_bytes(ds, 10) == 272004 + 39108392 + 544000 + 120000 + 44
    assert bench.assign_algorithmic_bytes(ds, 10) == 40044440
    # unpacked int32 column + count pairs: four more bytes per entry
    extra = bench.assign_algorithmic_bytes(ds, 10, packed=False) - bench.assign_algorithmic_bytes(ds, 10)
    assert extra == 4 * ds.nnz


def test_step_bytes_add_the_statistics_pass_and_the_draws():
    ds = _pbmc68k_sizes()
    K, D = 10, ds.D
    stats = 4 * (ds.N + 1) + 4 * ds.nnz + 4 * ds.N + 8 * K * D
    draws = 8 * K * D + 12 * K * D
    assert bench.step_algorithmic_bytes(ds, K) == bench.assign_algorithmic_bytes(ds, K) + stats + draws
    assert bench.step_algorithmic_bytes(ds, K) == 79976836


def _traffic_fixture(tmp_path, monkeypatch, source_bytes):
    csrc = tmp_path / "paper_1812_10048_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = csrc / "tile.cu"
    src.write_bytes(source_bytes)
    rec = {"k_assign_tc": {"bytes_per_launch": 43069781, "source": "tile.cu",
                           "source_sha256": hashlib.sha256(b"kernel as captured").hexdigest(),
                           "workload": "pbmc68k"}}
    path = tmp_path / "ncu_traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(path))
    return src


def test_traffic_is_reported_only_for_the_captured_source_and_workload(tmp_path, monkeypatch):
    src = _traffic_fixture(tmp_path, monkeypatch, b"kernel as captured")
    assert bench.traffic_for("k_assign_tc", "pbmc68k") == 43069781
    assert bench.traffic_for("k_assign_tc", "large") is None       # another workload
    assert bench.traffic_for("k_assign", "pbmc68k") is None        # no record
    src.write_bytes(b"kernel changed since")
    assert bench.traffic_for("k_assign_tc", "pbmc68k") is None     # counters are stale


def test_traffic_without_a_record_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(tmp_path / "absent.json"))
    assert bench.traffic_for("k_assign_tc", "pbmc68k") is None


def test_hbm_peak_prefers_the_measured_file(tmp_path, monkeypatch):
    p = tmp_path / "peaks.json"
    p.write_text(json.dumps({"hbm_gbs": 6688.8, "bf16_tflops": 1900.0}))
    monkeypatch.setattr(bench, "PEAKS_PATH", str(p))
    assert bench.hbm_peak() == (6688.8, "measured")
    monkeypatch.setattr(bench, "PEAKS_PATH", str(tmp_path / "absent.json"))
    assert bench.hbm_peak() == (bench.FALLBACK_HBM_GBS, "fallback")


class _FinishedSampler:
    """Stands in for the nvidia-smi process once its samples are read."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _summary(lines, monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    cs = bench.ClockSampler(0)
    cs.proc = _FinishedSampler()
    cs.lines = list(lines)
    return cs.stop()


def test_clock_summary_median_max_and_power_cap(monkeypatch):
    out = _summary([
        "0, 2070, 2070, 250.10, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 900.50, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1200.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 10.00, 0x0, Not Active, Not Active, Not Active, Not Active",   # unreadable
        "0, 2070",                                                                      # cut off
    ], monkeypatch)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["power_w_max"] == 1200.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_names_every_slowdown_seen(monkeypatch):
    out = _summary([
        "0, 1400, 2070, 1300.00, 0x8, Active, Not Active, Not Active, Not Active",
        "0, 1500, 2070, 1300.00, 0x20, Not Active, Active, Not Active, Active",
        "0, 1600, 2070, 1300.00, 0x40, Not Active, Not Active, Active, Not Active",
    ], monkeypatch)
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap",
                              "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1500.0


def test_clock_summary_without_nvidia_smi():
    cs = bench.ClockSampler(0)
    out = cs.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_job_rate_is_all_ranks_steps_over_the_slowest_time():
    assert bench.job_rate(1, 2000, 200.0) == 10000.0
    assert bench.job_rate(4, 100, 50.0) == 8000.0
