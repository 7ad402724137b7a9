"""Host-side logic of bench.py that needs no GPU: the algorithmic byte counts
behind the roofline fractions, the ingestion of an ncu DRAM capture into the
machine-read traffic record, and the clock-sample summary that decides
whether a run is kept."""
import csv
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_seg_alg_bytes_by_tier():
    # below 2^13 keys: one read and one write of each pair (16 B); from 2^13
    # on: a 4-byte counting read plus 16 B per digit group
    sizes = np.array([1, 63, 4096, 8191, 8192, 20_000], np.int64)
    small = 1 + 63 + 4096 + 8191
    large = 8192 + 20_000
    assert bench.seg_alg_bytes(sizes) == 16 * small + (4 + 4 * 16) * large
    assert bench.seg_alg_bytes(sizes, passes=2) == 16 * small + (4 + 2 * 16) * large
    assert bench.seg_alg_bytes(np.array([], np.int64)) == 0


def _ncu_csv(path, launches):
    """An ncu --csv capture in the layout ncu writes: one row per (launch,
    metric), more than ten columns."""
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream",
           "Block Size", "Grid Size", "Device", "CC", "Section Name", "Metric Name",
           "Metric Unit", "Metric Value"]
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(hdr)
        for i, (rd_mb, wr_mb, us) in enumerate(launches):
            name = "void rs::pass_kernel<rs::CodecU32, unsigned int, 40, 256>(rs::PassArgs)"
            base = [str(i), "1", "python", "h", name, "1", "7", "(256, 1, 1)", "(6554, 1, 1)",
                    "0", "10.3", "Command line profiler metrics"]
            w.writerow(base + ["dram__bytes_read.sum", "Mbyte", f"{rd_mb:,.2f}"])
            w.writerow(base + ["dram__bytes_write.sum", "Mbyte", f"{wr_mb:,.2f}"])
            w.writerow(base + ["gpu__time_duration.sum", "us", f"{us:.2f}"])
        # another kernel in the same capture is ignored
        w.writerow(["99", "1", "python", "h", "void rs::count_kernel<rs::CodecU32>(rs::CountArgs)",
                    "1", "7", "(256, 1, 1)", "(152, 1, 1)", "0", "10.3", "x",
                    "dram__bytes_read.sum", "Mbyte", "999.00"])


def test_ingest_dram_csv_and_profile_traffic(tmp_path, monkeypatch):
    record = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(record))
    n = 1 << 20
    src = tmp_path / "dram.csv"
    _ncu_csv(src, [(8.5, 7.5, 10.0), (8.3, 7.7, 12.0)])
    d = bench.ingest_dram_csv(str(src), n)
    assert d["launches"] == 2 and d["n_captured"] == n
    assert d["dram_bytes_read_per_launch"] == pytest.approx(8.4e6)
    assert d["dram_bytes_write_per_launch"] == pytest.approx(7.6e6)
    assert d["alg_bytes_per_launch"] == 16 * n
    assert d["traffic_over_alg"] == pytest.approx(16.0e6 / (16 * n))
    assert d["ncu_ms_per_launch"] == pytest.approx(0.011)
    assert d["kernel_source_sha256"] == bench.kernel_source_hash()
    assert json.loads(record.read_text()) == d

    # reported scaled by the units processed, and only for the same source
    t = bench.profile_traffic(bench.kernel_source_hash(), 4 * n)
    assert t["bytes_per_launch"] == pytest.approx(4 * 16.0e6)
    assert t["read_over_alg"] == pytest.approx(8.4e6 / (8 * n))
    assert bench.profile_traffic("0" * 16, n) is None
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(tmp_path / "absent.json"))
    assert bench.profile_traffic(bench.kernel_source_hash(), n) is None


def test_ingest_rejects_a_capture_without_the_kernel(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(tmp_path / "traffic.json"))
    src = tmp_path / "dram.csv"
    _ncu_csv(src, [])
    with pytest.raises(SystemExit):
        bench.ingest_dram_csv(str(src), 1 << 20)
    assert not (tmp_path / "traffic.json").exists()


def _clock_summary(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    s.proc = object()  # a sampler that ran
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return s.summary()


def test_clock_summary_median_under_load_and_reasons(tmp_path):
    na, act = "Not Active", "Active"
    rows = [f"2070, 2070, 900.5, 0x0, {na}, {na}, {na}, {na}"] * 5
    rows += [f"345, 2070, 90.0, 0x0, {na}, {na}, {na}, {na}"] * 3     # idle samples
    rows += [f"1980, 2070, 1400.0, 0x4, {na}, {na}, {na}, {act}"] * 2  # power cap
    got = _clock_summary(tmp_path, rows)
    assert got["sm_max_mhz"] == 2070
    assert got["sm_mhz"] == 2070          # idle samples below half the max are left out
    assert got["reasons"] == ["sw_power_cap"]
    assert got["samples"] == 10


def test_clock_summary_flags_thermal_and_missing_samples(tmp_path):
    na, act = "Not Active", "Active"
    got = _clock_summary(tmp_path, [f"1500, 2070, 1300.0, 0x40, {na}, {act}, {na}, {na}"])
    assert got["reasons"] == ["hw_thermal_slowdown"]
    assert _clock_summary(tmp_path, ["garbage"])["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]
