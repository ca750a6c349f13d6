"""bench.py's host-side helpers: the per-field targets (--psnr), the launch
table and the DRAM traffic file built from ncu --csv logs (no GPU)."""
import json
import os
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402

HEADER = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
          '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
          '"Metric Value"')


def _row(lid, kernel, metric, unit, value):
    return (f'"{lid}","1","python3","127.0.0.1","{kernel}","1","13","(128, 1, 1)","(10, 1, 1)",'
            f'"0","10.3","Command line profiler metrics","{metric}","{unit}","{value}"')


def _log(tmp_path, rows):
    p = tmp_path / "log.csv"
    p.write_text("==PROF== Connected to process 1\n" + HEADER + "\n" + "\n".join(rows) + "\n")
    return str(p)


def test_targets():
    old = sys.argv
    try:
        sys.argv = ["bench.py"]
        assert bench.targets(bench.parse(), 7) == [40.0, 60.0, 80.0, 100.0, 120.0, 40.0, 60.0]
        sys.argv = ["bench.py", "--psnr", "90"]
        a = bench.parse()
        assert bench.targets(a, 3) == [90.0, 90.0, 90.0]
        assert "target PSNR 90 dB for every field" in bench.workload_config(a, None)["workload"]
    finally:
        sys.argv = old


def test_launch_table(tmp_path):
    rows = [_row(1, "void fp::k_pq<2, 1024, 1, 1, 2>(fp::Batch<fp::PQArgs>)", "gpu__time_duration.sum", "us", "30"),
            _row(2, "void fp::k_decode<128>(fp::Batch<fp::DecArgs>)", "gpu__time_duration.sum", "ns", "10000"),
            _row(3, "void fp::k_pq<2, 1024, 1, 1, 2>(fp::Batch<fp::PQArgs>)", "gpu__time_duration.sum", "us", "30"),
            _row(4, "void at::vectorized_elementwise_kernel<2>(int)", "gpu__time_duration.sum", "us", "999")]
    tab = bench.launch_table(_log(tmp_path, rows)).splitlines()
    assert tab[2] == "| `k_pq<2, 1024, 1, 1, 2>` | 2 | 60.0 | 85.7% |"
    assert tab[3] == "| `k_decode<128>` | 1 | 10.0 | 14.3% |"
    assert len(tab) == 4  # torch's kernel is left out


def test_write_traffic(tmp_path, monkeypatch):
    rows = []
    for lid in (1, 2):  # two launches of the predictor
        k = "void fp::k_pq<2, 1024, 1, 1, 2>(fp::Batch<fp::PQArgs>)"
        rows += [_row(lid, k, "dram__bytes_read.sum", "Mbyte", "200"),
                 _row(lid, k, "dram__bytes_write.sum", "byte", "1000000"),
                 _row(lid, k, "gpu__time_duration.sum", "us", "150")]
    for lid, k in ((3, "void fp::k_enc_pack(fp::Batch<fp::EncArgs>)"),
                   (4, "void fp::k_enc_scan(fp::Batch<fp::EncArgs>)"),
                   (5, "void fp::k_enc_copy(fp::Batch<fp::EncArgs>)")):
        rows += [_row(lid, k, "dram__bytes_read.sum", "byte", "100"),
                 _row(lid, k, "dram__bytes_write.sum", "byte", "10")]
    out = tmp_path / "profiles"
    out.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src = tmp_path / "paper_1805_07384_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "compress.cu").write_text("kernel source\n")
    (src / "common.cuh").write_text("shared header\n")
    (src.parent / "build.py").write_text("flags\n")
    bench.write_traffic(_log(tmp_path, rows))
    t = json.load(open(out / "traffic.json"))
    pq = t["predict_quantize"]
    assert pq["launches"] == 2 and pq["dram_read"] == 200_000_000 and pq["dram_write"] == 1_000_000
    assert pq["dram_bytes_per_launch"] == 201_000_000
    enc = t["encode"]
    assert enc["launches"] == 1 and enc["dram_bytes_per_launch"] == 330
    assert sorted(enc["kernels"]) == ["k_enc_copy", "k_enc_pack", "k_enc_scan"]
    import hashlib
    assert pq["source_sha1"] == hashlib.sha1(b"kernel source\n").hexdigest()
    assert "decode" not in t
    # the SHA-1 check: traffic is reported only while the source is unchanged
    assert bench.measured_traffic("predict_quantize") == 201_000_000
    # ... and while the shared header and the compiler flags are unchanged
    (src.parent / "build.py").write_text("other flags\n")
    assert bench.measured_traffic("predict_quantize") is None
    (src.parent / "build.py").write_text("flags\n")
    (src / "common.cuh").write_text("changed header\n")
    assert bench.measured_traffic("predict_quantize") is None
    (src / "common.cuh").write_text("shared header\n")
    assert bench.measured_traffic("predict_quantize") == 201_000_000
    (src / "compress.cu").write_text("changed\n")
    assert bench.measured_traffic("predict_quantize") is None


def test_cpu_baseline_summary():
    """Whole-batch GB/s over the pool's wall time, plus each field's one-core
    GB/s from its worker's own time."""
    res = [(2.0, 10, 80.0), (1.0, 10, 60.0), (4.0, 10, 40.0)]
    c = bench.cpu_baseline_summary(3_000_000_000, 5.0, 3, [1e9, 1e9, 1e9], res)
    assert c["value"] == 0.6 and c["cores"] == 3 and c["kind"] == "oracle"
    assert c["one_core_gbs_per_field"] == {"median": 0.5, "min": 0.25, "max": 1.0}
    assert "3 fields" in c["sample"]
