"""bench.py's host-side helpers: the workloads and their targets, the CPU
baseline's tasks, field file and summary, the launch table and the DRAM
traffic file built from ncu --csv logs (no GPU)."""
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


def _args(*argv):
    old = sys.argv
    try:
        sys.argv = ["bench.py", *argv]
        return bench.parse()
    finally:
        sys.argv = old


def test_targets_per_workload():
    a = _args()
    assert a.workload == "c3" and a.fields == 6
    assert bench.targets(a, 6) == [40.0, 60.0, 80.0, 40.0, 60.0, 80.0]
    assert bench.field_shape(a) == (512, 512, 512)
    a = _args("--workload", "c1")
    assert a.fields == 24
    assert bench.targets(a, 7) == [40.0, 60.0, 80.0, 100.0, 120.0, 40.0, 60.0]
    a = _args("--workload", "c2")
    assert a.fields == 13 and bench.field_shape(a) == (100, 500, 500)
    assert bench.targets(a, 13)[:11] == [30.0 + 10 * k for k in range(10)] + [30.0]
    a = _args("--workload", "c0")
    assert a.fields == 1 and bench.targets(a, 1) == [80.0]
    assert "fit the 129 MB L2" in bench.workload_config(a, None)["l2"]
    a = _args("--workload", "c1", "--psnr", "90")
    assert bench.targets(a, 3) == [90.0, 90.0, 90.0]
    assert "target PSNR 90 dB for every field" in bench.workload_config(a, None)["workload"]
    for wl in bench.WORKLOADS:
        c = bench.workload_config(_args("--workload", wl), 3)
        assert c["name"] == wl and c["workload"].startswith(wl + ":")
    with pytest.raises(SystemExit):
        _args("--workload", "c3", "--fields", "7")


def test_cpu_tasks():
    """c3 is cut into 64-plane z-slabs covering every plane of every field;
    the other workloads take whole fields."""
    a = _args()
    t = bench.cpu_tasks(a, (512, 512, 512))
    assert len(t) == 48 and len(set(t)) == 48
    for f in range(6):
        planes = sorted((z0, z1) for g, z0, z1 in t if g == f)
        assert planes[0][0] == 0 and planes[-1][1] == 512
        assert all(p[1] == q[0] for p, q in zip(planes, planes[1:]))
    a = _args("--workload", "c2")
    assert bench.cpu_tasks(a, (100, 500, 500)) == [(f, 0, 100) for f in range(13)]


def test_host_fields_and_oracle_task():
    """The shared field file holds every field at its offset; a task runs the
    oracle on its planes and reports the oracle's own PSNR."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(0)
    xs = [rng.standard_normal((6, 5, 7)).astype(np.float32), rng.standard_normal((3, 9)).astype(np.float32)]
    hf = bench.HostFields(xs)
    try:
        args = hf.args((0, 2, 5), [60.0, 80.0], 256)
        v = np.memmap(args[0], dtype=np.float32, mode="r", offset=args[1], shape=args[2])
        assert np.array_equal(v, xs[0])
        assert hf.task_bytes((0, 2, 5)) == 4 * 3 * 5 * 7
        dt, nb, p = bench.oracle_task(args)
        blob, st = oracle.compress(xs[0][2:5], 60.0)
        assert nb == len(blob) and p == st["psnr_actual"] and dt > 0
        args = hf.args((1, 0, 3), [60.0, 80.0], 256)
        v = np.memmap(args[0], dtype=np.float32, mode="r", offset=args[1], shape=args[2])
        assert np.array_equal(v, xs[1])
    finally:
        hf.close()
    assert not os.path.exists(args[0])


def test_stage_bytes():
    assert bench.stage_bytes("predict_quantize", 10, 3) == 60
    assert bench.stage_bytes("scan_final_dequant", 10, 3, 2) == 60
    assert bench.stage_bytes("scan_final_dequant", 10, 3, 3) == 60
    assert bench.stage_bytes("band_sum", 10, 3, 3) == 20
    assert bench.stage_bytes("scan_y", 10, 3, 3) == 80 and bench.stage_bytes("scan_y", 10, 3, 2) is None
    assert bench.stage_bytes("decode", 10, 3, 3) == 23


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
    """Bytes per point per workload and stage from separate one-kernel
    captures; reported for a launch of any size while the sources match."""
    rows = []
    for lid in (1, 2):  # two launches of the predictor
        k = "void fp::k_pq<3, 128, 8, 1, 1>(fp::Batch<fp::PQArgs>)"
        rows += [_row(lid, k, "dram__bytes_read.sum", "Mbyte", "200"),
                 _row(lid, k, "dram__bytes_write.sum", "byte", "1000000")]
    out = tmp_path / "profiles"
    out.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src = tmp_path / "paper_1805_07384_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "compress.cu").write_text("kernel source\n")
    (src / "common.cuh").write_text("shared header\n")
    (src.parent / "build.py").write_text("flags\n")
    bench.write_traffic(_log(tmp_path, rows), "c3", 10**8, "ncu ... k_pq")
    # the encoder's kernels captured one at a time add up
    enc = [_row(3, "void fp::k_enc_pack(fp::Batch<fp::EncArgs>)", "dram__bytes_read.sum", "byte", "100"),
           _row(3, "void fp::k_enc_pack(fp::Batch<fp::EncArgs>)", "dram__bytes_write.sum", "byte", "10")]
    bench.write_traffic(_log(tmp_path, enc), "c3", 10, "ncu ... k_enc_pack")
    cp = [_row(4, "void fp::k_enc_copy(fp::Batch<fp::EncArgs>)", "dram__bytes_read.sum", "byte", "30"),
          _row(4, "void fp::k_enc_copy(fp::Batch<fp::EncArgs>)", "dram__bytes_write.sum", "byte", "20")]
    bench.write_traffic(_log(tmp_path, cp), "c3", 10, "ncu ... k_enc_copy")
    t = json.load(open(out / "traffic.json"))
    pq = t["c3"]["predict_quantize"]
    assert pq["dram_bytes_per_point"] == pytest.approx(2.01)
    assert pq["kernels"]["k_pq<3, 128, 8, 1, 1>"]["launches"] == 2
    assert t["c3"]["encode"]["dram_bytes_per_point"] == pytest.approx(16.0)
    assert sorted(t["c3"]["encode"]["kernels"]) == ["k_enc_copy", "k_enc_pack"]
    import hashlib
    assert pq["sources"]["paper_1805_07384_gb300/csrc/compress.cu"] == hashlib.sha1(b"kernel source\n").hexdigest()
    assert "decode" not in t["c3"] and "c1" not in t
    # scaled to the launch of the benchmark's own size
    assert bench.measured_traffic("c3", "predict_quantize", 10**9) == 2_010_000_000
    assert bench.measured_traffic("c1", "predict_quantize", 10**9) is None
    # reported only while the source, the shared header and the flags are unchanged
    (src.parent / "build.py").write_text("other flags\n")
    assert bench.measured_traffic("c3", "predict_quantize", 10**9) is None
    (src.parent / "build.py").write_text("flags\n")
    (src / "common.cuh").write_text("changed header\n")
    assert bench.measured_traffic("c3", "predict_quantize", 10**9) is None
    (src / "common.cuh").write_text("shared header\n")
    assert bench.measured_traffic("c3", "predict_quantize", 10**9) == 2_010_000_000
    (src / "compress.cu").write_text("changed\n")
    assert bench.measured_traffic("c3", "predict_quantize", 10**9) is None


def test_cpu_baseline_summary():
    """Median over the steps of each round's GB/s, plus each task's one-core
    GB/s from its worker's own time."""
    a = _args("--workload", "c1")
    runs = [(2.0, 2 * 10**9, [((0, 0, 1), 10**9, (2.0, 10, 80.0)), ((1, 0, 1), 10**9, (1.0, 10, 60.0))]),
            (1.0, 2 * 10**9, [((2, 0, 1), 10**9, (4.0, 10, 40.0)), ((3, 0, 1), 10**9, (0.5, 10, 40.0))]),
            (4.0, 2 * 10**9, [((0, 0, 1), 10**9, (1.0, 10, 80.0)), ((1, 0, 1), 10**9, (1.0, 10, 60.0))])]
    c = bench.cpu_baseline_summary(a, runs, 2, 24)
    assert c["value"] == 1.0 and c["cores"] == 2 and c["kind"] == "oracle"
    assert c["steps_gbs"] == [1.0, 2.0, 0.5]
    assert c["one_core_gbs_per_task"] == {"median": 1.0, "min": 0.25, "max": 2.0}
    assert "3 steps" in c["sample"] and "24 fields" in c["sample"]


def test_serve_requests():
    """The served stream: Poisson arrivals at the stated rate, every shape and
    both kinds, targets in [30, 120] dB, request ids unique per seed."""
    reqs = bench.serve_requests(4000, 5000.0, seed=5)
    assert len(reqs) == 4000 and len({r[4] for r in reqs}) == 4000
    t = [r[0] for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    rate = len(t) / (t[-1] / 1e6)
    assert 4500 < rate < 5500
    assert {r[1] for r in reqs} == set(bench.SERVE_SHAPES)
    assert {r[3] for r in reqs} == {0, 1}
    assert all(30.0 <= r[2] <= 120.0 for r in reqs)
    assert bench.serve_requests(4000, 5000.0, seed=5) == reqs
    assert bench.ServeSetup.bucket(44.9) == 40.0 and bench.ServeSetup.bucket(115.1) == 120.0
