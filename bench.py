#!/usr/bin/env python
"""Throughput of fixed-PSNR compression + decompression on GB300.

One step compresses every field of a batch at its target PSNR and decompresses
it again; metric = original bytes / (compress + decompress time).  Workloads
(--workload, seeded synthetic stand-ins shaped like the paper's data sets,
Table 1):

  c3 (default)  6 NYX-like 3D fields of 512^3 points (3.2 GB): two lognormal
                densities, three velocity components, one temperature; field i
                at {40, 60, 80}[i mod 3] dB; 3D Lorenzo
  c2            13 hurricane-like 3D fields of 100 x 500 x 500 points (1.3 GB);
                field i at 30 + 10 (i mod 10) dB; 3D Lorenzo
  c1            24 climate-like 2D fields of 1800 x 3600 points (622 MB); field
                i at {40, 60, 80, 100, 120}[i mod 5] dB; 2D Lorenzo
  c0            one 512 x 512 2D field at 80 dB (1 MiB: fits L2, which is
                flushed between timed steps)

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on the
host cores instead (the reference arm of this method: the paper ships no GPU
code).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compress+decompress GB/s at target PSNR"
STAGE_BYTES_NOTE = "algorithmic bytes per launch, N = points of one field"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--sub-batches", type=int, default=3,
                    help="batch mode: sub-batches, one per stream")
    ap.add_argument("--e2e-sub-batches", type=int, default=24,
                    help="batch mode, end-to-end run: finer sub-batches so each field's "
                         "copy in, compression + decompression and copy out pipeline")
    ap.add_argument("--mode", choices=["batch", "streams"], default="batch",
                    help="batch: one batched compress + decompress call per step; "
                         "streams: one plain call per field, fields spread over --streams")
    ap.add_argument("--workload", choices=WORKLOADS, default="c3",
                    help="c3: 6 NYX-like 512^3 fields (default); c2: 13 hurricane-like "
                         "100x500x500 fields; c1: 24 climate-like 1800x3600 fields; c0: one "
                         "512x512 field")
    ap.add_argument("--fields", type=int, default=0, help="0 = the workload's field count")
    ap.add_argument("--ny", type=int, default=1800, help="c1: rows")
    ap.add_argument("--nx", type=int, default=3600, help="c1: columns")
    ap.add_argument("--n3", type=int, default=512, help="c3: points per axis")
    ap.add_argument("--cpu-steps", type=int, default=3,
                    help="CPU baseline: oracle steps (rounds of one task per worker); the "
                         "median is reported")
    ap.add_argument("--chunk", type=int, default=256)
    ap.add_argument("--autotune", action="store_true",
                    help="pick chunk size and tile shapes per target PSNR with fpsnr_autotune "
                         "(timed on the first field of each target, outside the timed region)")
    ap.add_argument("--serve", action="store_true",
                    help="serving workload instead of the batch: requests of mixed shapes and "
                         "targets with Poisson arrivals through the request server")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rates", type=str, default="1000,5000,10000,20000",
                    help="arrival rates (requests per second), one run each")
    ap.add_argument("--serve-serial", type=int, default=1000,
                    help="requests of the serial plain-call baseline")
    ap.add_argument("--tune-tol", type=float, default=0.01,
                    help="autotune: largest accepted compressed-size increase over the smallest")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve-run", action="store_true",
                    help="leave out the short served run (2,000 requests at 5,000 req/s) of the line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-roofline", action="store_true")
    ap.add_argument("--cpu-workers", type=int, default=0, help="0 = all host cores")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every call eagerly instead of replaying one CUDA graph per step")
    ap.add_argument("--psnr", type=float, default=0.0,
                    help="one target PSNR (dB) for every field instead of the mixed sweep "
                         "(field i -> {40,60,80,100,120}[i mod 5])")
    ap.add_argument("--write-traffic", metavar="CSV",
                    help="read an ncu --csv log of dram__bytes_{read,write}.sum and add it to "
                         "profiles/traffic.json under --workload (no GPU work)")
    ap.add_argument("--traffic-points", type=int, default=0,
                    help="--write-traffic: points one captured launch covers")
    ap.add_argument("--traffic-command", type=str, default="",
                    help="--write-traffic: the command line of the capture, recorded with it")
    ap.add_argument("--launch-table", metavar="CSV",
                    help="print the per-kernel launch table of an ncu --csv log of "
                         "gpu__time_duration.sum (no GPU work)")
    a = ap.parse_args()
    a.fields = a.fields or DEFAULT_FIELDS[a.workload]
    if a.workload == "c3" and a.fields > 6:
        ap.error("c3 has six fields")
    return a


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

WORKLOADS = ("c0", "c1", "c2", "c3")
DEFAULT_FIELDS = {"c0": 1, "c1": 24, "c2": 13, "c3": 6}
COSMO_TARGETS = (40.0, 60.0, 80.0)
HURRICANE_SHAPE = (100, 500, 500)


def field_shape(a):
    """numpy (C-order) shape of every field of the workload."""
    return {"c0": (512, 512), "c1": (a.ny, a.nx), "c2": HURRICANE_SHAPE,
            "c3": (a.n3, a.n3, a.n3)}[a.workload]


def targets(a, count):
    """Target PSNR of every field, or one value for all (--psnr)."""
    from paper_1805_07384_gb300 import synth
    if a.psnr > 0:
        return [a.psnr] * count
    if a.workload == "c0":
        return [80.0] * count
    if a.workload == "c1":
        return [synth.mixed_psnr(i) for i in range(count)]
    if a.workload == "c2":
        return [synth.psnr_sweep_3d(i) for i in range(count)]
    return [COSMO_TARGETS[i % 3] for i in range(count)]


def make_fields(a, seed, device):
    """The workload's float32 fields as torch tensors on `device`, drawn there
    (c1-c3) or on the host (c0, numpy); generation is never timed."""
    import torch
    from paper_1805_07384_gb300 import synth
    if a.workload == "c0":
        return [torch.from_numpy(synth.single_2d(512, seed=seed - 1)).to(device)
                for _ in range(a.fields)]
    if a.workload == "c1":
        return synth.climate_batch(a.fields, a.ny, a.nx, seed=seed, device=device)[0]
    if a.workload == "c2":
        return synth.hurricane_batch(a.fields, *HURRICANE_SHAPE, seed=seed, device=device)[0]
    fields, _ = synth.cosmology_fields(a.n3, seed=seed + 2, device=device)
    return [f.contiguous() for f in fields[:a.fields]]


def cpu_tasks(a, shape):
    """CPU-baseline tasks: (field index, first plane, end plane) of one oracle
    compress + decompress each.  Whole fields, except for c3, whose 512^3
    fields are cut into z-slabs of 64 planes so that every host core takes a
    share of every step (a slab is compressed as a field of its own)."""
    if a.workload == "c3":
        slab = 64
        return [(f, z0, min(z0 + slab, shape[0])) for z0 in range(0, shape[0], slab)
                for f in range(a.fields)]
    return [(f, 0, shape[0]) for f in range(a.fields)]


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

class ClockSampler:
    """SM clock, power and clock-event reasons of this process's GPU, read
    through NVML (libnvidia-ml, read-only queries) every 2 ms on a thread while
    the timed region runs; falls back to `nvidia-smi -lms 200` without NVML."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []          # (sm_mhz, reasons bitmask, power mW)
        self.smi_rows = []
        self.max_mhz = None
        self.proc = None
        self.thread = None
        self.stop_flag = threading.Event()
        self.nvml = None
        self.handle = None

    def _nvml_open(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
        except OSError:
            return False
        if lib.nvmlInit_v2() != 0:
            return False
        h = ctypes.c_void_p()
        props = None
        try:
            import torch
            props = torch.cuda.get_device_properties(self.device)
        except Exception:
            pass
        ok = False
        if props is not None and hasattr(props, "pci_bus_id"):
            bus = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0".encode()
            ok = lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(h)) == 0
        if not ok:
            idx = self.device.index if hasattr(self.device, "index") and self.device.index is not None else 0
            ok = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(h)) == 0
        if not ok:
            return False
        self.nvml, self.handle = lib, h
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
        return True

    def _poll(self):
        import ctypes
        lib, h = self.nvml, self.handle
        mhz, rs, mw = ctypes.c_uint(), ctypes.c_ulonglong(), ctypes.c_uint()
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop_flag.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0 and \
                    get_reasons(h, ctypes.byref(rs)) == 0:
                p = mw.value if lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(mw)) == 0 else None
                self.rows.append((float(mhz.value), int(rs.value), p))
            time.sleep(0.002)

    def start(self):
        if self._nvml_open():
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            t0 = time.perf_counter()
            while not self.rows and time.perf_counter() - t0 < 1.0:
                time.sleep(0.001)
            self.rows.clear()  # samples from here on fall inside the timed region
            return
        try:
            idx = self.device.index if self.device.index is not None else 0
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read_smi, daemon=True)
        self.thread.start()

    def _read_smi(self):
        for line in self.proc.stdout:
            self.smi_rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        self.stop_flag.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        if self.nvml is not None:
            rows = list(self.rows)
            if not rows:
                return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"],
                        "samples": 0, "source": "nvml"}
            reasons = sorted({name for _, r, _ in rows for bit, name in self.REASONS.items() if r & bit})
            pw = [p for _, _, p in rows if p is not None]
            return {"sm_mhz": statistics.median(m for m, _, _ in rows), "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(rows), "source": "nvml, 2 ms",
                    "power_w_max": round(max(pw) / 1000.0, 1) if pw else None}
        if not self.smi_rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[0]) for r in self.smi_rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.smi_rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.smi_rows for k in range(4)
                          if len(r) > 4 + k and r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.smi_rows), "source": "nvidia-smi, 200 ms"}


def oracle_task(args):
    """One oracle compress + decompress of planes [z0, z1) of a field held in
    the host field file (worker process).  Returns (seconds, blob bytes, PSNR)."""
    path, offset, shape, z0, z1, psnr, chunk = args
    import numpy as np
    import oracle
    x = np.memmap(path, dtype=np.float32, mode="r", offset=offset, shape=shape)[z0:z1]
    t0 = time.perf_counter()
    blob, st = oracle.compress(x, psnr, chunk=chunk)
    oracle.decompress(blob, x.shape)
    dt = time.perf_counter() - t0
    del x
    return dt, len(blob), st["psnr_actual"]


def _worker_ready(_):
    import oracle  # noqa: F401  (loads the oracle library in the worker)
    return os.getpid()


def cpu_pool(workers: int):
    """Spawned worker pool, returned once every worker has started and loaded
    the oracle, so that no worker start-up overlaps a timed region."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(workers)
    pool.map(_worker_ready, range(4 * workers), chunksize=1)
    return pool


class HostFields:
    """The workload's fields written once into one file (in /dev/shm when it
    has room, else the temporary directory), so that an oracle task carries
    only a path and an offset (no field crosses a pipe inside a timed
    region) and the workers read the pages from memory."""

    def __init__(self, arrays):
        import tempfile
        import numpy as np
        self.shapes = [tuple(x.shape) for x in arrays]
        self.offsets, off = [], 0
        for x in arrays:
            self.offsets.append(off)
            off += (4 * x.size + 4095) & ~4095
        d = "/dev/shm"
        try:
            st = os.statvfs(d)
            if st.f_bavail * st.f_frsize < off + (1 << 30):
                d = tempfile.gettempdir()
        except OSError:
            d = tempfile.gettempdir()
        fd, self.path = tempfile.mkstemp(prefix="fpsnr_fields_", suffix=".f32", dir=d)
        os.close(fd)
        m = np.memmap(self.path, dtype=np.uint8, mode="w+", shape=(max(off, 4096),))
        for x, o in zip(arrays, self.offsets):
            m[o:o + 4 * x.size] = np.ascontiguousarray(x, dtype=np.float32).reshape(-1).view(np.uint8)
        m.flush()
        del m

    def args(self, task, psnrs, chunk):
        f, z0, z1 = task
        return (self.path, self.offsets[f], self.shapes[f], z0, z1, psnrs[f], chunk)

    def task_bytes(self, task):
        f, z0, z1 = task
        plane = 4 * math.prod(self.shapes[f][1:])
        return plane * (z1 - z0)

    def close(self):
        try:
            os.unlink(self.path)
        except OSError:
            pass


def run_cpu_steps(pool, hf, tasks, psnrs, chunk, workers, steps, first=0):
    """`steps` oracle steps; step k runs the next round of `workers` tasks
    (cycling through the task list) on the pool.  Returns [(wall s, bytes,
    [(task, task bytes, result)])]."""
    out = []
    k = first
    per = min(workers, len(tasks))
    for _ in range(steps):
        batch = [tasks[(k + j) % len(tasks)] for j in range(per)]
        k += per
        t0 = time.perf_counter()
        res = pool.map(oracle_task, [hf.args(t, psnrs, chunk) for t in batch], chunksize=1)
        wall = time.perf_counter() - t0
        tb = [hf.task_bytes(t) for t in batch]
        out.append((wall, sum(tb), list(zip(batch, tb, res))))
    return out


def cpu_baseline_summary(a, runs, workers, ntasks):
    """The cpu_baseline object: the median over the steps of a round's bytes
    over its wall time, and the single-core GB/s of every task (each worker
    runs one task on one core)."""
    rates = [b / w / 1e9 for w, b, _ in runs]
    one_core = [b / r[0] / 1e9 for _, _, tr in runs for _, b, r in tr if r[0] > 0]
    per = len(runs[0][2]) if runs else 0
    unit = "64-plane z-slab" if a.workload == "c3" else "field"
    out = {"value": round(statistics.median(rates), 4), "unit": "GB/s", "cores": workers,
           "kind": "oracle",
           "sample": f"{len(runs)} steps, each {per} oracle compress + decompress tasks (one "
                     f"{unit} per worker process, cycling through the workload's {ntasks} "
                     f"{unit}s); value = median over the steps of the round's original bytes "
                     f"over its wall time ({', '.join(f'{w:.3g}' for w, _, _ in runs)} s)",
           "steps_gbs": [round(v, 4) for v in rates]}
    if one_core:
        out["one_core_gbs_per_task"] = {"median": round(statistics.median(one_core), 4),
                                        "min": round(min(one_core), 4),
                                        "max": round(max(one_core), 4)}
    return out


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------

def host_fields(a, seed):
    """The workload's fields as numpy float32 arrays: drawn with torch on the
    GPU when there is one (the same inputs the GPU arm compresses), else on
    the host."""
    import torch
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
    xs = make_fields(a, seed, dev)
    out = [x.cpu().numpy() for x in xs]
    del xs
    if dev.type == "cuda":
        torch.cuda.empty_cache()
    return out


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    workers = a.cpu_workers or os.cpu_count() or 1
    shape = field_shape(a)
    tasks = cpu_tasks(a, shape)
    workers = max(1, min(workers, len(tasks)))
    pool = cpu_pool(workers)  # spawned before the first GPU call
    hf = HostFields(host_fields(a, rank_seed(0)))
    psnrs = targets(a, a.fields)
    try:
        run_cpu_steps(pool, hf, tasks, psnrs, a.chunk, workers, a.warmup)
        runs = run_cpu_steps(pool, hf, tasks, psnrs, a.chunk, workers, a.steps,
                             first=a.warmup * workers)
    finally:
        pool.close()
        hf.close()
    wall = sum(w for w, _, _ in runs)
    nbytes = sum(b for _, b, _ in runs)
    value = nbytes / wall / 1e9
    ms = 1e3 * wall / len(runs)
    cpu = cpu_baseline_summary(a, runs, workers, len(tasks))
    cpu["value"] = round(value, 4)
    cpu["sample"] = cpu["sample"].replace("median over the steps of", "total over the steps of")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(a, streams=None),
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


WORKLOAD_TEXT = {
    "c0": "one 2D float32 GRF field 512x512 (P(k)~k^-3, rescaled to [-1,1], seed 0), 2D Lorenzo",
    "c1": "{F} climate-like 2D float32 GRF fields {ny}x{nx} (alpha~U[2,4], affine offsets "
          "1e-3..1e5, 1 field with a constant rectangle), 2D Lorenzo",
    "c2": "{F} hurricane-like 3D float32 fields 100x500x500 (anisotropic GRFs, correlation length "
          "4x longer horizontally; field 0 with a vortex mean; 2 fields with 0.1% spikes at "
          "50 std), 3D Lorenzo",
    "c3": "{F} NYX-like 3D float32 fields {n}^3 (2 lognormal densities exp(2G), G a GRF with "
          "P(k)~k^-2; 3 velocity GRFs P(k)~k^-3; 1 temperature exp(G)), 3D Lorenzo",
}
TARGET_TEXT = {"c0": "target PSNR 80 dB",
               "c1": "target PSNR field i -> {40,60,80,100,120}[i mod 5] dB",
               "c2": "target PSNR field i -> 30 + 10 (i mod 10) dB",
               "c3": "target PSNR field i -> {40,60,80}[i mod 3] dB"}


def workload_config(a, streams):
    shape = field_shape(a)
    total = a.fields * 4 * math.prod(shape)
    text = WORKLOAD_TEXT[a.workload].format(F=a.fields, ny=a.ny, nx=a.nx, n=a.n3)
    tgt = f"target PSNR {a.psnr:g} dB for every field" if a.psnr > 0 else TARGET_TEXT[a.workload]
    c = {"workload": f"{a.workload}: {text}, {tgt}, R=32768, chunk {a.chunk}",
         "name": a.workload, "fields": a.fields, "shape": list(shape), "radius": 32768,
         "chunk": a.chunk, "lorenzo_dims": len(shape),
         "l2": (f"inputs {total / 1e6:.0f} MB > 129 MB L2, no flush" if total > L2_FLUSH_BELOW else
                f"inputs {total / 1e6:.1f} MB fit the 129 MB L2: a 512 MB buffer is written "
                f"between timed steps (outside the events) to flush it")}
    if streams is not None:
        c["mode"] = getattr(a, "mode", "batch")
        if c["mode"] == "streams":
            c["streams"] = streams
        else:
            c["sub_batches"] = max(1, min(a.sub_batches, a.fields, streams))
        c["launch"] = "eager" if getattr(a, "no_graph", False) else "one CUDA graph per step"
    return c


# inputs at most this large are timed step by step with an L2 flush in between
L2_FLUSH_BELOW = 256 * 10**6


# ---------------------------------------------------------------------------
# multi-rank helpers (one process per GPU; fields shard with no data-path collective)
# ---------------------------------------------------------------------------

def max_over_ranks(ms: float, world: int, dist=None, device=None) -> float:
    """Step time of the slowest rank (the only collective: one float)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gbs(bytes_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: every rank processes its own batch (weak scaling)."""
    return world * bytes_per_rank / (ms / 1e3) / 1e9


def rank_seed(rank: int) -> int:
    """Each rank compresses its own seeded batch."""
    return 1 + 1000 * rank


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def measured_traffic(workload, stage, points):
    """DRAM bytes of one launch of `stage` over `points` points, from the
    committed ncu capture of the same workload (bytes per point on a smaller
    case, times the points), or None when the capture is missing or a file the
    kernel's binary depends on changed since the counters were taken."""
    import hashlib
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tf):
        return None
    e = json.load(open(tf)).get(workload, {}).get(stage)
    if not e:
        return None
    for rel, sha in e["sources"].items():
        src = os.path.join(ROOT, rel)
        if not os.path.exists(src) or hashlib.sha1(open(src, "rb").read()).hexdigest() != sha:
            return None
    return int(round(e["dram_bytes_per_point"] * points))


# ncu --csv logs -> per-launch figures (profiles/ summaries and traffic.json)

# files every kernel's traffic depends on besides its own source: the shared
# device header, the build script with the compiler flags, and the plan set-up
# that chooses tile shapes and slab depths
_TRAFFIC_DEPS = (os.path.join("paper_1805_07384_gb300", "csrc", "common.cuh"),
                 os.path.join("paper_1805_07384_gb300", "build.py"),
                 os.path.join("paper_1805_07384_gb300", "csrc", "api.cu"))
_UNITS = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9,
          "ns": 1e-3, "nsecond": 1e-3, "us": 1, "usecond": 1, "ms": 1e3, "msecond": 1e3}
# benchmark stages by kernel-name prefix, with the source file that holds them
_STAGE_KERNELS = [("range_plan", ("k_range_plan",), "compress.cu"),
                  ("predict_quantize", ("k_pq",), "compress.cu"),
                  ("encode", ("k_enc_pack", "k_enc_scan", "k_enc_copy"), "compress.cu"),
                  ("decode", ("k_decode",), "decompress.cu"),
                  ("band_sum", ("k_band_sum", "k_vol_sum"), "decompress.cu"),
                  ("scan_final_dequant", ("k_band_scan", "k_vol_scan"), "decompress.cu")]


def _ncu_rows(path):
    """(launch id, short kernel name, metric, value in bytes or microseconds)."""
    import csv
    lines = open(path).read().splitlines()
    start = next(i for i, l in enumerate(lines) if l.startswith('"ID"'))
    out = []
    for r in csv.DictReader(lines[start:]):
        name = r["Kernel Name"]
        short = name.split("(")[0].replace("void ", "").strip()
        if short.startswith("fp::"):
            short = short[4:]
        elif not short.startswith("k_"):
            continue  # not one of the library's kernels (input generation, torch)
        v = float(r["Metric Value"].replace(",", "")) * _UNITS.get(r["Metric Unit"], 1)
        out.append((int(r["ID"]), short, r["Metric Name"], v))
    return out


def launch_table(path):
    """Markdown table: launches, total device time and share per kernel."""
    per = {}
    for lid, k, m, v in _ncu_rows(path):
        if m == "gpu__time_duration.sum":
            n, t = per.get(k, (0, 0.0))
            per[k] = (n + 1, t + v)
    tot = sum(t for _, t in per.values()) or 1.0
    rows = ["| kernel | launches | total us | share |", "|---|---:|---:|---:|"]
    for k, (n, t) in sorted(per.items(), key=lambda kv: -kv[1][1]):
        rows.append(f"| `{k}` | {n} | {t:.1f} | {100 * t / tot:.1f}% |")
    return "\n".join(rows)


def write_traffic(path, workload, points, command):
    """Adds to profiles/traffic.json, under `workload`, the DRAM bytes per
    point of every benchmark stage found in an ncu --csv log of
    dram__bytes_{read,write}.sum (each launch covering `points` points), with
    the SHA-1 of the kernel's source file and of the files every kernel build
    depends on (the shared device header and the build script with the
    compiler flags).  A stage of several kernels needs all of them in the log
    (or in logs added one after another: entries of a stage's other kernels
    are kept)."""
    import hashlib
    launches = {}
    for lid, k, m, v in _ncu_rows(path):
        if m in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            launches.setdefault((lid, k), {})[m] = v
    dst = os.path.join(ROOT, "profiles", "traffic.json")
    out = json.load(open(dst)) if os.path.exists(dst) else {}
    out["_about"] = ("DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per point of each "
                     "benchmark stage, per workload: the average over the captured launches of a "
                     "small case of the workload (one kernel per capture, at most three launches), "
                     "divided by the points one launch covers; bench.py reports it, times the points "
                     "of its own launch, as roofline.traffic only while the recorded SHA-1s match.")
    wl = out.setdefault(workload, {})
    for stage, prefixes, src in _STAGE_KERNELS:
        per_kernel = {}
        for (lid, k), mv in launches.items():
            if k.startswith(prefixes):
                e = per_kernel.setdefault(k, [0, 0.0, 0.0])
                e[0] += 1
                e[1] += mv.get("dram__bytes_read.sum", 0.0)
                e[2] += mv.get("dram__bytes_write.sum", 0.0)
        if not per_kernel:
            continue
        entry = wl.setdefault(stage, {"kernels": {}})
        for k, (n, rd, wr) in per_kernel.items():
            entry["kernels"][k] = {"launches": n, "read_per_point": rd / n / points,
                                   "write_per_point": wr / n / points, "points_per_launch": points,
                                   "command": command}
        rel = os.path.join("paper_1805_07384_gb300", "csrc", src)
        deps = {d: hashlib.sha1(open(os.path.join(ROOT, d), "rb").read()).hexdigest()
                for d in (rel,) + _TRAFFIC_DEPS if os.path.exists(os.path.join(ROOT, d))}
        entry["sources"] = deps
        entry["dram_bytes_per_point"] = round(sum(v["read_per_point"] + v["write_per_point"]
                                                  for v in entry["kernels"].values()), 4)
    with open(dst, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(dst)


# algorithmic bytes per launch of each stage (N points, B compressed bytes of one
# field; ndim of the predictor)
def stage_bytes(stage, N, B, ndim=2):
    # decode writes 16-bit symbols; the tile (3D) or band (2D) sums read them,
    # and the final scan reads them again and writes the floats (the sums and
    # their prefixes, N / 16 to N / 4 bytes, are not counted).  3D rows wider
    # than a tile covers take look-back scans instead: the x pass reads the
    # symbols and writes int32 lattice sums, the y pass reads and writes them,
    # the z pass reads them and writes the floats.
    table = {"range_plan": 4 * N, "predict_quantize": 6 * N, "encode": 2 * N + B,
             "decode": B + 2 * N, "band_sum": 2 * N, "scan_final_dequant": 6 * N}
    if ndim == 3:
        table.update({"scan_x": 6 * N, "scan_y": 8 * N})
    return table.get(stage)


# ---------------------------------------------------------------------------
# serving workload
# ---------------------------------------------------------------------------

SERVE_SHAPES = [(64, 64), (512, 512), (1800, 3600), (64, 64, 64), (100, 500, 500), (256, 256, 256)]
SERVE_BUCKETS = [30.0 + 10.0 * k for k in range(10)]


def serve_field(shape, seed, device):
    """The workload generators by shape: 512^2-style isotropic GRF, climate-like
    field with an affine offset, hurricane-like anisotropic 3D GRF (z stretched
    4x), cosmology-like 3D velocity GRF; float32 on `device`."""
    import torch
    from paper_1805_07384_gb300 import synth
    if len(shape) == 2 and shape != (1800, 3600):
        g = synth.grf_torch(shape, 3.0, seed, device)
    elif len(shape) == 2:
        g = synth.grf_torch(shape, 3.0, seed, device) * 1e2 + 5e3
    elif shape == (100, 500, 500):
        g = synth.grf_torch(shape, 3.0, seed, device, stretch=(4.0, 1.0, 1.0))
    else:
        g = synth.grf_torch(shape, 3.0, seed, device)
    return g.to(torch.float32).contiguous()


SERVE_LARGE_POOL = 8  # distinct seeded inputs of each large shape (>= 16 MB)


class ServeSetup:
    """Inputs, blobs and output buffers of a request stream.  Requests are
    drawn first (Poisson arrivals, shape uniform over SERVE_SHAPES, target
    U[30, 120] dB, compress or decompress at even odds); every request's input
    is seeded by its own id for the small shapes, and is one of
    SERVE_LARGE_POOL seeded fields for the large ones (1800x3600, 100x500x500,
    256^3), to bound the memory held.  A decompression request gets the blob of
    its input at the nearest 10 dB target, made beforehand."""

    def __init__(self, dev, request_lists):
        import numpy as np
        import torch
        from paper_1805_07384_gb300 import fpsnr
        self.nbytes = {s: 4 * int(np.prod(s)) for s in SERVE_SHAPES}
        self.large = {s: self.nbytes[s] >= (16 << 20) for s in SERVE_SHAPES}
        self.fields, need_blob = {}, set()
        for reqs in request_lists:
            for (ta, s, psnr, kind, rid) in reqs:
                key = (s, self.input_id(s, rid))
                if key not in self.fields:
                    self.fields[key] = serve_field(s, 7919 * SERVE_SHAPES.index(s) + key[1], dev)
                if kind == 1:
                    need_blob.add((key, self.bucket(psnr)))
        self.blobs = {}
        plans = {s: fpsnr.Plan(s, 60.0) for s in SERVE_SHAPES}
        for (key, b) in sorted(need_blob):
            p = plans[key[0]]
            p.set_psnr(b)
            out, nb, st = p.compress(self.fields[key])
            torch.cuda.synchronize()
            n = int(nb.item())
            assert fpsnr.parse_stats(st)["status"] == 0
            self.blobs[(key, b)] = (out[:n].clone(), n)
            del out
        for p in plans.values():
            p.close()
        # output buffers per shape (a compressed blob may take up to 4n + 1 MiB)
        self.pool_n = {s: (64 if self.nbytes[s] <= (4 << 20) else (16 if self.nbytes[s] <= (64 << 20) else 8))
                       for s in SERVE_SHAPES}
        cap = {s: self.nbytes[s] + (1 << 20) for s in SERVE_SHAPES}
        self.bufs = {s: [torch.empty(cap[s], dtype=torch.uint8, device=dev) for _ in range(self.pool_n[s])]
                     for s in SERVE_SHAPES}

    def input_id(self, s, rid):
        return rid % SERVE_LARGE_POOL if self.large[s] else rid

    @staticmethod
    def bucket(psnr):
        return min(SERVE_BUCKETS, key=lambda v: abs(v - psnr))

    def describe(self):
        return ("requests with Poisson arrivals; shape uniform over "
                + ", ".join("x".join(map(str, s)) for s in SERVE_SHAPES)
                + "; target PSNR U[30,120] dB; half compress, half decompress of a blob made "
                  "beforehand at the nearest 10 dB target; every request's input seeded by its id "
                  f"for the small shapes, one of {SERVE_LARGE_POOL} seeded fields for the shapes of "
                  "16 MB and more; inputs resident on the device")


def serve_requests(n, rate, seed):
    """(arrival us, shape, target, kind 0 compress / 1 decompress, request id)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1e6 / rate, size=n)
    out = []
    t = 0.0
    for i in range(n):
        t += gaps[i]
        s = SERVE_SHAPES[int(rng.integers(len(SERVE_SHAPES)))]
        psnr = float(rng.uniform(30.0, 120.0))
        kind = int(rng.integers(2))
        out.append((t, s, psnr, kind, i + 1000000 * seed))
    return out


def serve_session(srv, setup, reqs, rate):
    """Submits the requests at their arrival times through the server and
    returns latency percentiles and served GB/s."""
    import torch
    free = {s: list(range(setup.pool_n[s])) for s in SERVE_SHAPES}
    owner, lat, done_t, failed = {}, [], [], 0
    total_bytes = 0
    st0 = srv.stats()

    def collect(block):
        nonlocal total_bytes, failed
        while True:
            item = srv.take_any()
            if item is None:
                if not block:
                    return
                time.sleep(20e-6)
                continue
            t, r = item
            s, bi = owner.pop(t)
            free[s].append(bi)
            if r["status"]:
                failed += 1
            else:
                lat.append(r["done_us"] - r["arrival_us"])
                total_bytes += setup.nbytes[s]
            done_t.append(r["done_us"])
            return

    t0 = srv.now() + 20000.0
    for (ta, s, psnr, kind, rid) in reqs:
        while not free[s]:
            collect(True)
        collect(False)
        bi = free[s].pop()
        buf = setup.bufs[s][bi]
        key = (s, setup.input_id(s, rid))
        if kind == 0:
            t = srv.submit_compress(setup.fields[key], psnr, buf, arrival_us=t0 + ta)
        else:
            blob, n = setup.blobs[(key, setup.bucket(psnr))]
            t = srv.submit_decompress(blob, n, buf[:setup.nbytes[s]].view(torch.float32).view(s),
                                      arrival_us=t0 + ta)
        owner[t] = (s, bi)
    while owner:
        collect(True)
    st1 = srv.stats()
    span = (max(done_t) - t0) / 1e6
    lat_ms = sorted(v / 1e3 for v in lat)
    q = lambda f: lat_ms[min(len(lat_ms) - 1, int(f * (len(lat_ms) - 1) + 0.5))]
    nb = st1["batches"] - st0["batches"]
    return {"rate_rps": rate, "requests": len(reqs), "failed": failed,
            "p50_ms": round(q(0.5), 3), "p99_ms": round(q(0.99), 3),
            "max_ms": round(lat_ms[-1], 3), "gbs": round(total_bytes / span / 1e9, 2),
            "offered_gbs": round(sum(setup.nbytes[s] for _, s, _, _, _ in reqs) /
                                 (reqs[-1][0] / 1e6) / 1e9, 2),
            "batches": nb, "mean_batch": round(len(reqs) / max(nb, 1), 2)}


SERVER_OPTS = {"hbm_budget": 40 << 30, "max_batch": 16, "streams": 4}


def warm_server(srv, setup):
    """One request of each kind per shape, so that every plan is cached."""
    import torch
    for s in SERVE_SHAPES:
        key = next(k for k in setup.fields if k[0] == s)
        srv.wait(srv.submit_compress(setup.fields[key], 60.0, setup.bufs[s][0]))
        bk = next((k for k in setup.blobs if k[0][0] == s), None)
        if bk is not None:
            blob, n = setup.blobs[bk]
            srv.wait(srv.submit_decompress(blob, n, setup.bufs[s][0][:setup.nbytes[s]].view(torch.float32).view(s)))


def served_short(dev, rate=5000.0, n=2000):
    """The short served run of the default benchmark line."""
    from paper_1805_07384_gb300 import fpsnr
    reqs = serve_requests(n, rate, seed=5)
    setup = ServeSetup(dev, [reqs])
    srv = fpsnr.Server(**SERVER_OPTS)
    try:
        warm_server(srv, setup)
        r = serve_session(srv, setup, reqs, rate)
    finally:
        srv.close()
    r["inputs"] = setup.describe()
    r["latency"] = "completion observed by the server minus scheduled arrival"
    return r


def run_serve(a):
    import torch
    from paper_1805_07384_gb300 import build as fbuild
    fbuild.build()
    from paper_1805_07384_gb300 import fpsnr
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rates = [float(r) for r in a.serve_rates.split(",")]
    lists = [serve_requests(a.serve_requests, rate, seed=int(rate)) for rate in rates]
    serial = serve_requests(a.serve_serial, rates[0], seed=1)
    setup = ServeSetup(dev, lists + [serial])
    srv = fpsnr.Server(**SERVER_OPTS)
    warm_server(srv, setup)
    runs = [serve_session(srv, setup, reqs, rate) for reqs, rate in zip(lists, rates)]
    pst = srv.stats()
    srv.close()

    # serial plain calls
    plans = {s: fpsnr.Plan(s, 60.0) for s in SERVE_SHAPES}
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    tot = 0
    for (ta, s, psnr, kind, rid) in serial:
        p = plans[s]
        buf = setup.bufs[s][0]
        key = (s, setup.input_id(s, rid))
        if kind == 0:
            p.set_psnr(psnr)
            p.compress(setup.fields[key], out=buf)
        else:
            blob, n = setup.blobs[(key, setup.bucket(psnr))]
            p.decompress(blob, n, out=buf[:setup.nbytes[s]].view(torch.float32).view(s))
        torch.cuda.synchronize()
        tot += setup.nbytes[s]
    serial_gbs = tot / (time.perf_counter() - w0) / 1e9
    for p in plans.values():
        p.close()
    line = {"metric": "served compress/decompress requests: p50/p99 latency and aggregate GB/s",
            "unit": "ms / GB/s", "n_gpus": 1, "data": "synthetic", "impl": "ours",
            "config": {"workload": setup.describe(), "server": SERVER_OPTS,
                       "latency": "completion observed by the server minus scheduled arrival"},
            "runs": runs,
            "serial_plain": {"gbs": round(serial_gbs, 2), "requests": len(serial),
                             "note": "one plain call per request, synchronized after each"},
            "plans_cached": pst["plans"], "plan_bytes": pst["plan_bytes"]}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.write_traffic:
        write_traffic(a.write_traffic, a.workload, a.traffic_points, a.traffic_command)
        return
    if a.launch_table:
        print(launch_table(a.launch_table))
        return
    if a.impl == "reference":
        run_reference(a)
        return
    if a.serve:
        run_serve(a)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    shape = field_shape(a)
    N = math.prod(shape)
    ndim = len(shape)
    # CPU baseline pool first (spawn, before the first GPU call), rank 0 only
    pool = None
    tasks = cpu_tasks(a, shape)
    if rank == 0 and not a.no_cpu_baseline:
        workers = a.cpu_workers or os.cpu_count() or 1
        workers = max(1, min(workers, len(tasks)))
        import oracle
        oracle.build()
        pool = cpu_pool(workers)
        pool_workers = workers

    from paper_1805_07384_gb300 import build as fbuild
    fbuild.build()
    from paper_1805_07384_gb300 import fpsnr

    F, S = a.fields, max(1, a.streams)
    fields = make_fields(a, rank_seed(rank), dev)
    psnrs = targets(a, F)
    tuning = None
    if a.autotune:
        tuning = {}
        for ps in sorted(set(psnrs)):
            i0 = psnrs.index(ps)
            tuning[ps] = fpsnr.autotune(fields[i0], ps, max_size_increase=a.tune_tol, chunk=a.chunk)
        plans = []
        for i in range(F):
            t = tuning[psnrs[i]]
            p = fpsnr.Plan(shape, psnrs[i], chunk=t["chunk"])
            # the decoder's block size is left to each batched launch
            p.set_tuning({"pq_tile_x": t["pq_tile_x"], "band_rows": t["band_rows"]})
            plans.append(p)
    else:
        plans = [fpsnr.Plan(shape, psnrs[i], chunk=a.chunk) for i in range(F)]
    outs = [p.alloc_out() for p in plans]
    nbs = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(F)]
    sts = [torch.zeros(fpsnr.STATS_BYTES, dtype=torch.uint8, device=dev) for _ in range(F)]
    recs = [torch.empty(shape, dtype=torch.float32, device=dev) for _ in range(F)]
    dsts = [torch.zeros(1, dtype=torch.int32, device=dev) for _ in range(F)]
    streams = [torch.cuda.Stream(device=dev) for _ in range(S)]
    main_s = torch.cuda.current_stream(dev)


    # batch mode: the fields split into `nsub` sub-batches, one per stream, so
    # that one sub-batch's latency-bound stages overlap another's bandwidth work
    nsub = max(1, min(a.sub_batches, F, S))
    # fields dealt round-robin in order of decreasing target (the dearest
    # first), so that every sub-batch gets a share of the expensive ones
    dealt = sorted(range(F), key=lambda i: (-psnrs[i], i))
    groups = [sorted(dealt[g::nsub]) for g in range(nsub)]
    nb_all = [torch.zeros(len(g), dtype=torch.int64, device=dev) for g in groups]
    st_all = [torch.zeros((len(g), fpsnr.STATS_BYTES), dtype=torch.uint8, device=dev) for g in groups]
    dst_all = [torch.zeros(len(g), dtype=torch.int32, device=dev) for g in groups]
    # the end-to-end run pipelines copies with compute over finer sub-batches
    # (contiguous fields, one stream each); outputs are per field as above
    ne = max(1, min(a.e2e_sub_batches, F))
    # pipeline order: cheap and dear fields (by target: high targets have wide
    # alphabets) alternate, cheapest first, so that the compute load is even
    # along the pipeline and the copy-out side starts early and never starves
    by_cost = sorted(range(F), key=lambda i: (psnrs[i], i))
    lo, hi = by_cost[:F // 2], by_cost[F // 2:][::-1]
    order = [v for pair in zip(lo, hi) for v in pair] + lo[len(hi):] + hi[len(lo):]
    egroups = [order[F * g // ne:F * (g + 1) // ne] for g in range(ne)]
    estreams = [torch.cuda.Stream(device=dev) for _ in range(ne)]
    cin = torch.cuda.Stream(device=dev)
    enb = [torch.zeros(len(g), dtype=torch.int64, device=dev) for g in egroups]
    est = [torch.zeros((len(g), fpsnr.STATS_BYTES), dtype=torch.uint8, device=dev) for g in egroups]
    edst = [torch.zeros(len(g), dtype=torch.int32, device=dev) for g in egroups]

    def step_batch(h2d=None, d2h=None, serial=False):
        cur = torch.cuda.current_stream(dev)
        ev = torch.cuda.Event()
        ev.record(cur)
        if h2d is not None and not serial:
            # copies in, in pipeline order, on one stream (each field's input
            # lands as early as it can); each sub-batch computes on its own stream
            # once its inputs are in and copies its results out right after (no
            # sub-batch waits behind a slower one)
            cin.wait_event(ev)
            done_in = []
            with torch.cuda.stream(cin):
                for idx in egroups:
                    for i in idx:
                        fields[i].copy_(h2d[i], non_blocking=True)
                    e = torch.cuda.Event()
                    e.record(cin)
                    done_in.append(e)
            for gi, idx in enumerate(egroups):
                s = estreams[gi]
                s.wait_event(done_in[gi])
                with torch.cuda.stream(s):
                    gp = [plans[i] for i in idx]
                    fpsnr.compress_batch(gp, [fields[i] for i in idx], outs=[outs[i] for i in idx],
                                         nbytes=enb[gi], stats=est[gi], stream=s)
                    fpsnr.decompress_batch(gp, [outs[i] for i in idx], outs=[recs[i] for i in idx],
                                           status=edst[gi], stream=s)
                    for i in idx:
                        d2h[0][i].copy_(recs[i], non_blocking=True)
                    d2h[1][gi].copy_(est[gi], non_blocking=True)
                e = torch.cuda.Event()
                e.record(s)
                cur.wait_event(e)
            return
        for gi, idx in enumerate(groups):
            s = cur if serial else streams[gi]
            if not serial:
                s.wait_event(ev)
            with torch.cuda.stream(s):
                if h2d is not None:
                    for i in idx:
                        fields[i].copy_(h2d[i], non_blocking=True)
                gp = [plans[i] for i in idx]
                fpsnr.compress_batch(gp, [fields[i] for i in idx], outs=[outs[i] for i in idx],
                                     nbytes=nb_all[gi], stats=st_all[gi], stream=s)
                fpsnr.decompress_batch(gp, [outs[i] for i in idx], outs=[recs[i] for i in idx],
                                       status=dst_all[gi], stream=s)
                if d2h is not None:
                    for i in idx:
                        d2h[0][i].copy_(recs[i], non_blocking=True)
                    d2h[1][gi].copy_(st_all[gi], non_blocking=True)
        for gi in range(len(groups) if not serial else 0):
            e = torch.cuda.Event()
            e.record(streams[gi])
            cur.wait_event(e)

    def step(nstreams, h2d=None, d2h=None):
        if a.mode == "batch":
            step_batch(h2d, d2h, serial=(nstreams == 1))
            return
        cur = torch.cuda.current_stream(dev)
        ev = torch.cuda.Event()
        ev.record(cur)
        for s in streams[:nstreams]:
            s.wait_event(ev)
        for i in range(F):
            s = streams[i % nstreams]
            if h2d is not None:
                with torch.cuda.stream(s):
                    fields[i].copy_(h2d[i], non_blocking=True)
            plans[i].compress(fields[i], out=outs[i], nbytes=nbs[i], stats=sts[i], stream=s)
            plans[i].decompress(outs[i], outs[i].numel(), out=recs[i], status=dsts[i], stream=s)
            if d2h is not None:
                with torch.cuda.stream(s):
                    d2h[0][i].copy_(recs[i], non_blocking=True)
                    d2h[1][i].copy_(sts[i], non_blocking=True)
        for s in streams[:nstreams]:
            e = torch.cuda.Event()
            e.record(s)
            cur.wait_event(e)

    graphs = {}

    def run_step(nstreams, graph, **kw):
        """One step: a replay of the captured graph, or eager launches."""
        if not graph:
            step(nstreams, **kw)
            return
        key = (nstreams, "h2d" in kw and kw["h2d"] is not None)
        if key not in graphs:
            torch.cuda.synchronize(dev)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step(nstreams, **kw)
            torch.cuda.synchronize(dev)
            graphs[key] = g
        graphs[key].replay()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # inputs that fit L2 are timed step by step, with a 512 MB write between
    # the steps (outside the events) that evicts them
    flush = (torch.empty(512 * 2**20, dtype=torch.uint8, device=dev)
             if 4 * N * F <= L2_FLUSH_BELOW else None)

    def timed(k, nstreams, graph=False, **kw):
        barrier()
        wall0 = time.perf_counter()
        if flush is None:
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(main_s)
            for _ in range(k):
                run_step(nstreams, graph, **kw)
            t1.record(main_s)
            barrier()
            total = t0.elapsed_time(t1)
        else:
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(k)]
            for e0, e1 in ev:
                flush.zero_()
                e0.record(main_s)
                run_step(nstreams, graph, **kw)
                e1.record(main_s)
            barrier()
            total = sum(e0.elapsed_time(e1) for e0, e1 in ev)
        ms = max_over_ranks(total / k, world, dist, dev)
        return ms, (time.perf_counter() - wall0)

    use_graph = not a.no_graph
    for _ in range(max(3, a.warmup)):
        step(S)
    # kernels one step launches (the same kernels run eagerly or inside the graph)
    barrier()
    for p in plans:
        fpsnr.fpsnr_plan_profile_read(p.handle)
    step(S)
    barrier()
    launches_per_step = 0
    for p in plans:
        launches_per_step += sum(v[1] for v in fpsnr.fpsnr_plan_profile_read(p.handle).values())
    if use_graph:
        run_step(S, True)  # capture
        for _ in range(2):
            run_step(S, True)
    barrier()
    for p in plans:
        fpsnr.fpsnr_plan_profile_read(p.handle)  # reset launch counters

    clocks = ClockSampler(dev)
    clocks.start()
    ms, wall = timed(a.steps, S, graph=use_graph)
    clk = clocks.stop()
    launches = launches_per_step * a.steps

    total_bytes = 4 * N * F
    value = aggregate_gbs(total_bytes, world, ms)

    # per-field results (outside the timed region)
    per_field = []
    dev_abs, meets, crs = [], [], []
    if a.mode == "batch":
        order = [i for g in groups for i in g]
        stat_rows = [None] * F
        dec_status = [None] * F
        for gi, g in enumerate(groups):
            for j, i in enumerate(g):
                stat_rows[i] = st_all[gi][j]
                dec_status[i] = dst_all[gi][j]
    else:
        stat_rows, dec_status = sts, dsts
    for i in range(F):
        st = fpsnr.parse_stats(stat_rows[i])
        assert st["status"] == 0 and int(dec_status[i].item()) == 0, (i, st["status"])
        p_meas, _, _ = fpsnr.psnr(fields[i], recs[i])
        assert p_meas == st["psnr_actual"] or abs(p_meas - st["psnr_actual"]) < 1e-9
        cr = 4 * N / st["bytes"]
        per_field.append({"target": psnrs[i], "actual": round(st["psnr_actual"], 6),
                          "model": round(st["psnr_model"], 6), "cr": round(cr, 3),
                          "outliers": st["n_outlier"], "verbatims": st["n_verbatim"],
                          "symbols": st["n_sym"]})
        if math.isfinite(st["psnr_actual"]):
            dev_abs.append(abs(st["psnr_actual"] - psnrs[i]))
            meets.append(st["psnr_actual"] >= psnrs[i])
        crs.append(cr)

    # roofline pass: same K steps, one stream, per-launch events
    roof = None
    stage_table = None
    if not a.no_roofline:
        for p in plans:
            fpsnr.fpsnr_plan_profile(p.handle, True)
            fpsnr.fpsnr_plan_profile_read(p.handle)
        ms1, _ = timed(a.steps, 1)
        agg = {}
        comp_bytes = [fpsnr.parse_stats(stat_rows[i])["bytes"] for i in range(F)]
        for p in plans:
            for name, (t, n) in fpsnr.fpsnr_plan_profile_read(p.handle).items():
                e = agg.setdefault(name, [0.0, 0, 0])
                e[0] += t
                e[1] += n
            fpsnr.fpsnr_plan_profile(p.handle, False)
        for name, e in agg.items():
            # algorithmic bytes of the stage for every field, every timed step
            sb = [stage_bytes(name, N, comp_bytes[i], ndim) for i in range(F)]
            e[2] = a.steps * sum(sb) if e[1] and all(v is not None for v in sb) else 0
        step_ms = ms1
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
        peak = peaks["hbm_gbs"] if peaks else 6800.0
        stage_table = {}
        for k, v in agg.items():
            if not v[1]:
                continue
            gbs = v[2] / (v[0] / 1e3) / 1e9 if v[0] > 0 and v[2] else None
            stage_table[k] = {"ms_per_step": round(v[0] / a.steps, 4),
                              "launches_per_step": v[1] // a.steps,
                              "share": round(v[0] / a.steps / step_ms, 4),
                              "gbs": round(gbs, 1) if gbs else None,
                              "frac_of_hbm": round(gbs / peak, 4) if gbs else None}
        bw_stages = {k: v for k, v in agg.items() if stage_bytes(k, N, 1, ndim) is not None and v[0] > 0}
        dom = max(bw_stages.items(), key=lambda kv: kv[1][0]) if bw_stages else None
        if dom:
            name, (t, n, byts) = dom
            bytes_pts = a.steps * N * F  # points of every call of the stage in the timed pass
            # one stage call per batched call: a sub-batch per call in batch mode,
            # a field per call in streams mode (a stage can launch several kernels)
            n = a.steps * (len(groups) if a.mode == "batch" else F)
            achieved = byts / (t / 1e3) / 1e9
            traffic = measured_traffic(a.workload, name, bytes_pts // n)
            roof = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1),
                    "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                    "traffic": traffic, "peak_source": "measured" if peaks else "fallback",
                    "bytes_per_launch": byts // n, "launch_ms": round(t / n, 5),
                    "timing": f"CUDA events around each stage call over a second timed pass of "
                              f"{a.steps} steps on one stream ({a.mode} mode); a launch here is "
                              f"one stage call over one batched call",
                    "step_ms_one_stream": round(ms1, 4)}

    # end to end through host buffers
    e2e = None
    if not a.no_e2e:
        h2d = [f.cpu().pin_memory() for f in fields]
        d2h = ([torch.empty(shape, dtype=torch.float32).pin_memory() for _ in range(F)],
               [torch.empty((len(g), fpsnr.STATS_BYTES), dtype=torch.uint8).pin_memory()
                for g in egroups]
               if a.mode == "batch" else
               [torch.empty(fpsnr.STATS_BYTES, dtype=torch.uint8).pin_memory() for _ in range(F)])
        step(S, h2d=h2d, d2h=d2h)
        if use_graph:
            run_step(S, True, h2d=h2d, d2h=d2h)
        ms_e, _ = timed(a.steps, S, graph=use_graph, h2d=h2d, d2h=d2h)
        e2e = {"value": round(aggregate_gbs(total_bytes, world, ms_e), 3), "unit": "GB/s",
               "h2d_bytes_per_step": total_bytes,
               "d2h_bytes_per_step": total_bytes + F * fpsnr.STATS_BYTES,
               "ms_per_step": round(ms_e, 4),
               "pipeline": f"{ne} sub-batches (cheap and dear targets alternating): inputs copied "
                           f"in pipeline order on one copy stream; each sub-batch compressed + "
                           f"decompressed on its own stream once its inputs are in, then its "
                           f"reconstructions and stats copied out on that stream"}

    cpu = None
    if pool is not None:
        hf = HostFields([f.cpu().numpy() for f in fields])
        try:
            runs = run_cpu_steps(pool, hf, tasks, psnrs, a.chunk, pool_workers, max(1, a.cpu_steps))
        finally:
            pool.close()
            hf.close()
        cpu = cpu_baseline_summary(a, runs, pool_workers, len(tasks))
        if a.workload != "c3":
            # whole fields: the oracle's PSNR and seconds beside the GPU's
            for _, _, tr in runs:
                for (f, _, _), _, (t, nbyt, p_or) in tr:
                    per_field[f]["oracle_psnr"] = round(p_or, 6)
                    per_field[f]["oracle_s"] = round(t, 3)

    served = None
    if rank == 0 and not a.no_serve_run:
        graphs.clear()
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
        served = served_short(dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": a.steps, "warmup": max(3, a.warmup), "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(workload_config(a, S),
                           **({"chunk": "autotuned per target",
                               "tuning": {str(k): {kk: v[kk] for kk in ("chunk", "pq_tile_x", "band_rows")}
                                          for k, v in tuning.items()}} if tuning else {})),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "served": served,
            "hbm_frac_of_step": round(value / (6775.6 if roof is None else roof["peak"]), 4),
            "psnr": {"mean_abs_dev_db": round(sum(dev_abs) / len(dev_abs), 4) if dev_abs else None,
                     "meet_rate": round(sum(meets) / len(meets), 4) if meets else None},
            "cr_mean": round(sum(crs) / len(crs), 3),
            "stages": stage_table, "per_field": per_field,
        }
        print(json.dumps(line), flush=True)
    for p in plans:
        p.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
